"""GPU parity under 4-connectivity (edge neighbours only), through every entry point,
against the oracle's CCLRemSP run with 4-connectivity.  Labels are integers: the bar is
bit-exact equality, plus K and a clean device status word.

The GPU path runs the same passes as under 8-connectivity with one-row strips (a strip
run is a run of one row) and 32 x 256 tiles; a run joins the runs of the row above that
share a column with it, and across a tile edge only the pixel straight across counts."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _defs import check_invariants, closed_forms, load_golden
from _gpu import mosaic_4x4_all, run_label, stream_handle

pytestmark = pytest.mark.gpu


def _same(img, **kw):
    ref, rk = oracle.cclremsp(img, 4)
    rc, lab, k, flags = run_label(img, conn=4, **kw)
    assert rc == 0 and flags == 0, (rc, flags)
    assert k == rk, (k, rk)
    assert np.array_equal(lab, ref), int((lab != ref).sum())
    return lab, k


def test_1024_bernoulli_half():
    img = synth.bernoulli(1024, 1024, 0.5, 1)
    lab, k = _same(img)
    assert check_invariants(img, lab, k, 4) == []


def test_every_4x4_image_in_one_mosaic():
    _same(mosaic_4x4_all())


def test_golden_fixtures():
    for g in load_golden():
        rc, lab, k, flags = run_label(g["image"], conn=4)
        assert rc == 0 and flags == 0
        assert k == g["k4"] and np.array_equal(lab, g["labels4"]), g["name"]


def test_closed_forms():
    n = 0
    for name, img, conn, ek, exp in closed_forms():
        if conn != 4:
            continue
        rc, lab, k, flags = run_label(img, conn=4)
        assert rc == 0 and flags == 0
        assert k == ek and (exp is None or np.array_equal(lab, exp)), name
        n += 1
    assert n > 20


@pytest.mark.parametrize("h", [1, 2, 3, 31, 32, 33, 63, 65, 129])
@pytest.mark.parametrize("w", [1, 5, 31, 33, 255, 256, 257, 513])
def test_ragged_shapes(h, w):
    for p in (0.3, 0.59, 0.75):
        _same(synth.bernoulli(h, w, p, h * 7919 + w * 31 + int(p * 100)))


@pytest.mark.parametrize("sigma", [1.0, 4.0, 16.0])
def test_blobs(sigma):
    _same(synth.blobs(777, 1500, sigma, int(sigma * 5)))


def test_long_chains_and_diagonals():
    for h, w in [(1024, 1024), (2049, 777), (130, 4097)]:
        _same(synth.serpentine(h, w))
        _same(np.ascontiguousarray(synth.serpentine(w, h).T))
    # a diagonal staircase of 2-pixel steps is one component under 4-connectivity and
    # crosses every tile corner
    n = 1500
    st = np.zeros((n, n), np.uint8)
    i = np.arange(n)
    st[i, i] = 1
    st[i[:-1], i[:-1] + 1] = 1
    _same(st)
    _same(np.eye(700, 900, dtype=np.uint8))
    _same(synth.checkerboard(600, 700))


def test_pitch_offsets_and_unaligned_labels():
    img = synth.bernoulli(333, 1000, 0.6, 12)
    for pitch, off, loff in [(1000, 0, 0), (1024, 16, 0), (1001, 1, 0), (1040, 3, 3)]:
        _same(img, pitch=pitch, offset=off, label_offset=loff)


def test_8192_bernoulli_threshold_and_blobs():
    import torch

    import paper_1606_05973_gb300 as ccl

    for img in (synth.bernoulli(8192, 8192, 0.59, 31), None):
        if img is None:
            t = synth.blobs_device(8192, 8192, 4.0, 32, "cuda")
            img = t.cpu().numpy()
        else:
            t = torch.from_numpy(img).cuda()
        lab, k = ccl.label(t, connectivity=4)
        ref, rk = oracle.cclremsp(img, 4)
        assert k == rk
        got = lab.cpu().numpy()
        assert np.array_equal(got, ref), int((got != ref).sum())
        del t, lab
        torch.cuda.empty_cache()


def test_batch_host_async_and_static():
    import torch

    import paper_1606_05973_gb300 as ccl

    specs = synth.batch_specs(n=40, seed=41, lo=1, hi=900)
    imgs = [synth.make_batch_image(s) if s["h"] > 1 else np.zeros((s["h"], s["w"]), np.uint8) for s in specs]
    imgs[3] = np.zeros((0, 9), np.uint8)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ks = ccl.label_batch(dev, connectivity=4)
    ks = ks.cpu().numpy()
    for i, (im, o, k) in enumerate(zip(imgs, outs, ks)):
        ref, rk = oracle.cclremsp(im, 4)
        assert k == rk, i
        assert np.array_equal(o.cpu().numpy(), ref), i

    img = synth.bernoulli(1500, 2100, 0.6, 42)
    ref, rk = oracle.cclremsp(img, 4)
    lab, k = ccl.label_host(img, connectivity=4)
    assert k == rk and np.array_equal(lab, ref)
    lab, kd = ccl.label(torch.from_numpy(img).cuda(), connectivity=4, sync=False)
    torch.cuda.synchronize()
    assert int(kd.item()) == rk and np.array_equal(lab.cpu().numpy(), ref)

    small = synth.bernoulli(700, 900, 0.6, 43)
    ref, rk = oracle.cclremsp(small, 4)
    d = torch.from_numpy(small).cuda()
    out = torch.full(small.shape, -1, dtype=torch.int32, device="cuda")
    k_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = ccl.lib().ccl_label_static(d.data_ptr(), 700, 900, 900, 4, out.data_ptr(), k_dev.data_ptr(),
                                    stream_handle())
    assert rc == 0
    torch.cuda.synchronize()
    assert int(k_dev.item()) == rk and np.array_equal(out.cpu().numpy(), ref)
    flags = ctypes.c_int32(0)
    assert ccl.lib().ccl_device_status(stream_handle(), ctypes.byref(flags)) == 0 and flags.value == 0


def test_server_with_4_connectivity():
    import torch

    import paper_1606_05973_gb300 as ccl

    specs = synth.batch_specs(n=24, seed=44, lo=8, hi=1000)
    imgs = [synth.make_batch_image(s) for s in specs]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full(tuple(t.shape), -1, dtype=torch.int32, device="cuda") for t in dev]
    with ccl.Server(mem_cap_bytes=1 << 30, lanes=2, max_batch=8, connectivity=4) as srv:
        ids = [srv.submit(t, o) for t, o in zip(dev, outs)]
        ks = [srv.wait(r, timeout_ms=60000) for r in ids]
    torch.cuda.synchronize()
    for im, o, k in zip(imgs, outs, ks):
        ref, rk = oracle.cclremsp(im, 4)
        assert k == rk and np.array_equal(o.cpu().numpy(), ref)
