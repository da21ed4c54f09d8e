"""GPU tests of the other entry points: batch, host buffers, asynchronous K, argument
errors, kernel timing and launch counts."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _gpu import run_label, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccl():
    import paper_1606_05973_gb300 as m

    return m


def test_batch_equals_single(ccl):
    import torch

    specs = synth.batch_specs(n=40, seed=100, lo=16, hi=700)
    imgs = [synth.make_batch_image(s) for s in specs]
    imgs.append(np.zeros((0, 5), np.uint8))
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ks = ccl.label_batch(dev)
    ks = ks.cpu().numpy()
    for im, o, k in zip(imgs, outs, ks):
        ref, rk = oracle.cclremsp(im)
        assert k == rk
        assert np.array_equal(o.cpu().numpy(), ref)


def test_host_buffers(ccl):
    import torch

    img = synth.bernoulli(1500, 2100, 0.55, 5)
    pinned = torch.from_numpy(img).pin_memory()
    out = torch.empty(img.shape, dtype=torch.int32).pin_memory()
    lab, k = ccl.label_host(pinned, out=out)
    ref, rk = oracle.cclremsp(img)
    assert k == rk and np.array_equal(lab.numpy(), ref)
    lab2, k2 = ccl.label_host(img)  # pageable numpy
    assert k2 == rk and np.array_equal(lab2, ref)


def test_async_count(ccl):
    import torch

    img = synth.bernoulli(999, 1234, 0.35, 6)
    lab, kd = ccl.label(torch.from_numpy(img).cuda(), sync=False)
    torch.cuda.synchronize()
    ref, rk = oracle.cclremsp(img)
    assert int(kd.item()) == rk and np.array_equal(lab.cpu().numpy(), ref)


def test_argument_errors(ccl):
    import torch

    lib = ccl.lib()
    s = stream_handle()
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lab = torch.zeros(64, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(0)
    assert lib.ccl_label(buf.data_ptr(), 4, 4, 4, 5, lab.data_ptr(), ctypes.byref(k), s) == 2
    assert lib.ccl_label(buf.data_ptr(), 4, 4, 3, 4, lab.data_ptr(), ctypes.byref(k), s) == 1
    assert lib.ccl_label(buf.data_ptr(), 4, 4, 4, 6, lab.data_ptr(), ctypes.byref(k), s) == 2
    assert lib.ccl_label(buf.data_ptr(), 4, 4, 3, 8, lab.data_ptr(), ctypes.byref(k), s) == 1
    assert lib.ccl_label(None, 4, 4, 4, 8, lab.data_ptr(), ctypes.byref(k), s) == 1
    assert lib.ccl_label(buf.data_ptr(), -1, 4, 4, 8, lab.data_ptr(), ctypes.byref(k), s) == 1
    assert lib.ccl_label(buf.data_ptr(), 1 << 16, 1 << 15, 1 << 15, 8, lab.data_ptr(), ctypes.byref(k), s) == 1


def test_profile_counts_launches(ccl):
    import torch

    img = torch.from_numpy(synth.bernoulli(512, 512, 0.5, 1)).cuda()

    def counts(mode):
        assert ccl.lib().ccl_set_launch_mode(mode) == 0
        try:
            ccl.ccl_profile_reset()
            ccl.ccl_profile_enable(1)
            ccl.label(img)
            ccl.label(img)
            ccl.ccl_profile_enable(0)
            return ccl.kernel_times()
        finally:
            ccl.lib().ccl_set_launch_mode(0)

    kt = counts(2)  # forced persistent launch: one launch per image
    assert kt["persistent"][0] == 2 and kt["tile_local"][0] == 0 and kt["persistent"][1] > 0.0
    kt = counts(1)  # three kernels per image
    assert kt["tile_local"][0] == 2 and kt["final_labels"][0] == 2 and kt["persistent"][0] == 0
    assert kt["final_labels"][1] > 0.0
    ccl.ccl_profile_reset()


def test_batch_uneven_with_empty_images_matches_single_calls(ccl):
    import torch

    specs = synth.batch_specs(n=120, seed=7, lo=1, hi=1500)
    imgs = [synth.make_batch_image(s) if s["h"] > 1 else np.zeros((s["h"], s["w"]), np.uint8) for s in specs]
    imgs[5] = np.zeros((0, 17), np.uint8)
    imgs[50] = np.zeros((9, 0), np.uint8)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ks = ccl.label_batch(dev)
    ks = ks.cpu().numpy()
    for i, (im, o, k) in enumerate(zip(imgs, outs, ks)):
        ref, rk = oracle.cclremsp(im)
        assert k == rk, i
        assert np.array_equal(o.cpu().numpy(), ref), i
        lab1, k1 = ccl.label(dev[i])
        assert k1 == rk and np.array_equal(lab1.cpu().numpy(), ref), i
    flags = ctypes.c_int32(0)
    assert ccl.lib().ccl_device_status(stream_handle(), ctypes.byref(flags)) == 0 and flags.value == 0


def test_batch_graph_replay(ccl):
    import torch

    specs = synth.batch_specs(n=30, seed=9, lo=32, hi=600)
    imgs = [synth.make_batch_image(s) for s in specs]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        outs, ks = ccl.label_batch(dev, stream=s)  # warm-up: sizes the workspace
        s.synchronize()
        for o in outs:
            o.fill_(-1)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            outs2, ks2 = ccl.label_batch(dev, outs=outs, stream=s)
        g.replay()
        s.synchronize()
    for im, o, k in zip(imgs, outs2, ks2.cpu().numpy()):
        ref, rk = oracle.cclremsp(im)
        assert k == rk and np.array_equal(o.cpu().numpy(), ref)


def test_host_async_two_streams():
    import torch

    imgs = [synth.bernoulli(900 + 37 * i, 1300 - 41 * i, 0.4 + 0.05 * i, 30 + i) for i in range(5)]
    pinned = [torch.from_numpy(im).pin_memory() for im in imgs]
    outs = [torch.full(im.shape, -1, dtype=torch.int32).pin_memory() for im in imgs]
    ks = torch.full((len(imgs),), -1, dtype=torch.int32).pin_memory()
    streams = [torch.cuda.Stream() for _ in range(2)]
    lib = __import__("paper_1606_05973_gb300").lib()
    for i, (p, o) in enumerate(zip(pinned, outs)):
        H, W = p.shape
        rc = lib.ccl_label_host_async(p.data_ptr(), H, W, W, 8, o.data_ptr(),
                                      ctypes.c_void_p(ks.data_ptr() + 4 * i),
                                      ctypes.c_void_p(streams[i % 2].cuda_stream))
        assert rc == 0, rc
    for st in streams:
        st.synchronize()
    for i, im in enumerate(imgs):
        ref, rk = oracle.cclremsp(im)
        assert int(ks[i]) == rk and np.array_equal(outs[i].numpy(), ref), i


def test_global_ctas_per_sm_cap_and_two_streams(ccl):
    """With the global kernel capped at one CTA per SM (a grid of fewer CTAs than its
    work items and segments, so its loops wrap), images labelled on two streams at once
    match the oracle; a negative cap is rejected and the default is restored after."""
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_global_ctas_per_sm(-1) == 1
    imgs = [synth.bernoulli(3000, 4000, p, 40 + i) for i, p in enumerate((0.3, 0.5, 0.6, 0.7))]
    refs = [oracle.cclremsp(im) for im in imgs]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    try:
        for cap in (1, 0):
            assert lib.ccl_set_global_ctas_per_sm(cap) == 0
            outs = [torch.empty(im.shape, dtype=torch.int32, device="cuda") for im in imgs]
            kd = torch.zeros(len(imgs), dtype=torch.int32, device="cuda")
            for rep in range(3):
                for i, t in enumerate(dev):
                    st = streams[i % 2]
                    rc = lib.ccl_label_async(t.data_ptr(), t.shape[0], t.shape[1], t.stride(0), 8,
                                             outs[i].data_ptr(), ctypes.c_void_p(kd.data_ptr() + 4 * i),
                                             ctypes.c_void_p(st.cuda_stream))
                    assert rc == 0
            torch.cuda.synchronize()
            for (ref, rk), o, k in zip(refs, outs, kd.cpu().tolist()):
                assert k == rk and np.array_equal(o.cpu().numpy(), ref)
            flags = ctypes.c_int32(0)
            for st in streams:
                assert lib.ccl_device_status(ctypes.c_void_p(st.cuda_stream), ctypes.byref(flags)) == 0
                assert flags.value == 0
    finally:
        lib.ccl_set_global_ctas_per_sm(0)


def test_half_size_global_kernel_at_one_cta_per_sm(ccl):
    """At one CTA per SM the global kernel takes CTAs of 512 threads (each thread then walks
    twice the items and segments); labels under every mode it serves against the oracle:
    the three 8-connected tile shapes, 4-connectivity and classes, on a serpentine (one
    component whose parent chains need several pointer-jumping rounds) and dense noise."""
    import torch

    lib = ccl.lib()
    imgs = [synth.serpentine(2000, 2600), synth.bernoulli(2500, 3100, 0.6, 51)]
    rng = np.random.default_rng(52)
    cls = rng.integers(0, 3, size=(1500, 2100), dtype=np.uint8)
    try:
        assert lib.ccl_set_global_ctas_per_sm(1) == 0
        for policy in (0, 2, 3):
            assert lib.ccl_set_tile_policy(policy) == 0
            for im in imgs:
                ref, rk = oracle.cclremsp(im)
                lab, k = ccl.label(torch.from_numpy(im).cuda())
                assert k == rk and np.array_equal(lab.cpu().numpy(), ref), (policy, im.shape)
        lib.ccl_set_tile_policy(0)
        for im in imgs:
            ref, rk = oracle.cclremsp(im, 4)
            lab, k = ccl.label(torch.from_numpy(im).cuda(), connectivity=4)
            assert k == rk and np.array_equal(lab.cpu().numpy(), ref), im.shape
        for conn in (8, 4):
            ref, rk = oracle.classes(cls, conn)
            lab, k = ccl.label(torch.from_numpy(cls).cuda(), connectivity=conn, classes=True)
            assert k == rk and np.array_equal(lab.cpu().numpy(), ref), conn
        flags = ctypes.c_int32(0)
        assert lib.ccl_device_status(stream_handle(), ctypes.byref(flags)) == 0 and flags.value == 0
    finally:
        lib.ccl_set_global_ctas_per_sm(0)
        lib.ccl_set_tile_policy(0)


def test_tile_policies_give_identical_labels(ccl):
    """The 8-connected path on 64 x 256 tiles (policy 1), 64 x 128 tiles (policy 2), 64 x 512
    tiles of 512 threads (policy 3) and the size rule (policy 0): single images on both sides
    of the size thresholds, ragged sizes and a padded pitch, and a batch, all equal to the
    oracle under every policy."""
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_tile_policy(4) == 1 and lib.ccl_set_tile_policy(-1) == 1
    singles = [synth.bernoulli(h, w, p, 60 + i) for i, (h, w, p) in
               enumerate(((1, 1, 1.0), (63, 129, 0.5), (700, 1000, 0.3), (1500, 2333, 0.6),
                          (3100, 3100, 0.45), (2000, 5000, 0.9), (1100, 12400, 0.55)))]
    singles.append(synth.serpentine(777, 3333))
    singles.append(synth.serpentine(12300, 12300))  # above the size rule's big-tile threshold
    specs = synth.batch_specs(n=24, seed=101, lo=16, hi=1500)
    batch = [synth.make_batch_image(s) for s in specs]
    refs = [oracle.cclremsp(im) for im in singles]
    brefs = [oracle.cclremsp(im) for im in batch]
    try:
        for policy in (1, 2, 3, 0):
            assert lib.ccl_set_tile_policy(policy) == 0
            for im, (ref, rk) in zip(singles, refs):
                lab, k = ccl.label(torch.from_numpy(im).cuda())
                assert k == rk and np.array_equal(lab.cpu().numpy(), ref), (policy, im.shape)
            rc, lab, k, flags = run_label(singles[3], pitch=singles[3].shape[1] + 48)
            assert rc == 0 and flags == 0 and k == refs[3][1] and np.array_equal(lab, refs[3][0])
            outs, ks = ccl.label_batch([torch.from_numpy(im).cuda() for im in batch])
            for o, kk, (ref, rk) in zip(outs, ks.cpu().tolist(), brefs):
                assert kk == rk and np.array_equal(o.cpu().numpy(), ref), policy
    finally:
        lib.ccl_set_tile_policy(0)
