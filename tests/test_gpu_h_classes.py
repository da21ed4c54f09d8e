"""GPU parity of multi-class labelling (ccl_label_classes, ccl_label_batch_classes):
neighbours connect when their bytes are equal and non-zero.  Compared element by element
with the oracle's flood fill (oracle.classes); labels are integers, so the bar is
equality of every label and of K."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _gpu import stream_handle

pytestmark = pytest.mark.gpu


def _run(img, conn=8, pitch=None, offset=0, lib=None):
    import torch

    import paper_1606_05973_gb300 as ccl

    lib = lib or ccl.lib()
    h, w = img.shape
    pitch = pitch or max(w, 1)
    buf = torch.full((offset + h * pitch + 16,), 77, dtype=torch.uint8, device="cuda")
    if h and w:
        buf[offset:offset + h * pitch].copy_(torch.from_numpy(synth.pad_pitch(img, pitch, 77).reshape(-1)))
    out = torch.full((h, w), -3, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(-1)
    rc = lib.ccl_label_classes(ctypes.c_void_p(buf.data_ptr() + offset), h, w, pitch, conn,
                               ctypes.c_void_p(out.data_ptr()), ctypes.byref(k), stream_handle())
    assert rc == 0, rc
    flags = ctypes.c_int32(0)
    lib.ccl_device_status(stream_handle(), ctypes.byref(flags))
    assert flags.value == 0, flags.value
    return out.cpu().numpy(), k.value


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("ncls", [1, 2, 3, 7, 255])
def test_random_classes(conn, ncls):
    rng = np.random.default_rng(ncls * 31 + conn)
    for h, w in [(1, 1), (1, 300), (300, 1), (31, 255), (33, 257), (97, 770), (500, 600)]:
        img = rng.integers(0, ncls + 1, size=(h, w), dtype=np.uint8)
        ref, rk = oracle.classes(img, conn)
        lab, k = _run(img, conn)
        assert k == rk and np.array_equal(lab, ref), (h, w)


def test_checked_build_and_pitch():
    import paper_1606_05973_gb300 as ccl

    dbg = ccl.load(debug=True)
    rng = np.random.default_rng(4)
    img = rng.integers(0, 4, size=(130, 700), dtype=np.uint8)
    for conn in (8, 4):
        ref, rk = oracle.classes(img, conn)
        for pitch, off in [(700, 0), (704, 0), (705, 3)]:
            lab, k = _run(img, conn, pitch=pitch, offset=off, lib=dbg)
            assert k == rk and np.array_equal(lab, ref), (conn, pitch, off)


def test_one_class_equals_binary():
    import torch

    import paper_1606_05973_gb300 as ccl

    img = synth.bernoulli(1000, 1200, 0.55, 3) * 5
    lab, k = _run(img)
    b, bk = ccl.label(torch.from_numpy(img).cuda())
    assert k == bk and np.array_equal(lab, b.cpu().numpy())


def test_land_cover_8192():
    import torch

    import paper_1606_05973_gb300 as ccl

    for conn in (8, 4):
        c = synth.classes_device(8192, 8192, 4.0, 8, 15, "cuda")
        ref, rk = oracle.classes(c.cpu().numpy(), conn)
        lab, k = ccl.label(c, connectivity=conn, classes=True)
        assert k == rk
        got = lab.cpu().numpy()
        assert np.array_equal(got, ref), int((got != ref).sum())
        del c, lab
        torch.cuda.empty_cache()


def test_batch_classes():
    import torch

    import paper_1606_05973_gb300 as ccl

    rng = np.random.default_rng(8)
    imgs = [rng.integers(0, 5, size=(int(rng.integers(1, 500)), int(rng.integers(1, 500))), dtype=np.uint8)
            for _ in range(25)]
    imgs.append(np.zeros((0, 3), np.uint8))
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    for conn in (8, 4):
        outs, ks = ccl.label_batch(dev, connectivity=conn, classes=True)
        ks = ks.cpu().numpy()
        for i, (im, o) in enumerate(zip(imgs, outs)):
            ref, rk = oracle.classes(im, conn)
            assert ks[i] == rk and np.array_equal(o.cpu().numpy(), ref), (conn, i)
