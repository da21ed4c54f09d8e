"""GPU parity of fused binarisation (object = byte > threshold, ccl_label_threshold and
ccl_label_batch_threshold) against the oracle's CCLRemSP of the binarised image, bit-exact
labels and K.  Section V binarises with im2bw(0.5), i.e. threshold 127 on 8-bit data."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _gpu import stream_handle

pytestmark = pytest.mark.gpu


def _run(img, t, conn=8, pitch=None, offset=0):
    import torch

    import paper_1606_05973_gb300 as ccl

    h, w = img.shape
    pitch = pitch or max(w, 1)
    buf = torch.full((offset + h * pitch + 16,), 255, dtype=torch.uint8, device="cuda")
    if h and w:
        buf[offset:offset + h * pitch].copy_(torch.from_numpy(synth.pad_pitch(img, pitch, 255).reshape(-1)))
    out = torch.full((h, w), -3, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(-1)
    rc = ccl.lib().ccl_label_threshold(ctypes.c_void_p(buf.data_ptr() + offset), h, w, pitch, conn, t,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(k), stream_handle())
    assert rc == 0, rc
    return out.cpu().numpy(), k.value


@pytest.mark.parametrize("t", [0, 1, 63, 127, 128, 200, 254, 255])
def test_random_bytes_every_threshold(t):
    img = np.random.default_rng(t + 1).integers(0, 256, size=(1000, 1500), dtype=np.uint8)
    ref, rk = oracle.cclremsp(oracle.binarize(img, t))
    lab, k = _run(img, t)
    assert k == rk and np.array_equal(lab, ref)


def test_threshold_zero_is_plain_labelling():
    import paper_1606_05973_gb300 as ccl
    import torch

    img = np.random.default_rng(5).integers(0, 4, size=(700, 900), dtype=np.uint8)
    lab, k = _run(img, 0)
    plain, pk = ccl.label(torch.from_numpy(img).cuda())
    assert k == pk and np.array_equal(lab, plain.cpu().numpy())


@pytest.mark.parametrize("h,w", [(1, 1), (3, 17), (63, 255), (65, 257), (130, 700), (7, 1000)])
def test_ragged_pitch_and_offset(h, w):
    img = np.random.default_rng(h * w).integers(0, 256, size=(h, w), dtype=np.uint8)
    ref, rk = oracle.cclremsp(oracle.binarize(img, 127))
    for pitch, off in [(w, 0), (((w + 15) // 16) * 16, 0), (w + 5, 3)]:
        lab, k = _run(img, 127, pitch=pitch, offset=off)
        assert k == rk and np.array_equal(lab, ref), (pitch, off)


def test_4_connectivity():
    img = np.random.default_rng(9).integers(0, 256, size=(900, 1100), dtype=np.uint8)
    for t in (100, 127):
        ref, rk = oracle.cclremsp(oracle.binarize(img, t), 4)
        lab, k = _run(img, t, conn=4)
        assert k == rk and np.array_equal(lab, ref)


def test_gray_field_8192():
    import torch

    import paper_1606_05973_gb300 as ccl

    g = synth.gray_field_device(8192, 8192, 4.0, 12, "cuda")
    host = g.cpu().numpy()
    ref, rk = oracle.cclremsp(oracle.binarize(host, 127))
    lab, k = ccl.label(g, threshold=127)
    assert k == rk
    got = lab.cpu().numpy()
    assert np.array_equal(got, ref), int((got != ref).sum())
    del g, lab
    torch.cuda.empty_cache()


def test_batch_threshold():
    import torch

    import paper_1606_05973_gb300 as ccl

    rng = np.random.default_rng(21)
    imgs = [rng.integers(0, 256, size=(int(rng.integers(1, 600)), int(rng.integers(1, 600))), dtype=np.uint8)
            for _ in range(30)]
    imgs.append(np.zeros((0, 5), np.uint8))
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    for t in (0, 127, 250):
        outs, ks = ccl.label_batch(dev, threshold=t)
        ks = ks.cpu().numpy()
        for i, (im, o) in enumerate(zip(imgs, outs)):
            ref, rk = oracle.cclremsp(oracle.binarize(im, t))
            assert ks[i] == rk and np.array_equal(o.cpu().numpy(), ref), (t, i)


def test_threshold_out_of_range_is_rejected():
    import paper_1606_05973_gb300 as ccl
    import torch

    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lab = torch.zeros(64, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(0)
    for t in (-1, 256):
        assert ccl.lib().ccl_label_threshold(buf.data_ptr(), 4, 4, 4, 8, t, lab.data_ptr(), ctypes.byref(k),
                                             stream_handle()) == 1
