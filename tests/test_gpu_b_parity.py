"""GPU parity against the CPU oracle, element by element, through the C ABI (release
build).  Labels are integers, so the bar is bit-exact equality, plus K and a clean
device status word."""
import numpy as np
import pytest

import oracle
import synth
from _defs import check_invariants, closed_forms, load_golden
from _gpu import mosaic_4x4_all, run_label

pytestmark = pytest.mark.gpu


def _same(img, **kw):
    ref, rk = oracle.cclremsp(img)
    rc, lab, k, flags = run_label(img, **kw)
    assert rc == 0 and flags == 0, (rc, flags)
    assert k == rk, (k, rk)
    assert np.array_equal(lab, ref), int((lab != ref).sum())
    return lab, k


def test_config_1024_bernoulli_half():
    """1024 x 1024, Bernoulli(0.5), seed 1, 8-connectivity: the small configuration."""
    img = synth.bernoulli(1024, 1024, 0.5, 1)
    lab, k = _same(img)
    assert check_invariants(img, lab, k, 8) == []


def test_every_4x4_image_in_one_mosaic():
    _same(mosaic_4x4_all())


def test_golden_fixtures():
    for g in load_golden():
        rc, lab, k, flags = run_label(g["image"])
        assert rc == 0 and flags == 0
        assert k == g["k8"] and np.array_equal(lab, g["labels8"]), g["name"]


def test_closed_forms():
    for name, img, conn, ek, exp in closed_forms():
        if conn != 8:
            continue
        rc, lab, k, flags = run_label(img)
        assert rc == 0 and flags == 0
        assert k == ek and np.array_equal(lab, exp), name


@pytest.mark.parametrize("h", [1, 2, 3, 62, 63, 64, 65, 66, 127, 129, 191, 257])
@pytest.mark.parametrize("w", [1, 5, 31, 33, 255, 256, 257, 511, 513, 771])
def test_ragged_shapes(h, w):
    for p in (0.2, 0.5, 0.75):
        _same(synth.bernoulli(h, w, p, h * 7919 + w * 31 + int(p * 10)))


@pytest.mark.parametrize("sigma", [1.0, 2.0, 8.0, 32.0])
def test_blobs(sigma):
    _same(synth.blobs(777, 1500, sigma, int(sigma * 3)))


def test_long_chains():
    for h, w in [(1024, 1024), (2049, 777), (130, 4097)]:
        _same(synth.serpentine(h, w))
        _same(np.ascontiguousarray(synth.serpentine(w, h).T))


def test_non_binary_bytes_are_object():
    img = synth.bernoulli(300, 500, 0.5, 3)
    vals = np.random.default_rng(3).integers(1, 256, size=img.shape).astype(np.uint8)
    _same(img * vals)


def test_pitch_offsets_and_unaligned_labels():
    img = synth.bernoulli(333, 1000, 0.6, 12)
    for pitch, off, loff in [(1000, 0, 0), (1008, 0, 0), (1024, 16, 0), (1001, 1, 0), (1000, 0, 1),
                             (1040, 3, 3)]:
        _same(img, pitch=pitch, offset=off, label_offset=loff)


def test_repeat_runs_identical():
    img = synth.bernoulli(2000, 3000, 0.6, 21)
    outs = [run_label(img)[1] for _ in range(4)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_empty_images():
    for h, w in [(0, 0), (0, 10), (10, 0)]:
        rc, lab, k, flags = run_label(np.zeros((h, w), np.uint8))
        assert rc == 0 and k == 0


def test_all_background_and_all_object():
    _same(np.zeros((700, 900), np.uint8))
    _same(np.ones((700, 900), np.uint8))
