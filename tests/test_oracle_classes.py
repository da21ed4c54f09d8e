"""Pins of the multi-class oracle (neighbours connect when their bytes are equal and
non-zero) by routes that share none of its code: each class's binary mask labelled by
CCLRemSP, merged and renumbered by first pixel; scipy's labelling per class; closed forms;
and the reduction to binary labelling when one class is present."""
import numpy as np
import pytest

import oracle
from _defs import first_occurrence


def _by_class_masks(img, conn):
    """Label every class separately with CCLRemSP, give each component a distinct id, then
    renumber all components by their first pixel in raster order."""
    out = np.zeros(img.shape, np.int64)
    base = 0
    for c in np.unique(img):
        if c == 0:
            continue
        lab, k = oracle.cclremsp((img == c).astype(np.uint8), conn)
        out[lab > 0] = lab[lab > 0] + base
        base += k
    return first_occurrence(out)[0], base


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("ncls", [2, 3, 7])
def test_matches_per_class_labelling(conn, ncls):
    rng = np.random.default_rng(ncls * 10 + conn)
    for h, w in [(1, 1), (1, 40), (40, 1), (17, 23), (64, 65), (130, 257)]:
        img = rng.integers(0, ncls + 1, size=(h, w), dtype=np.uint8)
        lab, k = oracle.classes(img, conn)
        ref, rk = _by_class_masks(img, conn)
        assert k == rk and np.array_equal(lab, ref), (h, w)


def test_matches_scipy_per_class():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    img = rng.integers(0, 5, size=(90, 110), dtype=np.uint8)
    lab, k = oracle.classes(img, 8)
    out = np.zeros(img.shape, np.int64)
    base = 0
    for c in range(1, 5):
        l, n = ndimage.label(img == c, structure=np.ones((3, 3), int))
        out[l > 0] = l[l > 0] + base
        base += n
    assert k == base and np.array_equal(lab, first_occurrence(out)[0])


def test_one_class_is_binary_labelling():
    rng = np.random.default_rng(7)
    img = (rng.random((60, 70)) < 0.55).astype(np.uint8) * 9
    for conn in (8, 4):
        lab, k = oracle.classes(img, conn)
        ref, rk = oracle.cclremsp(img, conn)
        assert k == rk and np.array_equal(lab, ref)


def test_closed_forms():
    # vertical stripes of alternating classes 1, 2: every column its own component
    img = np.tile(np.array([1, 2], np.uint8), (5, 4))
    lab, k = oracle.classes(img, 8)
    assert k == 8 and np.array_equal(lab, np.tile(np.arange(1, 9, dtype=np.int32), (5, 1)))
    # a checkerboard of classes 1 and 2: 8-connected diagonals join equal classes
    y, x = np.indices((6, 6))
    cb = (1 + (y + x) % 2).astype(np.uint8)
    lab, k = oracle.classes(cb, 8)
    assert k == 2 and np.array_equal(lab, cb.astype(np.int32))
    lab4, k4 = oracle.classes(cb, 4)
    assert k4 == 36
