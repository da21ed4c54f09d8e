"""Pins the CPU oracle to references that are not the oracle itself.

* hand-derived fixtures under tests/golden (problem definition, Section III);
* closed forms (all-zero, all-one, checkerboard, dot lattice, striped rows, serpentine);
* every image of several tiny shapes against a pure-Python flood fill (the definition)
  and against scipy.ndimage.label (a library flood fill);
* random images of many shapes, densities and row pitches against scipy, plus the
  invariants that hold for any correct answer;
* agreement of the paper's three algorithms (CCLRemSP, ARemSP, PARemSP at several thread
  counts) with each other.
"""
import numpy as np
import pytest

import oracle
import synth
from _defs import bfs_py, check_invariants, scipy_labels
from _pins import _all_images, run_battery


def test_battery_passes():
    errs = run_battery(oracle.default())
    assert errs == [], errs[:10]


@pytest.mark.parametrize("shape", [(4, 4), (5, 3), (3, 5), (1, 16), (16, 1), (2, 8), (8, 2)])
def test_exhaustive_against_pure_python_flood_fill(shape):
    orc = oracle.default()
    h, w = shape
    for img in _all_images(h, w):
        for conn in (8, 4):
            ref, rk = bfs_py(img, conn)
            lab, k = orc.cclremsp(img, conn)
            assert k == rk and np.array_equal(lab, ref), (img.tolist(), conn)
        lab, k = orc.aremsp(img)
        ref, rk = bfs_py(img, 8)
        assert k == rk and np.array_equal(lab, ref), img.tolist()


@pytest.mark.parametrize("h,w", [(1001, 777), (512, 2048), (999, 1), (1, 999), (3, 4097)])
@pytest.mark.parametrize("p", [0.1, 0.41, 0.5, 0.7, 0.95])
def test_paper_algorithms_agree(h, w, p):
    orc = oracle.default()
    img = synth.bernoulli(h, w, p, 31 + h + w)
    a, ka = orc.cclremsp(img)
    b, kb = orc.aremsp(img)
    assert ka == kb and np.array_equal(a, b)
    for t in (1, 2, 3, 7, 8, 16):
        c, kc = orc.paremsp(img, t)
        assert kc == ka and np.array_equal(a, c), t
    d, kd = orc.bfs(img)
    assert kd == ka and np.array_equal(a, d)
    assert check_invariants(img, a, ka, 8) == []


@pytest.mark.parametrize("sigma", [2.0, 4.0, 16.0])
def test_blobs_against_scipy(sigma):
    img = synth.blobs(700, 900, sigma, 5)
    for conn in (8, 4):
        ref, rk = scipy_labels(img, conn)
        lab, k = oracle.cclremsp(img, conn)
        assert k == rk and np.array_equal(lab, ref)
    lab, k = oracle.paremsp(img, 5)
    assert np.array_equal(lab, scipy_labels(img, 8)[0])


def test_invariants_large():
    img = synth.bernoulli(2048, 2048, 0.45, 77)
    lab, k = oracle.cclremsp(img)
    assert check_invariants(img, lab, k, 8) == []
    ref, rk = scipy_labels(img, 8)
    assert rk == k and np.array_equal(ref, lab)


def test_unnormalised_flatten_order_differs_for_two_row_scan():
    """ARemSP without renumbering numbers components by first provisional label, which is
    column-pair order; a component starting at (1,0) comes before one starting at (0,5)."""
    img = np.zeros((2, 8), np.uint8)
    img[0, 5] = 1
    img[1, 0] = 1
    raw, k = oracle.aremsp(img, remap=False)
    assert k == 2 and raw[1, 0] == 1 and raw[0, 5] == 2
    canon, k = oracle.aremsp(img)
    assert canon[0, 5] == 1 and canon[1, 0] == 2


def test_empty_and_bad_arguments():
    lab, k = oracle.cclremsp(np.zeros((0, 5), np.uint8))
    assert k == 0 and lab.shape == (0, 5)
    lab, k = oracle.paremsp(np.zeros((3, 0), np.uint8), 4)
    assert k == 0
    with pytest.raises(RuntimeError):
        oracle.default().cclremsp(np.ones((2, 2), np.uint8), conn=6)
