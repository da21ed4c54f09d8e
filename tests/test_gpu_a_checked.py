"""GPU parity with the bounds-checked build (CCL_DEBUG): every index that comes from data
is range-checked on the device (a bad one sets a status bit and the access is skipped),
so these small cases cannot fault even if the path had an indexing mistake.  They run
first; the status word must stay 0 and the labels must equal the oracle's."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from _gpu import run_label

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    import paper_1606_05973_gb300 as ccl

    return ccl.load(debug=True)


SHAPES = [(1, 1), (2, 3), (1, 300), (300, 1), (63, 255), (64, 256), (65, 257), (128, 513),
          (130, 700), (200, 31), (7, 1000)]


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("h,w", SHAPES)
def test_checked_random(dbg, h, w, conn):
    for p in (0.1, 0.45, 0.7, 0.95):
        img = synth.bernoulli(h, w, p, 1000 * h + w + int(100 * p))
        ref, rk = oracle.cclremsp(img, conn)
        rc, lab, k, flags = run_label(img, lib=dbg, conn=conn)
        assert rc == 0 and flags == 0, (rc, flags)
        assert k == rk and np.array_equal(lab, ref)


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("maker", ["serpentine", "checkerboard", "dot_lattice", "striped_rows"])
def test_checked_patterns(dbg, maker, conn):
    for h, w in [(64, 256), (129, 511), (200, 300)]:
        img = getattr(synth, maker)(h, w)
        ref, rk = oracle.cclremsp(img, conn)
        rc, lab, k, flags = run_label(img, lib=dbg, conn=conn)
        assert rc == 0 and flags == 0
        assert k == rk and np.array_equal(lab, ref)


def test_checked_pitch_and_alignment(dbg):
    img = synth.bernoulli(150, 333, 0.55, 9)
    ref, rk = oracle.cclremsp(img)
    for pitch, off, loff in itertools.product((333, 336, 350, 512), (0, 1, 16), (0, 1)):
        rc, lab, k, flags = run_label(img, lib=dbg, pitch=pitch, offset=off, label_offset=loff)
        assert rc == 0 and flags == 0
        assert k == rk and np.array_equal(lab, ref), (pitch, off, loff)
