"""GPU parity on the full-size workloads, in the launch configuration the benchmark uses
(one ccl_label call per image on the current stream):

* 8192 x 8192: Bernoulli p in {0.1, 0.3, 0.5, 0.7, 0.9} (seeds 2..6) and a sigma=4
  thresholded Gaussian field (seed 7) - compared element by element with the oracle;
* 21568 x 21568 (~465 MB): sigma=16 blobs (seed 8), Bernoulli(0.6) (seed 9) and the
  serpentine - compared element by element with the oracle as well (it labels 465 M
  pixels in seconds).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _label_dev(t):
    import paper_1606_05973_gb300 as ccl

    lab, k = ccl.label(t)
    return lab, k


def _check_full(img_np, t=None):
    import torch

    if t is None:
        t = torch.from_numpy(img_np).cuda()
    lab, k = _label_dev(t)
    ref, rk = oracle.cclremsp(img_np)
    assert k == rk, (k, rk)
    got = lab.cpu().numpy()
    assert np.array_equal(got, ref), int((got != ref).sum())


@pytest.mark.parametrize("kind,arg,seed", synth.SWEEP_8192)
def test_sweep_8192(kind, arg, seed):
    import torch

    if kind == "bernoulli":
        img = synth.bernoulli(8192, 8192, arg, seed)
        _check_full(img)
    else:
        t = synth.blobs_device(8192, 8192, arg, seed, "cuda")
        _check_full(t.cpu().numpy(), t)
    torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", ["blobs16", "bernoulli0.6", "serpentine"])
def test_465mb_image(variant):
    import torch

    side = 21568
    if variant == "blobs16":
        t = synth.blobs_device(side, side, 16.0, 8, "cuda")
        img = t.cpu().numpy()
    elif variant == "bernoulli0.6":
        img = synth.bernoulli(side, side, 0.6, 9)
        t = None
    else:
        img = synth.serpentine(side, side)
        t = None
    _check_full(img, t)
    del t
    torch.cuda.empty_cache()


def test_repeated_near_critical_blobs():
    """Thresholded Gaussian fields at density 0.5 are at the percolation threshold: giant
    tortuous components cross thousands of tile edges, so many boundary unions run on the
    same trees at once.  Before splices became compare-and-swaps of the parent read, about
    1% of these labellings lost a union (K + 1, one component split); 300 repetitions of
    each image would have shown it with high probability."""
    import torch

    import paper_1606_05973_gb300 as ccl

    images = [synth.batch_device([{"h": 8192, "w": 8192, "kind": "blobs", "p": 0.5, "sigma": 2.0,
                                   "seed": 991}], "cuda")[0],
              synth.blobs_device(8192, 8192, 4.0, 7, "cuda")]
    for t in images:
        ref, rk = oracle.cclremsp(t.cpu().numpy())
        ref = torch.from_numpy(ref).cuda()
        out = torch.empty_like(ref)
        bad = 0
        for _ in range(300):
            _, k = ccl.label(t, out=out)
            if k != rk or not torch.equal(out, ref):
                bad += 1
        assert bad == 0, bad
        del ref, out
        torch.cuda.empty_cache()
