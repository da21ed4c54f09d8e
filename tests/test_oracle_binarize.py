"""Pins of the oracle's binarisation for fused thresholding: object = byte > threshold.
Section V binarises with im2bw(0.5), which on 8-bit data keeps bytes above 127.5."""
import numpy as np

import oracle


def test_binarize_special_cases():
    vals = np.arange(256, dtype=np.uint8).reshape(16, 16)
    assert np.array_equal(oracle.binarize(vals, 0), (vals != 0).astype(np.uint8))
    assert not oracle.binarize(vals, 255).any()
    assert np.array_equal(oracle.binarize(vals, 127), (vals >= 128).astype(np.uint8))
    assert oracle.binarize(vals, 127).sum() == 128
    for t in (1, 63, 200, 254):
        assert oracle.binarize(vals, t).sum() == 255 - t


def test_threshold_labels_by_flood_fill():
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=(40, 53), dtype=np.uint8)
    for t in (0, 50, 127, 220):
        b = oracle.binarize(img, t)
        lab, k = oracle.cclremsp(b)
        ref, rk = oracle.bfs(b)
        assert k == rk and np.array_equal(lab, ref)
