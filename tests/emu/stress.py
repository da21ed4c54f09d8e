"""Stress run of the emulated GPU path against the oracle (run in a child process so that
the sanitizer runtime can be preloaded).  Exit code 0 = every case matched."""
import os
import sys

import numpy as np

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]

import oracle  # noqa: E402
import synth  # noqa: E402
from emu.emu import Emu  # noqa: E402


def main(path, n_random, sizes=None):
    emu = Emu(path)
    bad = 0
    imgs = []
    all_sizes = [(8, 64), (9, 65), (7, 63), (16, 128), (33, 97), (66, 300), (129, 257)]
    for h, w in (all_sizes if sizes is None else all_sizes[:sizes]):
        imgs += [synth.serpentine(h, w), synth.checkerboard(h, w), synth.dot_lattice(h, w),
                 synth.striped_rows(h, w), synth.blobs(h, w, 2.0, h + w), np.ones((h, w), np.uint8),
                 np.ascontiguousarray(synth.serpentine(w, h).T)]
        for p in (0.2, 0.41, 0.6, 0.8):
            imgs.append(synth.bernoulli(h, w, p, int(p * 1000) + h))
    for i, img in enumerate(imgs):
        for conn, small, large in ((8, (1, 2), (0, 3, 4)), (4, (6, 7, 8), (5,))):
            ref, rk = oracle.cclremsp(img, conn)
            # small tiles (one or two warps) for every pattern; the 256-thread tile shapes
            # on every sixth pattern only, to keep the run short
            shapes = small + large if i % 6 == 0 else small
            for shape in shapes:
                for seed in range(2 if shape in small else 1):
                    pitch = None if seed == 0 else img.shape[1] + 3 + (i % 16)
                    lab, k, st = emu.label(img, seed=i * 7 + seed, shape=shape, pitch=pitch)
                    if not (k == rk and st == 0 and np.array_equal(lab, ref)):
                        bad += 1
                        print("mismatch", conn, img.shape, shape, seed, k, rk, st)
    # multi-class images (0 = background, 1..n classes): single images and batches
    crng = np.random.default_rng(17)
    for i, (h, w) in enumerate(all_sizes if sizes is None else all_sizes[:sizes]):
        for ncls in (1, 2, 3, 9):
            img = crng.integers(0, ncls + 1, size=(h, w), dtype=np.uint8)
            for conn, small, large in ((8, (9, 10), (11,)), (4, (12,), (13,))):
                ref, rk = oracle.classes(img, conn)
                for shape in small + (large if i % 3 == 0 else ()):
                    pitch = None if ncls % 2 else w + 5
                    lab, k, st = emu.label(img, seed=i * 11 + ncls, shape=shape, pitch=pitch)
                    if not (k == rk and st == 0 and np.array_equal(lab, ref)):
                        bad += 1
                        print("classes mismatch", conn, img.shape, ncls, shape, k, rk, st)
    for trial in range(4):
        batch = [crng.integers(0, 4, size=(int(crng.integers(1, 40)), int(crng.integers(1, 150))), dtype=np.uint8)
                 for _ in range(int(crng.integers(1, 6)))]
        shape, conn = ((9, 8), (12, 4))[trial % 2]
        labs, ks, st = emu.label_batch(batch, seed=trial, shape=shape)
        for img, lab, kk in zip(batch, labs, ks):
            ref, rk = oracle.classes(img, conn)
            if not (kk == rk and st == 0 and np.array_equal(lab, ref)):
                bad += 1
                print("classes batch mismatch", img.shape, kk, rk, st)
    rng = np.random.default_rng(5)
    for i in range(n_random):
        h = int(rng.integers(1, 20))
        w = int(rng.integers(1, 140))
        img = (rng.random((h, w)) < rng.uniform(0.15, 0.9)).astype(np.uint8)
        conn = 8 if i % 2 == 0 else 4
        ref, rk = oracle.cclremsp(img, conn)
        shape = (1, 2)[(i // 2) % 2] if conn == 8 else (6, 7, 8)[(i // 2) % 3]
        lab, k, st = emu.label(img, seed=i, shape=shape)
        if not (k == rk and st == 0 and np.array_equal(lab, ref)):
            bad += 1
            print("random mismatch", conn, shape, h, w, k, rk, st)
    # batches of uneven images (the batched kernels), every image checked on its own
    for trial in range(8):
        k = int(rng.integers(1, 7))
        batch = []
        for _ in range(k):
            h = int(rng.integers(1, 40))
            w = int(rng.integers(1, 150))
            batch.append((rng.random((h, w)) < rng.uniform(0.1, 0.9)).astype(np.uint8))
        shape, conn = ((1, 8), (2, 8), (6, 4), (7, 4))[trial % 4]
        labs, ks, st = emu.label_batch(batch, seed=trial, shape=shape)
        for img, lab, kk in zip(batch, labs, ks):
            ref, rk = oracle.cclremsp(img, conn)
            if not (kk == rk and st == 0 and np.array_equal(lab, ref)):
                bad += 1
                print("batch mismatch", img.shape, kk, rk, st)
    for img in (np.zeros((0, 3), np.uint8), np.zeros((3, 0), np.uint8)):
        lab, k, st = emu.label(img)
        if k != 0:
            bad += 1
    print("bad", bad)
    return bad


if __name__ == "__main__":
    sizes = int(sys.argv[3]) if len(sys.argv) > 3 else None
    sys.exit(1 if main(sys.argv[1], int(sys.argv[2]), sizes) else 0)
