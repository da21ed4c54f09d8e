"""Runs the GPU path's tile phases on the CPU (tests/emu) against the oracle.

The emulator compiles the same kernel bodies (ccl_core.cuh) the CUDA kernels run, with one
OS thread per CUDA thread (barriers for __syncthreads, exchange slots for warp shuffles,
host atomics), poisons shared memory and workspace before use, and enables the
checked-index build.  With AddressSanitizer preloaded, any
out-of-range access or read of unwritten memory in the kernels' arithmetic fails here,
on the CPU, instead of on a GPU.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _stress(sanitize, n_random, sizes=None):
    sys.path.insert(0, HERE)
    from emu import emu

    rt = emu.asan_runtime() if sanitize else None
    so = emu.build(sanitize=rt is not None)
    env = dict(os.environ)
    if rt:
        env["LD_PRELOAD"] = rt
        env["ASAN_OPTIONS"] = "detect_leaks=0"
    args = [sys.executable, os.path.join(HERE, "emu", "stress.py"), so, str(n_random)]
    if sizes is not None:
        args.append(str(sizes))
    r = subprocess.run(args, capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_emulated_path_matches_oracle():
    """Every pattern size, 400 random images and the batches, without the sanitizer."""
    _stress(False, 400)


def test_emulated_path_matches_oracle_under_sanitizers():
    """The same checks on the smaller sizes with AddressSanitizer preloaded."""
    _stress(True, 120, sizes=5)


def test_emulated_path_tile_variants_quick():
    sys.path.insert(0, HERE)
    import numpy as np

    import oracle
    import synth
    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    img = synth.bernoulli(300, 700, 0.5, 1)
    ref, rk = oracle.cclremsp(img)
    for shape in (0, 1, 2, 16):
        lab, k, st = e.label(img, seed=shape, shape=shape)
        assert st == 0 and k == rk and np.array_equal(lab, ref)
    for im in (synth.serpentine(130, 1100), synth.bernoulli(200, 1500, 0.6, 3)):  # big tiles, ragged
        ref, rk = oracle.cclremsp(im)
        lab, k, st = e.label(im, seed=5, shape=16)
        assert st == 0 and k == rk and np.array_equal(lab, ref)


@pytest.mark.parametrize("shape", [14, 15])
def test_emulated_sweep_tile_shapes(shape):
    """The extra 8-connected tile shapes of the offline tile-shape sweep (32 x 256 and
    64 x 128, the library's narrow tiles) against the oracle: densities across the
    percolation threshold, ragged sizes, a serpentine, a padded pitch, and (64 x 128) a
    batch."""
    sys.path.insert(0, HERE)
    import numpy as np

    import oracle
    import synth
    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    cases = [synth.bernoulli(h, w, p, s) for (h, w, p, s) in
             ((130, 300, 0.1, 1), (97, 517, 0.45, 2), (200, 260, 0.6, 3), (64, 128, 0.9, 4), (33, 777, 0.5, 5))]
    cases.append(synth.serpentine(150, 390))
    for i, img in enumerate(cases):
        ref, rk = oracle.cclremsp(img)
        for pitch in (None, img.shape[1] + 5):
            lab, k, st = e.label(img, seed=i, shape=shape, pitch=pitch)
            assert st == 0 and k == rk and np.array_equal(lab, ref), (shape, img.shape, pitch)
    if shape == 15:  # the library's narrow tiles also run the batched path
        batch = [synth.make_batch_image(sp) for sp in synth.batch_specs(n=6, seed=7, lo=16, hi=300)]
        labs, ks, st = e.label_batch(batch, seed=3, shape=15)
        assert st == 0
        for im, lab, k in zip(batch, labs, ks):
            ref, rk = oracle.cclremsp(im)
            assert k == rk and np.array_equal(lab, ref)


def test_object_test_of_the_load_phase_is_byte_greater_than_threshold():
    """The load phase turns 16 bytes into 16 object bits with word arithmetic (the carry of
    byte + (255 - T) out of its byte).  Checked against byte > T for every byte value and
    every threshold, each byte in every one of the 16 positions."""
    sys.path.insert(0, HERE)
    import numpy as np

    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    vals = np.arange(256, dtype=np.uint8)
    for t in range(256):
        for k in range(16):
            block = np.roll(vals.reshape(16, 16), k, axis=1)  # every value in every position
            for row in block:
                got = e.gt_mask16(row, t)
                exp = int(sum(1 << i for i in range(16) if int(row[i]) > t))
                assert got == exp, (t, row.tolist(), hex(got), hex(exp))


def test_emulated_threshold_labelling_matches_oracle():
    sys.path.insert(0, HERE)
    import numpy as np

    import oracle
    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    rng = np.random.default_rng(3)
    for h, w in [(9, 65), (33, 97), (66, 300)]:
        img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        for t in (0, 1, 100, 127, 200, 255):
            ref, rk = oracle.cclremsp(oracle.binarize(img, t))
            for shape in (1, 2, 0, 6):
                conn = 4 if shape == 6 else 8
                if conn == 4:
                    ref4, rk4 = oracle.cclremsp(oracle.binarize(img, t), 4)
                # a pitch of whole 16-byte chunks takes the vector loads, w + 3 the byte loop
                pitch = ((w + 15) // 16) * 16 + 16 if t % 2 == 0 else w + 3
                lab, k, st = e.label(img, seed=t, shape=shape, threshold=t, pitch=pitch)
                exp, ek = (ref4, rk4) if conn == 4 else (ref, rk)
                assert st == 0 and k == ek and np.array_equal(lab, exp), (h, w, t, shape)


def test_byte_equality_test_of_the_class_load():
    """The multi-class load compares 4 bytes at a time (a zero-byte test of a ^ b).  Checked
    for every pair of byte values in every byte position, with random other bytes."""
    sys.path.insert(0, HERE)
    import numpy as np

    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    rng = np.random.default_rng(2)
    vals = np.arange(256, dtype=np.uint32)
    for pos in range(4):
        for a in range(256):
            others_a = int(rng.integers(0, 1 << 32)) & ~(0xFF << (8 * pos))
            others_b = int(rng.integers(0, 1 << 32)) & ~(0xFF << (8 * pos))
            for b in vals[::17].tolist() + [a, (a + 1) & 255, a ^ 128]:
                wa = others_a | (a << (8 * pos))
                wb = others_b | (b << (8 * pos))
                got = e.lib.emu_eq_nibble(wa, wb)
                exp = sum(1 << i for i in range(4) if (wa >> (8 * i)) & 255 == (wb >> (8 * i)) & 255)
                assert got == exp, (pos, hex(wa), hex(wb), got, exp)


def test_emulated_persistent_path():
    """The persistent single-launch body (tile pass, global phases and final pass in one
    grid, tiles from counters, the density probe choosing between two tile shapes) against
    the oracle: single images (inline descriptor) and batches, both shapes, the probe's
    three classes, 4-connectivity and multi-class, two to five CTAs."""
    sys.path.insert(0, HERE)
    import numpy as np

    import oracle
    import synth
    from emu import emu

    e = emu.Emu(emu.build(sanitize=False))
    rng = np.random.Generator(np.random.PCG64(11))
    for trial in range(24):
        n = int(rng.integers(1, 5))
        imgs = []
        for i in range(n):
            h, w = int(rng.integers(1, 70)), int(rng.integers(1, 150))
            kind = int(rng.integers(0, 3))
            if kind == 0:
                imgs.append(synth.bernoulli(h, w, float(rng.uniform(0.05, 0.95)), trial * 10 + i))
            elif kind == 1:
                imgs.append(synth.serpentine(h, w))
            else:
                imgs.append(np.ones((h, w), np.uint8))
        pick = tuple(int(x) for x in rng.integers(0, 2, 3))
        probe = int(rng.choice([0, 4, 16]))
        ctas = int(rng.integers(2, 6))
        pair = int(rng.choice([0, 0, 1, 2, 3]))
        if pair == 3:
            imgs = [(im * rng.integers(1, 4, im.shape)).astype(np.uint8) for im in imgs]
        labs, ks, st = e.label_fused(imgs, seed=trial, pair=pair, pick=pick, lo=300, hi=700, probe=probe,
                                     ctas=ctas)
        assert st == 0, (trial, st)
        for im, lab, k in zip(imgs, labs, ks):
            if pair == 3:
                ref, rk = oracle.classes(im, 8)
            else:
                ref, rk = oracle.cclremsp(im, 4 if pair == 2 else 8)
            assert k == rk and np.array_equal(lab, ref), (trial, pair, im.shape)
