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
    for shape in (0, 1, 2):
        lab, k, st = e.label(img, seed=shape, shape=shape)
        assert st == 0 and k == rk and np.array_equal(lab, ref)
