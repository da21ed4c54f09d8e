"""Per-phase cycle shares of the three kernels (a profiling tool).

    python -m paper_1606_05973_gb300.phase_timing

Builds ``_build/libccl_phase_timing.so``: the same kernels compiled with
CCL_PHASE_TIMING, where thread 0 of every CTA adds the clock64 cycles between the phase
barriers to per-phase sums (csrc/ccl_phase_timing.cu).  It then labels the 8192 x 8192
sweep images and the three 21568 x 21568 images (two warm-up calls, then three timed
calls each, one stream, the library's default grid) and prints, per image and kernel,
each phase's share of the summed CTA cycles.  The timing build does all the work of the
normal one; the ticks add a few instructions per phase.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PHASES = {
    "tile": ["load", "bits+runs", "unions", "roots", "mark", "prefix", "outputs"],
    "global": ["merge", "round0+count", "cta-sum scan", "labels+rounds"],
    "final": ["load bits", "runs", "run labels", "write"],
}


def build_timed() -> str:
    import importlib

    b = importlib.import_module("paper_1606_05973_gb300.build")
    os.makedirs(b.OUT, exist_ok=True)
    b.write_tuning_include()
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", b.OUT, *b.ARCH,
             "-DCCL_PHASE_TIMING"]
    objs = []
    for src in b.SOURCES:
        path = os.path.join(b.CSRC, "ccl_phase_timing.cu" if src == "ccl_kernels.cu" else src)
        obj = os.path.join(b.OUT, f"{os.path.splitext(src)[0]}.timing.o")
        subprocess.run([b.nvcc(), *flags, "-c", path, "-o", obj], check=True)
        objs.append(obj)
    target = os.path.join(b.OUT, "libccl_phase_timing.so")
    subprocess.run([b.nvcc(), "-shared", *b.ARCH, "-o", target, *objs, "-lcudart"], check=True)
    return target


def main():
    import numpy as np
    import torch

    import paper_1606_05973_gb300 as ccl
    import synth

    lib = ccl.load(path=build_timed())
    lib.ccl_phase_read.argtypes = [ctypes.c_void_p]
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    st = torch.cuda.Stream(device=dev)
    sp = ctypes.c_void_p(st.cuda_stream)
    kd = torch.zeros(1, dtype=torch.int32, device=dev)

    def run(name, img):
        H, W = img.shape
        lab = torch.empty((H, W), dtype=torch.int32, device=dev)

        def call():
            rc = lib.ccl_label_async(img.data_ptr(), H, W, img.stride(0), 8, lab.data_ptr(),
                                     ctypes.c_void_p(kd.data_ptr()), sp)
            if rc != 0:
                raise RuntimeError(f"ccl_label_async: {rc}")

        for _ in range(2):
            call()
        torch.cuda.synchronize()
        lib.ccl_phase_reset()
        n = 3
        for _ in range(n):
            call()
        torch.cuda.synchronize()
        buf = (ctypes.c_ulonglong * 48)()
        lib.ccl_phase_read(buf)
        t = np.array(buf[:], dtype=np.float64).reshape(3, 16)
        out = {}
        for k, kern in enumerate(PHASES):
            tot = t[k].sum()
            out[kern] = {p: round(t[k][i] / tot, 3) for i, p in enumerate(PHASES[kern])}
            out[kern]["Mcycles_per_launch"] = round(tot / n / 1e6, 2)
        print(name, json.dumps(out), flush=True)

    for side in (256, 1024):
        run(f"{side} bernoulli p=0.5", torch.from_numpy(synth.bernoulli(side, side, 0.5, 1)).to(dev))
    for kind, arg, seed in synth.SWEEP_8192:
        if kind == "bernoulli":
            run(f"8192 bernoulli p={arg}", torch.from_numpy(synth.bernoulli(8192, 8192, arg, seed)).to(dev))
        else:
            run(f"8192 blobs sigma={arg:g}", synth.blobs_device(8192, 8192, arg, seed, dev))
    s = 21568
    run("21568 blobs sigma=16", synth.blobs_device(s, s, 16.0, 8, dev))
    run("21568 bernoulli p=0.6", torch.from_numpy(synth.bernoulli(s, s, 0.6, 9)).to(dev))
    run("21568 serpentine", torch.from_numpy(synth.serpentine(s, s)).to(dev))


if __name__ == "__main__":
    main()
