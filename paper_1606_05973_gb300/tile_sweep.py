"""Offline tile-shape sweep (a tuning tool; the library compiles two shapes, picked by size).

    python -m paper_1606_05973_gb300.tile_sweep [--out PATH]

Builds the library once per tile shape TH x TW of the 8-connected path (compile-time
CCL_TILE_H / CCL_TILE_W; 256 threads per CTA) into ``_build/libccl_tile_<TH>x<TW>.so``,
each run with tile policy 1 (its own TH x TW at every size).
Each build then labels the same images: size classes from 128^2 to 8192^2, with Bernoulli
p in {0.1, 0.5, 0.9}, sigma = 4 blobs and the serpentine at 8192^2.  Each image gets two
warm-up calls, then CUDA events around 10 calls on one stream with the default global
grid.  K must equal the default build's K.  The tool prints one JSON object: ms per call
for every (shape, image), the default build under its size rule ("auto"), and, per image,
the fastest shape and its gain over 64 x 256.
The library's size rule (ccl_set_tile_policy, ccl_internal.h) follows this table: 64 x 128
tiles for small images, 64 x 256 for large ones.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes
import importlib
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SHAPES = [(64, 256), (32, 256), (64, 128), (128, 256), (64, 512)]
DEFAULT = (64, 256)


def build_shape(th: int, tw: int) -> str:
    b = importlib.import_module("paper_1606_05973_gb300.build")
    if (th, tw) == DEFAULT:
        return b.build()
    os.makedirs(b.OUT, exist_ok=True)
    b.write_tuning_include()
    tag = f"tile_{th}x{tw}"
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", b.OUT, *b.ARCH,
             f"-DCCL_TILE_H={th}", f"-DCCL_TILE_W={tw}"]

    def one(src):
        obj = os.path.join(b.OUT, f"{os.path.splitext(src)[0]}.{tag}.o")
        subprocess.run([b.nvcc(), *flags, "-c", os.path.join(b.CSRC, src), "-o", obj], check=True)
        return obj

    with cf.ThreadPoolExecutor(len(b.SOURCES)) as ex:
        objs = list(ex.map(one, b.SOURCES))
    target = os.path.join(b.OUT, f"libccl_{tag}.so")
    subprocess.run([b.nvcc(), "-shared", *b.ARCH, "-o", target, *objs, "-lcudart"], check=True)
    return target


def images(dev):
    import torch

    import synth

    out = []
    for side in (128, 512, 2048, 4096, 8192):
        for p, seed in ((0.1, 21), (0.5, 22), (0.9, 23)):
            out.append((f"{side}^2 bernoulli p={p}", torch.from_numpy(synth.bernoulli(side, side, p, seed)).to(dev)))
    out.append(("8192^2 blobs sigma=4", synth.blobs_device(8192, 8192, 4.0, 7, dev)))
    out.append(("8192^2 serpentine", torch.from_numpy(synth.serpentine(8192, 8192)).to(dev)))
    return out


def main():
    import torch

    import paper_1606_05973_gb300 as ccl

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="also write the JSON object to this file")
    args = ap.parse_args()
    with cf.ThreadPoolExecutor(len(SHAPES)) as ex:
        libs = dict(zip(SHAPES, ex.map(lambda s: build_shape(*s), SHAPES)))
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    st = torch.cuda.Stream(device=dev)
    sp = ctypes.c_void_p(st.cuda_stream)
    kd = torch.zeros(1, dtype=torch.int32, device=dev)
    imgs = images(dev)
    ms = {f"{th}x{tw}": {} for th, tw in SHAPES}
    ms["auto"] = {}
    ref_k = {}
    for shape in SHAPES + ["auto"]:
        # each build on its own shape at every size (policy 1); "auto": the library's size rule
        lib = ccl.load(path=libs[DEFAULT if shape == "auto" else shape])
        if lib.ccl_set_tile_policy(0 if shape == "auto" else 1) != 0:
            raise RuntimeError("ccl_set_tile_policy failed")
        key = "auto" if shape == "auto" else f"{shape[0]}x{shape[1]}"
        for name, img in imgs:
            H, W = img.shape
            lab = torch.empty((H, W), dtype=torch.int32, device=dev)

            def call():
                rc = lib.ccl_label_async(img.data_ptr(), H, W, img.stride(0), 8, lab.data_ptr(),
                                         ctypes.c_void_p(kd.data_ptr()), sp)
                if rc != 0:
                    raise RuntimeError(f"{key} {name}: ccl_label_async returned {rc}")

            for _ in range(2):
                call()
            st.synchronize()
            k = int(kd.item())
            if shape == DEFAULT:
                ref_k[name] = k
            elif ref_k.get(name) != k:
                raise RuntimeError(f"{key} {name}: K={k}, default build K={ref_k.get(name)}")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(10):
                call()
            e1.record(st)
            e1.synchronize()
            ms[key][name] = round(e0.elapsed_time(e1) / 10, 4)
            del lab
    best = {}
    d = f"{DEFAULT[0]}x{DEFAULT[1]}"
    for name, _ in imgs:
        k, v = min(((k, ms[k][name]) for k in ms if k != "auto"), key=lambda kv: kv[1])
        best[name] = {"shape": k, "ms": v, "gain_vs_default": round(ms[d][name] / v, 3)}
    total = {k: round(sum(ms[k].values()), 3) for k in ms}
    out = {"ms_per_call": ms, "best": best, "sum_ms": total}
    txt = json.dumps(out, indent=1)
    print(txt)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
