"""Offline tile-shape sweep and the autotuner of the persistent launch.

    python -m paper_1606_05973_gb300.tile_sweep [--out PATH]
    python -m paper_1606_05973_gb300.tile_sweep --write-table [--table-out PATH] [--summary-out PATH]

--write-table measures the persistent single launch over size classes x density classes x
the two compiled tile shapes x grids of 4, 6 and 8 CTAs per SM, single images under the
persistent launch against the three kernels, and batches of large images fanned out over
streams against three launches over the batch, and writes the library's tuning table
(tuning.json, compiled into libccl by build.py) from the fastest entries.
--streams-only measures only the last and updates streams_min_px in the table.

Without it:

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


# ---- autotuner of the persistent launch (--write-table) ------------------------------------
# Size classes (a batch's total pixels) and their representative batches: (count, side).
SIZE_CLASSES = [(1 << 20, (1, 1024)), (1 << 22, (1, 2048)), (1 << 24, (1, 4096)), (1 << 26, (64, 1024)),
                (None, (16, 4096))]
DENSITIES = (0.1, 0.5, 0.9)  # one Bernoulli density inside each class of density_bounds (0.3, 0.7)
CTAS = (4, 6, 8)
SINGLE_SIDES = (256, 512, 1024, 1536, 2048, 3072, 4096, 8192)
STREAM_SIDES = (4096, 6144, 8192, 12288, 16384)
FAN_MARGIN = 0.95


def fanout_threshold(sides, fan_ms, three_ms, margin=FAN_MARGIN):
    """The fan-out threshold from per-side timings (sides ascending): the pixel count of the
    smallest side from which the fan-out takes at most `margin` of the three-launch time at
    that side and at every larger one; -1 if it does not at the largest side."""
    best = -1
    for side, f, t in reversed(list(zip(sides, fan_ms, three_ms))):
        if not f < margin * t:
            break
        best = side * side
    return best


def streams_threshold(lines):
    """Batches of six images of each side in STREAM_SIDES (two each of sigma = 16 blobs,
    Bernoulli(0.6) and the serpentine; more images favour the launches over the whole batch),
    fanned out over streams (launch mode 3) against three launches over the batch (mode 1);
    returns the smallest side^2 from which the fan-out is at least 5% faster at that side
    and every larger one (-1: at none); below, the winner depends on the number of images."""
    import torch

    import paper_1606_05973_gb300 as ccl
    import synth

    lib = ccl.lib()
    dev = torch.device("cuda:0")
    sync = torch.cuda.synchronize
    fan, three = [], []
    lines.append("batches of six images, ms per call: fanned out over streams / three launches")
    for side in STREAM_SIDES:
        imgs = []
        for r in range(2):
            imgs += [synth.blobs_device(side, side, 16.0, 8 + 3 * r, dev),
                     torch.from_numpy(synth.bernoulli(side, side, 0.6, 9 + 3 * r)).to(dev),
                     torch.from_numpy(synth.serpentine(side, side)).to(dev)]
        outs = [torch.empty((side, side), dtype=torch.int32, device=dev) for _ in imgs]
        kd = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
        ms = {}
        ks = {}
        for mode in (3, 1):
            lib.ccl_set_launch_mode(mode)
            ms[mode] = _time(lambda: ccl.label_batch(imgs, outs=outs, k_out=kd), sync)
            ks[mode] = kd.cpu().tolist()
        lib.ccl_set_launch_mode(0)
        if ks[3] != ks[1]:
            raise RuntimeError(f"K differs between the batch forms at {side}^2")
        fan.append(ms[3])
        three.append(ms[1])
        lines.append(f"  {side}^2: {ms[3]:.4f} / {ms[1]:.4f}")
        del imgs, outs
        torch.cuda.empty_cache()
    best = fanout_threshold(STREAM_SIDES, fan, three)
    lines.append(f"batches whose smallest image has at least {best} px are fanned out over streams")
    return best


def _time(fn, sync, reps=10, warm=2):
    """ms per call of fn captured once in a CUDA graph and replayed (no host work between
    replays: the launch forms are compared on the device alone)."""
    import torch

    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for _ in range(warm):
            fn()  # sizes the stream's workspace before capture
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            fn()
        g.replay()
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            g.replay()
        e1.record(st)
    e1.synchronize()
    sync()
    return e0.elapsed_time(e1) / reps


def write_table(out_json, out_txt):
    """Measures the persistent launch for every size class x density class x tile shape x
    grid (CTAs per SM), and single images under the persistent launch against the three
    kernels; writes tuning.json (the fastest shape per class, the grid with the smallest
    sum over the densities, and the largest single-image size at which the persistent
    launch wins on every content) and a text summary of the measurements."""
    import torch

    import paper_1606_05973_gb300 as ccl
    import synth

    lib = ccl.lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    sync = torch.cuda.synchronize
    rows, lines = [], []
    for bound, (count, side) in SIZE_CLASSES:
        per = {}  # (density, shape, ctas) -> ms
        per3 = {}  # density -> ms of the three-launch batch
        for di, p in enumerate(DENSITIES):
            imgs = [torch.from_numpy(synth.bernoulli(side, side, p, 300 + 7 * di + i)).to(dev) for i in range(count)]
            outs = [torch.empty((side, side), dtype=torch.int32, device=dev) for _ in imgs]
            kd = torch.zeros(count, dtype=torch.int32, device=dev)
            ref = None
            lib.ccl_set_launch_mode(2)  # the persistent launch, whatever the current table says
            for shape, policy in (("64x128", 2), ("64x256", 1)):
                lib.ccl_set_tile_policy(policy)
                for c in CTAS:
                    lib.ccl_set_persistent_ctas_per_sm(c)
                    ms = _time(lambda: ccl.label_batch(imgs, outs=outs, k_out=kd), sync)
                    k = kd.cpu().tolist()
                    if ref is None:
                        ref = k
                    elif k != ref:
                        raise RuntimeError(f"K differs across shapes: {side} p={p} {shape} {c}")
                    per[(di, shape, c)] = ms
            # the same batch in three launches (the size rule's tile shape)
            lib.ccl_set_tile_policy(0)
            lib.ccl_set_persistent_ctas_per_sm(0)
            lib.ccl_set_launch_mode(1)
            per3[di] = _time(lambda: ccl.label_batch(imgs, outs=outs, k_out=kd), sync)
            lib.ccl_set_launch_mode(2)
            if kd.cpu().tolist() != ref:
                raise RuntimeError(f"K differs between the launch modes: {side} p={p}")
            del imgs, outs
            torch.cuda.empty_cache()
        lib.ccl_set_tile_policy(0)
        lib.ccl_set_persistent_ctas_per_sm(0)
        lib.ccl_set_launch_mode(0)
        best_shape = []
        for di in range(3):
            best_shape.append(min(("64x128", "64x256"), key=lambda sh: min(per[(di, sh, c)] for c in CTAS)))
        best_c = min(CTAS, key=lambda c: sum(per[(di, best_shape[di], c)] for di in range(3)))
        pers_ms = sum(per[(di, best_shape[di], best_c)] for di in range(3))
        rows.append({"max_px": bound, "shape": best_shape, "ctas_per_sm": best_c,
                     "persistent": bool(pers_ms < sum(per3.values()))})
        lines.append(f"class <= {bound if bound else 'inf'} px ({count} x {side}^2):")
        for di, p in enumerate(DENSITIES):
            cells = "  ".join(f"{sh}/{c}: {per[(di, sh, c)]:.4f}" for sh in ("64x128", "64x256") for c in CTAS)
            lines.append(f"  p={p}  {cells}  -> {best_shape[di]}")
        lines.append(f"  grid: {best_c} CTAs per SM; three launches: "
                     + "  ".join(f"p={p}: {per3[di]:.4f}" for di, p in enumerate(DENSITIES))
                     + f" -> {'persistent' if rows[-1]['persistent'] else 'three launches'}")
    # single images: persistent launch (a batch of one) against the three kernels
    single_max = 0
    lines.append("single images, ms per call: persistent / three kernels")
    for side in SINGLE_SIDES:
        wins = True
        for name, img in ((f"bernoulli p=0.5", torch.from_numpy(synth.bernoulli(side, side, 0.5, side)).to(dev)),
                          (f"blobs sigma=4", synth.blobs_device(side, side, 4.0, side + 1, dev)),
                          (f"bernoulli p=0.1", torch.from_numpy(synth.bernoulli(side, side, 0.1, side + 2)).to(dev))):
            out = torch.empty((side, side), dtype=torch.int32, device=dev)
            kd = torch.zeros(1, dtype=torch.int32, device=dev)
            lib.ccl_set_launch_mode(2)
            pers = _time(lambda: ccl.label_batch([img], outs=[out], k_out=kd), sync)
            k1 = int(kd.item())
            lib.ccl_set_launch_mode(1)
            three = _time(lambda: lib.ccl_label_async(img.data_ptr(), side, side, img.stride(0), 8, out.data_ptr(),
                                                      ctypes.c_void_p(kd.data_ptr()),
                                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), sync)
            lib.ccl_set_launch_mode(0)
            if int(kd.item()) != k1:
                raise RuntimeError(f"K differs between the launch modes at {side}^2 {name}")
            wins &= pers < three
            lines.append(f"  {side}^2 {name}: {pers:.4f} / {three:.4f}")
        if wins:
            single_max = side * side
    streams_min = streams_threshold(lines)
    t = {"about": json.load(open(TUNING_PATH))["about"],
         "written_by": "python -m paper_1606_05973_gb300.tile_sweep --write-table (GB300 measurements)",
         "density_bounds": [0.3, 0.7], "probe_samples": 64, "single_fused_max_px": single_max,
         "streams_min_px": streams_min, "rows": rows}
    txt = json.dumps(t, indent=2)
    with open(out_json, "w") as f:
        f.write(txt + "\n")
    lines.append(f"single images take the persistent launch up to {single_max} px")
    with open(out_txt, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))
    print(txt)


TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def main():
    import torch

    import paper_1606_05973_gb300 as ccl

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="also write the JSON object to this file")
    ap.add_argument("--write-table", action="store_true",
                    help="tune the persistent launch and write tuning.json (see write_table)")
    ap.add_argument("--streams-only", action="store_true",
                    help="measure only the fan-out threshold and update streams_min_px in the table")
    ap.add_argument("--table-out", default=TUNING_PATH)
    ap.add_argument("--summary-out", default=None)
    args = ap.parse_args()
    if args.streams_only:
        lines = []
        t = json.load(open(TUNING_PATH))
        t["streams_min_px"] = streams_threshold(lines)
        with open(args.table_out, "w") as f:
            f.write(json.dumps(t, indent=2) + "\n")
        txt = "\n".join(lines) + "\n"
        print(txt)
        if args.summary_out:
            with open(args.summary_out, "w") as f:
                f.write(txt)
        return
    if args.write_table:
        write_table(args.table_out, args.summary_out or os.path.join(os.getcwd(), "tuning_sweep.txt"))
        return
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
