"""Benchmark: labelled Gpixels/s of the GPU path, with its HBM roofline, an end-to-end
number through the host-buffer entry point, clocks, and the CPU oracle beside it.

Workload (default ``big21568``): the three ~465 MB images of the paper's largest raster
size (Table III's image_6, 465.20 MB at one byte per pixel, read as 21568 x 21568):
sigma=16 thresholded Gaussian-field blobs (seed 8), Bernoulli(0.6) (seed 9) and the
serpentine (one 1-px path through the whole image), 8-connectivity, int32 labels.  One
step labels all three (one ``ccl_label_async`` call each) with the inputs already
resident in HBM.  ``sweep8192`` (six 8192 x 8192 images: Bernoulli p in
{0.1,0.3,0.5,0.7,0.9} and a sigma=4 field) and ``small1024`` (1024 x 1024 Bernoulli(0.5))
can be timed the same way; the default run also reports both as extra keys, with the
1024 x 1024 call replayed from a CUDA graph.

The images of a step go round robin over three streams (``--streams``) with the cooperative
global kernel capped at one CTA per SM (``--global-ctas-per-sm``,
``ccl_set_global_ctas_per_sm``), so that one image's tile pass can run beside another's
global pass.  The line also carries the same steps on one stream with the library's
default grid (``one_stream``), per-kernel launch times taken on one stream, and per-image
median / p99 latency over at least 20 calls.  The device status word of every stream is
checked after every pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload big21568|sweep8192|small1024] [--streams S]
                    [--global-ctas-per-sm N]

Under torchrun each rank labels its own copy of the workload (independent replicas, no
collective on the data path); rank 0 prints one JSON line with the max time over ranks.
``--impl reference`` times the CPU oracle (the paper's PARemSP on OpenMP threads) on the
same images (identical bytes, SHA-256 in both lines), one image per step.
"""
from __future__ import annotations

import argparse
import atexit
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "Gpixels/s labeled (bit-exact) & % of HBM roofline; batched vs per-image; p99 ms"
UNIT = "Gpixels/s"
# algorithmic bytes per pixel: 1 B image read + 4 B label write (whole path)
PATH_BYTES_PER_PX = 5.0
# per kernel: tile_local reads the image (1 B/px) and writes the bit pack (1/8 B/px);
# final_labels reads the bit pack (1/8 B/px) and writes the labels (4 B/px)
KERNEL_BYTES_PER_PX = {"tile_local": 1.125, "final_labels": 4.125}
L2_NOTE = {"big21568": "inputs larger than L2: 3 x 465 MB images read and 3 x 1.86 GB labels written per step",
           "sweep8192": "inputs larger than L2: 6 x 64 MiB images read and 6 x 256 MiB labels written per step",
           "small1024": "one 1 MiB image: L2-resident (launch-bound case)"}
FALLBACK_HBM_GBS = 6800.0


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---- multi-rank helpers (independent replicas; a collective only for timing) ------------

def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (NCCL with a CUDA device, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gpx_s(px_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: every rank labels the same amount of work (weak scaling),
    the job lasts as long as its slowest rank."""
    return world * px_per_rank / seconds_max / 1e9


# ---- workloads ---------------------------------------------------------------------------

S_BIG = 21568
WORKLOAD_DESC = {
    "big21568": {"workload": "21568x21568 uint8 (~465 MB, Table III image_6 size) x3: sigma=16 thresholded "
                             "Gaussian-field blobs (seed 8), Bernoulli(0.6) (seed 9), serpentine; "
                             "8-connectivity; int32 labels",
                 "images": 3, "H": S_BIG, "W": S_BIG},
    "sweep8192": {"workload": "8192x8192 uint8 x6: Bernoulli p in {0.1,0.3,0.5,0.7,0.9} (seeds 2-6) "
                              "+ sigma=4 thresholded Gaussian field (seed 7); 8-connectivity; int32 labels",
                  "images": 6, "H": 8192, "W": 8192},
    "small1024": {"workload": "1024x1024 uint8 Bernoulli(0.5) seed 1; 8-connectivity; int32 labels",
                  "images": 1, "H": 1024, "W": 1024},
}


def workload_images(name, device=None, side=None):
    """The images of workload `name` as (label, image) pairs: uint8 torch tensors on
    `device` when one is given, else numpy arrays on the host.  Thresholded fields are
    smoothed on the GPU whenever one is present (also for host arrays), so that both
    benchmark arms see identical bytes; without a GPU the host generator of the same recipe
    is used (its bytes may differ near the threshold; the SHA-256 in the line says)."""
    import torch

    cuda = torch.cuda.is_available()
    gen_dev = device if device is not None else (torch.device("cuda", torch.cuda.current_device()) if cuda else None)

    def field(h, w, sigma, seed):
        if gen_dev is not None:
            t = synth.blobs_device(h, w, sigma, seed, gen_dev)
            return t if device is not None else t.cpu().numpy()
        img = synth.blobs(h, w, sigma, seed)
        return torch.from_numpy(img).to(device) if device is not None else img

    def host(img):
        return torch.from_numpy(img).to(device) if device is not None else img

    out = []
    if name == "sweep8192":
        for kind, arg, seed in synth.SWEEP_8192:
            if kind == "bernoulli":
                out.append((f"bernoulli_p{arg}", host(synth.bernoulli(8192, 8192, arg, seed))))
            else:
                out.append((f"blobs_sigma{arg:g}", field(8192, 8192, arg, seed)))
    elif name == "big21568":
        s = side or S_BIG  # a smaller side keeps the recipe for profiling captures
        out.append(("blobs_sigma16", field(s, s, 16.0, 8)))
        out.append(("bernoulli_p0.6", host(synth.bernoulli(s, s, 0.6, 9))))
        out.append(("serpentine", host(synth.serpentine(s, s))))
    elif name == "small1024":
        out.append(("bernoulli_p0.5", host(synth.bernoulli(1024, 1024, 0.5, 1))))
    else:
        raise SystemExit(f"unknown workload {name}")
    return out


def image_sha256(img):
    """SHA-256 of an image's bytes (torch tensor on any device, or numpy array)."""
    if hasattr(img, "cpu"):
        img = img.cpu().numpy()
    return synth.sha256(img)


def make_workload(name, device, only=None, side=None):
    """Returns (list of (label, uint8 CUDA tensor), description dict with input SHA-256s)."""
    imgs = workload_images(name, device, side)
    if only:
        imgs = [(n, t) for n, t in imgs if n == only]
    desc = {**WORKLOAD_DESC[name], "inputs_sha256": {n: image_sha256(t) for n, t in imgs}}
    if side and name == "big21568" and side != S_BIG:
        desc = {**desc, "H": side, "W": side,
                "workload": desc["workload"].replace("21568x21568 uint8 (~465 MB, Table III image_6 size)",
                                                     f"{side}x{side} uint8 (the 21568x21568 recipe at a smaller side)")}
    return imgs, desc


# ---- clocks ------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples (every 20 ms: a default step sequence runs for tens of
    milliseconds) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []  # (host time, csv line)
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Samples taken inside the timed region (marked on the host); if the region was
        too short to hold one, the samples within 0.5 s of it (warm-up and the kernel
        passes around it, the same work), and `window` says which."""
        if not self.lines:
            return None
        window = "timed region"
        t0, t1 = (self.t0 or 0.0), (self.t1 or float("inf"))
        picked = [ln for t, ln in self.lines if t0 <= t <= t1 + 0.02]
        if not picked:
            window = "within 0.5 s of the timed region (warm-up and kernel passes)"
            picked = [ln for t, ln in self.lines if t0 - 0.5 <= t <= t1 + 0.5]
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in picked:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


# ---- peaks and profiles ------------------------------------------------------------------

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ccl_core.cuh", "ccl_kernels.cu"):
        with open(os.path.join(ROOT, "paper_1606_05973_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary for this workload,
    or None if there is none or the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ":" in ln and not ln.startswith(" "):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---- our arm ------------------------------------------------------------------------------

def conn_desc(desc, conn):
    """The workload description under `conn`-connectivity (the workloads are stated for 8)."""
    if conn == 8:
        return desc
    return {**desc, "workload": desc["workload"].replace("8-connectivity", f"{conn}-connectivity")}


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1606_05973_gb300 as ccl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = ccl.lib()
    imgs, desc = make_workload(args.workload, dev, args.only, args.side)
    desc = conn_desc(desc, args.connectivity)
    if args.only:
        imgs = [(n, t) for n, t in imgs if n == args.only]
        if not imgs:
            raise SystemExit(f"--only {args.only}: no such image in {args.workload}")
        desc = {**desc, "images": 1, "only": args.only}
    labels = [torch.empty(tuple(t.shape), dtype=torch.int32, device=dev) for _, t in imgs]
    kdev = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    px_per_step = sum(t.shape[0] * t.shape[1] for _, t in imgs)
    # images alternate over `streams` streams (the library keeps one workspace per stream),
    # so one image's tile pass can run beside another's global pass
    side = [torch.cuda.Stream(device=dev) for _ in range(args.streams - 1)]
    step_streams = [stream] + side
    step_sptr = [ctypes.c_void_p(st.cuda_stream) for st in step_streams]
    if args.global_ctas_per_sm is not None:
        if lib.ccl_set_global_ctas_per_sm(args.global_ctas_per_sm) != 0:
            raise RuntimeError("ccl_set_global_ctas_per_sm rejected its argument")

    def step(nstreams=None):
        ns = nstreams or len(step_streams)
        for i, (_, t) in enumerate(imgs):
            H, W = t.shape
            rc = lib.ccl_label_async(t.data_ptr(), H, W, t.stride(0), args.connectivity, labels[i].data_ptr(),
                                     kdev.data_ptr() + 4 * i, step_sptr[i % ns])
            if rc != 0:
                raise RuntimeError(f"ccl_label_async: {ccl.ccl_status_string(rc)}")

    clk = ClockSampler(local_rank).__enter__()  # started early: nvidia-smi takes a while to start
    atexit.register(clk.__exit__, None, None, None)  # stopped on any way out
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def check_status(where, sptrs=step_sptr):
        """The device status word of every stream's workspace (a capped loop or barrier
        would leave a bit set); read and cleared after every pass."""
        flags = ctypes.c_int32(0)
        for sp in sptrs:
            rc = lib.ccl_device_status(sp, ctypes.byref(flags))
            if rc != 0 or flags.value:
                raise RuntimeError(f"device status {flags.value} (rc {rc}) after {where}")

    check_status("warm-up")

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # timed region: K steps between two events, barrier + synchronize on both sides
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clk.mark_start()
    e0.record(stream)
    for st in side:
        st.wait_stream(stream)
    for _ in range(args.steps):
        step()
    for st in side:
        stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    clk.mark_end()
    barrier()
    ms = e0.elapsed_time(e1)
    check_status("the timed pass")
    ms_max = max_over_ranks(ms, world, dev)

    # the same steps on one stream with the library's default global grid, for comparison
    lib.ccl_set_global_ctas_per_sm(0)
    o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        step(nstreams=1)
    barrier()
    torch.cuda.synchronize()
    o0.record(stream)
    for _ in range(args.steps):
        step(nstreams=1)
    o1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_one = max_over_ranks(o0.elapsed_time(o1), world, dev)
    check_status("the one-stream pass")
    if args.global_ctas_per_sm is not None:
        lib.ccl_set_global_ctas_per_sm(args.global_ctas_per_sm)

    # per-kernel device times: the same K steps again with the library's event pair around
    # every launch on its stream.  The events leave a small gap between launches (about 5%
    # of a sweep step), so this pass gives the kernel breakdown and the roofline's launch
    # durations, and the pass above gives `value`.
    ccl.ccl_profile_reset()
    ccl.ccl_profile_enable(1)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(args.steps):
        step(nstreams=1)  # one stream: each launch's duration is its own
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ccl.ccl_profile_enable(0)
    clk.__exit__(None, None, None)
    prof_ms = p0.elapsed_time(p1)
    kt = ccl.kernel_times()
    launches = sum(v[0] for v in kt.values())
    check_status("the per-kernel pass")

    # per-image latency: each image labelled alone, one stream, an event pair per call, with
    # the library's default global grid (the per-SM cap is for images on several streams)
    lib.ccl_set_global_ctas_per_sm(0)
    per_image = {}
    for i, (name, t) in enumerate(imgs):
        H, W = t.shape
        times = []
        for _ in range(max(20, args.steps)):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            rc = lib.ccl_label_async(t.data_ptr(), H, W, t.stride(0), args.connectivity, labels[i].data_ptr(),
                                     kdev.data_ptr() + 4 * i, sptr)
            a1.record(stream)
            if rc != 0:
                raise RuntimeError(f"ccl_label_async: {ccl.ccl_status_string(rc)}")
            times.append((a0, a1))
        torch.cuda.synchronize()
        ms_i = sorted(a.elapsed_time(b) for a, b in times)
        per_image[name] = {"runs": len(ms_i), "median_ms": round(statistics.median(ms_i), 4),
                           "p99_ms": round(ms_i[min(len(ms_i) - 1, int(0.99 * len(ms_i)))], 4),
                           "gpx_s_median": round(H * W / (statistics.median(ms_i) * 1e-3) / 1e9, 2)}
    check_status("the per-image pass", [sptr])
    if args.global_ctas_per_sm is not None:
        lib.ccl_set_global_ctas_per_sm(args.global_ctas_per_sm)

    # correctness spot check outside the timed region: K must match a fresh labelling
    ks = kdev.cpu().tolist()

    # the same images per step in one ccl_label_batch call (one launch per kernel over all
    # of them), replayed from a CUDA graph, for comparison with the per-image calls
    same_batch = None
    if len(imgs) > 1:
        kb = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
        lib.ccl_set_global_ctas_per_sm(0)  # one stream: the global kernel may fill every SM
        bst = torch.cuda.Stream(device=dev)
        bst.wait_stream(stream)
        with torch.cuda.stream(bst):
            def bcall():
                ccl.label_batch([t for _, t in imgs], connectivity=args.connectivity, outs=labels, stream=bst,
                                k_out=kb)

            bcall()
            bst.synchronize()
            gb = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gb, stream=bst):
                bcall()
            gb.replay()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(bst)
            for _ in range(args.steps):
                gb.replay()
            b1.record(bst)
        torch.cuda.synchronize()
        if args.global_ctas_per_sm is not None:
            lib.ccl_set_global_ctas_per_sm(args.global_ctas_per_sm)
        check_status("the same-images batch pass", [ctypes.c_void_p(bst.cuda_stream)])
        if kb.cpu().tolist() != ks:
            raise RuntimeError("batched and per-image component counts differ")
        bms = b0.elapsed_time(b1) / args.steps
        same_batch = {"ms_per_step": round(bms, 4), "value": round(px_per_step / (bms * 1e-3) / 1e9, 2),
                      "path_frac": round(PATH_BYTES_PER_PX * px_per_step / (bms * 1e-3) / 1e9 / hbm_peak()[0], 4),
                      "how": "the step's images in one ccl_label_batch call (the tuning table's launch form), "
                             "replayed from a CUDA graph"}

    # end to end through the host-buffer entry point (pinned memory), outside the timed region
    host_imgs = [t.cpu().pin_memory() for _, t in imgs]
    host_labs = [torch.empty(tuple(t.shape), dtype=torch.int32).pin_memory() for _, t in imgs]

    # two streams, images alternating, so that one image's label download overlaps the next
    # image's upload and labelling (each copy direction runs at about 200 GB/s)
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    e2e_sptr = [ctypes.c_void_p(st.cuda_stream) for st in e2e_streams]
    host_k = torch.zeros(len(host_imgs), dtype=torch.int32).pin_memory()

    def e2e_step():
        for i, (hi, hl) in enumerate(zip(host_imgs, host_labs)):
            H, W = hi.shape
            rc = lib.ccl_label_host_async(hi.data_ptr(), H, W, hi.stride(0), args.connectivity, hl.data_ptr(),
                                          ctypes.c_void_p(host_k.data_ptr() + 4 * i), e2e_sptr[i % 2])
            if rc != 0:
                raise RuntimeError(f"ccl_label_host_async: {ccl.ccl_status_string(rc)}")
        for st in e2e_streams:
            st.synchronize()

    e2e_step()
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    # the median step: host-memory copies vary from step to step far more than the kernels
    e2e_s = max_over_ranks(statistics.median(e2e_times), world, dev)
    check_status("the end-to-end pass", e2e_sptr)
    # what bounds it: one stream's device-to-host copy of one image's labels into pinned memory
    d2h0, d2h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d2h0.record(stream)
    host_labs[0].copy_(labels[0], non_blocking=True)
    d2h1.record(stream)
    torch.cuda.synchronize()
    d2h_gbs = 4 * labels[0].numel() / (d2h0.elapsed_time(d2h1) * 1e-3) / 1e9
    lib.ccl_set_global_ctas_per_sm(0)  # library default for the measurements below
    for i, hl in enumerate(host_labs):
        if int(hl.max()) != ks[i] or int(host_k[i]) != ks[i]:
            raise RuntimeError("host-buffer labels disagree with the device run")

    if rank != 0:
        return None
    step_ms = ms_max / args.steps
    value = aggregate_gpx_s(px_per_step, world, step_ms * 1e-3)
    peak, peak_kind = hbm_peak()
    # dominant kernel by summed device time (among those with an algorithmic byte model)
    overall = max(kt.items(), key=lambda kv: kv[1][1])[0]
    dom = max(((k, v) for k, v in kt.items() if k in KERNEL_BYTES_PER_PX), key=lambda kv: kv[1][1])
    dname, (dl, dms) = dom[0], dom[1]
    per_launch_px = px_per_step / len(imgs)  # each kernel launch covers one image
    roof = None
    if dname in KERNEL_BYTES_PER_PX and dl > 0:
        achieved = KERNEL_BYTES_PER_PX[dname] * per_launch_px / (dms / dl * 1e-3) / 1e9
        tr = ncu_traffic(dname, args.workload if args.connectivity == 8 else f"{args.workload}_conn{args.connectivity}")
        roof = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                "traffic": tr, "algorithmic_bytes_per_launch": KERNEL_BYTES_PER_PX[dname] * per_launch_px,
                "avg_launch_ms": round(dms / dl, 4), "dominant_overall": overall}
    path_gbs = PATH_BYTES_PER_PX * px_per_step / (step_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8->int32", "data": "synthetic",
        "config": {**desc, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "streams": args.streams, "global_ctas_per_sm": args.global_ctas_per_sm or "all that fit",
                   "l2": L2_NOTE.get(args.workload, "inputs larger than L2")},
        "roofline": roof,
        "path_roofline": {"bytes_per_px": PATH_BYTES_PER_PX, "achieved_gbs": round(path_gbs, 1),
                          "frac": round(path_gbs / peak, 4), "peak": peak, "peak_source": peak_kind},
        "one_stream": {"value": round(aggregate_gpx_s(px_per_step, world, ms_one / args.steps * 1e-3), 2),
                       "ms_per_step": round(ms_one / args.steps, 4),
                       "how": "the same steps on one stream, global kernel with as many CTAs per SM as fit"},
        "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 4),
                        "avg_launch_ms": round(v[1] / v[0], 4),
                        **({"achieved_gbs": round(KERNEL_BYTES_PER_PX[k] * per_launch_px / (v[1] / v[0] * 1e-3) / 1e9, 1),
                            "frac": round(KERNEL_BYTES_PER_PX[k] * per_launch_px / (v[1] / v[0] * 1e-3) / 1e9 / peak, 4)}
                           if k in KERNEL_BYTES_PER_PX else {})}
                    for k, v in kt.items() if v[0]},
        "per_image": per_image,
        "same_images_batched": same_batch,
        "kernels_pass": {"steps": args.steps, "ms_per_step": round(prof_ms / args.steps, 4),
                         "how": "a second timed pass of the same steps with an event pair around every "
                                "launch; `value` comes from the pass without them"},
        "gpu_launches": int(launches),
        "components": {name: int(k) for (name, _), k in zip(imgs, ks)},
        "e2e": {"value": round(aggregate_gpx_s(px_per_step, world, e2e_s), 3), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(t.numel() for t in host_imgs)),
                "d2h_bytes_per_step": int(sum(4 * t.numel() + 4 for t in host_labs)),
                "api": "ccl_label_host_async on two streams, images alternating (pinned host buffers, "
                       "copies inside the timed region, both streams synchronised at the end of each step)",
                "steps": e2e_steps, "step_ms_median": round(statistics.median(e2e_times) * 1e3, 2),
                "step_ms_min": round(min(e2e_times) * 1e3, 2), "step_ms_max": round(max(e2e_times) * 1e3, 2),
                "d2h_copy_gbs": round(d2h_gbs, 1),
                "d2h_copy_how": "one image's labels, device to pinned host memory, one copy on one stream"},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline([t for _, t in imgs], args)
    del imgs, labels, host_imgs, host_labs
    torch.cuda.empty_cache()
    if args.extras:
        for extra in ("sweep8192", "small1024"):
            if extra != args.workload:
                line[extra] = measure_plain(args, extra, dev, lib)
                torch.cuda.empty_cache()
    if args.batch_images > 0:
        line["batched"] = measure_batched(args, dev, lib, stream)
        torch.cuda.empty_cache()
    if args.served:
        line["served"] = measure_served(args, dev)
    if args.fused:
        line["fused_binarisation"] = measure_fused(args, dev, lib, stream)
        torch.cuda.empty_cache()
        line["multi_class"] = measure_classes(args, dev, lib, stream)
        torch.cuda.empty_cache()
    return line


def measure_plain(args, name, dev, lib):
    """Another plain-path workload as an extra key: images round robin over the headline's
    streams with the global kernel at one CTA per SM (as the headline), CUDA events around 10 steps
    after 3 warm-up steps; for single-image workloads also one call captured in a CUDA graph
    and replayed (a small image is launch-bound and L2-resident).  K is checked against
    the plain call, and the device status after each pass."""
    import torch

    import paper_1606_05973_gb300 as ccl

    imgs, desc = make_workload(name, dev)
    labels = [torch.empty(tuple(t.shape), dtype=torch.int32, device=dev) for _, t in imgs]
    kdev = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
    nstreams = max(1, args.streams)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    sptr = [ctypes.c_void_p(st.cuda_stream) for st in streams]
    px = sum(t.numel() for _, t in imgs)
    lib.ccl_set_global_ctas_per_sm(args.global_ctas_per_sm or 0)

    def step(ns=nstreams):
        for i, (_, t) in enumerate(imgs):
            H, W = t.shape
            rc = lib.ccl_label_async(t.data_ptr(), H, W, t.stride(0), args.connectivity, labels[i].data_ptr(),
                                     kdev.data_ptr() + 4 * i, sptr[i % ns])
            if rc != 0:
                raise RuntimeError(f"ccl_label_async: {ccl.ccl_status_string(rc)}")

    def status():
        flags = ctypes.c_int32(0)
        for sp in sptr:
            if lib.ccl_device_status(sp, ctypes.byref(flags)) != 0 or flags.value:
                raise RuntimeError(f"device status {flags.value} in {name}")

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    main = streams[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10 if len(imgs) > 1 else 200
    e0.record(main)
    for st in streams[1:]:
        st.wait_stream(main)
    for _ in range(reps):
        step()
    for st in streams[1:]:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize()
    status()
    ms = e0.elapsed_time(e1) / reps
    peak, kind = hbm_peak()
    gbs = PATH_BYTES_PER_PX * px / (ms * 1e-3) / 1e9
    res = {"workload": desc["workload"], "inputs_sha256": desc["inputs_sha256"], "ms_per_step": round(ms, 4),
           "value": round(px / (ms * 1e-3) / 1e9, 2), "unit": UNIT,
           "path_frac": round(gbs / peak, 4), "how": f"{reps} steps, images round robin over {nstreams} streams"}
    if len(imgs) == 1:
        ref_k = int(kdev[0])
        lib.ccl_set_global_ctas_per_sm(0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(main):
            step(1)  # the workspace of this stream is sized before capture
            main.synchronize()
            with torch.cuda.graph(g, stream=main):
                step(1)
            kdev.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(main)
            for _ in range(reps):
                g.replay()
            g1.record(main)
        torch.cuda.synchronize()
        status()
        if int(kdev[0]) != ref_k:
            raise RuntimeError("graph replay changed K")
        gms = g0.elapsed_time(g1) / reps
        res["graph_replay"] = {"us_per_image": round(gms * 1e3, 2), "value": round(px / (gms * 1e-3) / 1e9, 2),
                               "how": f"one ccl_label_async call captured in a CUDA graph, {reps} replays"}
        # the same with the persistent launch forced (ccl_set_launch_mode(2)), for comparison
        lib.ccl_set_launch_mode(2)
        g3 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(main):
            step(1)
            main.synchronize()
            with torch.cuda.graph(g3, stream=main):
                step(1)
            g3.replay()
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(main)
            for _ in range(reps):
                g3.replay()
            h1.record(main)
        torch.cuda.synchronize()
        lib.ccl_set_launch_mode(0)
        status()
        if int(kdev[0]) != ref_k:
            raise RuntimeError("persistent graph replay changed K")
        tms = h0.elapsed_time(h1) / reps
        res["graph_replay_persistent"] = {"us_per_image": round(tms * 1e3, 2),
                                          "value": round(px / (tms * 1e-3) / 1e9, 2)}
    lib.ccl_set_global_ctas_per_sm(0)  # library default for the single-stream measurements after
    return res


def measure_classes(args, dev, lib, stream):
    """Multi-class labelling of an 8192x8192 land-cover stand-in (8 classes cut from a
    sigma 4 field at equal-mass quantiles, 10% no-data; seed 15) by ccl_label_classes.
    Inputs resident in HBM; CUDA-event timing over 20 repetitions after 3 warm-ups."""
    import torch

    c = synth.classes_device(8192, 8192, 4.0, 8, 15, dev)
    H, W = c.shape
    lab = torch.empty((H, W), dtype=torch.int32, device=dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def run():
        rc = lib.ccl_label_classes(c.data_ptr(), H, W, c.stride(0), args.connectivity, lab.data_ptr(), None, sptr)
        if rc != 0:
            raise RuntimeError("ccl_label_classes failed")

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    return {"workload": "8192x8192 uint8, 8 classes from a sigma=4 field, 10% no-data (seed 15)",
            "ms": round(ms, 4), "gpx_s": round(H * W / (ms * 1e-3) / 1e9, 2)}


def measure_fused(args, dev, lib, stream):
    """Fused binarisation: an 8192x8192 8-bit grayscale field (sigma 4, seed 12) labelled
    as byte > 127 (Section V's im2bw(0.5)) by ccl_label_threshold in one pass, against a
    separate binarisation pass (torch) followed by ccl_label.  Inputs resident in HBM;
    CUDA-event timing over 20 repetitions after 3 warm-ups."""
    import torch

    g = synth.gray_field_device(8192, 8192, 4.0, 12, dev)
    H, W = g.shape
    lab = torch.empty((H, W), dtype=torch.int32, device=dev)
    binary = torch.empty((H, W), dtype=torch.uint8, device=dev)
    kd = torch.zeros(1, dtype=torch.int32, device=dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def fused():
        rc = lib.ccl_label_threshold(g.data_ptr(), H, W, g.stride(0), args.connectivity, 127, lab.data_ptr(),
                                     None, sptr)
        if rc != 0:
            raise RuntimeError("ccl_label_threshold failed")

    def two_pass():
        torch.gt(g, 127, out=binary)
        rc = lib.ccl_label_async(binary.data_ptr(), H, W, W, args.connectivity, lab.data_ptr(), kd.data_ptr(), sptr)
        if rc != 0:
            raise RuntimeError("ccl_label_async failed")

    res = {"workload": "8192x8192 uint8 grayscale field (sigma 4, seed 12), object = byte > 127"}
    for name, fn in (("fused", fused), ("binarise_then_label", two_pass)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        res[name] = {"ms": round(ms, 4), "gpx_s": round(H * W / (ms * 1e-3) / 1e9, 2)}
    res["speedup"] = round(res["binarise_then_label"]["ms"] / res["fused"]["ms"], 3)
    return res


def measure_served(args, dev):
    """Serving workload: a Poisson stream of square requests (side log-uniform in
    [256, 8192], mixed Bernoulli / blob content, seed 200) through the continuous-batching
    server (16 GiB workspace cap, 3 lanes, batches of up to 64).  Capacity is measured with
    every request submitted at once; then offered loads of 0.2 .. 1.0 x capacity, latency
    from submission to completion as the server records it."""
    import threading

    import torch

    import paper_1606_05973_gb300 as ccl

    sys.setswitchinterval(0.0005)
    specs = synth.served_specs(32, seed=200)
    pool = synth.batch_device(specs, dev)
    outs = [torch.empty(tuple(t.shape), dtype=torch.int32, device=dev) for t in pool for _ in range(2)]
    ref_k = [ccl.label(t, connectivity=args.connectivity)[1] for t in pool]
    torch.cuda.synchronize()
    mean_px = sum(t.numel() for t in pool) / len(pool)
    res = {"workload": "Poisson requests of square uint8 images, side log-uniform in [256, 8192], "
                       "p ~ U(0.2, 0.8), alternating Bernoulli / sigma in {2,4,8} blobs (32 distinct, seed 200)",
           "server": {"mem_cap_bytes": 16 << 30, "lanes": 3, "max_batch": 64}, "loads": []}
    rng = np.random.Generator(np.random.PCG64(200))
    with ccl.Server(mem_cap_bytes=16 << 30, lanes=3, max_batch=64, connectivity=args.connectivity) as srv:
        def run(arrivals):
            n = len(arrivals)
            ids = [0] * n
            bad = []

            def waiter():
                for i in range(n):
                    while ids[i] == 0:
                        time.sleep(0)
                    try:
                        k = srv.wait(ids[i], timeout_ms=60000)
                    except Exception as e:  # noqa: BLE001 - reported by the submitting thread
                        bad.append((i, repr(e)))
                        continue
                    if k != ref_k[i % len(pool)]:
                        bad.append((i, f"K {k} != {ref_k[i % len(pool)]}"))

            th = threading.Thread(target=waiter, daemon=True)
            th.start()
            t0 = time.perf_counter()
            for i, at in enumerate(arrivals):
                while time.perf_counter() - t0 < at:
                    pass
                img = pool[i % len(pool)]
                out = outs[2 * (i % len(pool)) + (i // len(pool)) % 2]  # one of this image's two buffers
                assert out.shape == img.shape
                ids[i] = srv.submit(img, out)
            th.join(timeout=120)
            if th.is_alive():
                raise RuntimeError("served requests did not complete")
            if bad:
                raise RuntimeError(f"served component counts differ for requests {bad[:5]}")
            return srv.stats()

        # capacity: everything submitted at once
        run([0.0] * (4 * len(pool)))
        srv.reset_stats()
        st = run([0.0] * (8 * len(pool)))
        cap = st["completed"] / st["elapsed_s"]
        res["capacity_img_s"] = round(cap, 1)
        res["capacity_gpx_s"] = round(st["gpx_per_s"], 2)
        for load in (0.2, 0.4, 0.6, 0.8, 1.0):
            rate = load * cap
            n = int(min(600, max(120, rate * 0.5)))
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n)).tolist()
            srv.reset_stats()
            st = run(arrivals)
            res["loads"].append({"load": load, "rate_img_s": round(rate, 1), "requests": n,
                                 "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                                 "max_ms": round(st["max_ms"], 3), "gpx_s": round(st["gpx_per_s"], 2),
                                 "mean_batch": round(st["mean_batch"], 2)})
    res["mean_request_mpx"] = round(mean_px / 1e6, 2)
    return res


def measure_batched(args, dev, lib, stream):
    """The uneven-batch workload (sides log-uniform in [64, 2048], p ~ U(0.2, 0.8), half
    Bernoulli, half sigma in {2,4,8} blobs, seed 100) labelled three ways on one stream:
    one ccl_label_async call per image, one ccl_label_batch call, and that call replayed
    from a CUDA graph.  Inputs resident in HBM; CUDA-event timing."""
    import torch

    import paper_1606_05973_gb300 as ccl

    specs = synth.batch_specs(args.batch_images, seed=100)
    imgs = synth.batch_device(specs, dev)
    labs = [torch.empty(tuple(t.shape), dtype=torch.int32, device=dev) for t in imgs]
    kd_single = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
    kd_batch = torch.zeros(len(imgs), dtype=torch.int32, device=dev)
    px = sum(t.numel() for t in imgs)
    # a side stream for all three (graph capture needs a non-default stream)
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def per_image():
        for i, t in enumerate(imgs):
            H, W = t.shape
            rc = lib.ccl_label_async(t.data_ptr(), H, W, t.stride(0), args.connectivity, labs[i].data_ptr(),
                                     kd_single.data_ptr() + 4 * i, sptr)
            if rc != 0:
                raise RuntimeError("ccl_label_async failed")

    def batched():
        ccl.label_batch(imgs, connectivity=args.connectivity, outs=labs, stream=stream, k_out=kd_batch)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def status():
        flags = ctypes.c_int32(0)
        if lib.ccl_device_status(sptr, ctypes.byref(flags)) != 0 or flags.value:
            raise RuntimeError(f"device status {flags.value} in the batched measurement")

    def graph_ms(fn, reps):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        kd_batch.fill_(-1)
        ms = timed(g.replay, reps)
        if not torch.equal(kd_batch, ref_k):
            raise RuntimeError("graph replay changed the component counts")
        return ms

    reps = max(2, min(args.steps, 5))
    res = {"workload": f"{len(imgs)} uint8 images, H and W each log-uniform in [64, 2048], "
                       "p ~ U(0.2, 0.8), half Bernoulli / half sigma in {2,4,8} blobs, seed 100",
           "images": len(imgs), "pixels": int(px)}
    with torch.cuda.stream(stream):
        ms_single = timed(per_image, reps)
        ref_k = kd_single.clone()
        status()
        out = {}
        for mode, tag in ((0, "tuned"), (2, "persistent"), (1, "three_launches")):
            lib.ccl_set_launch_mode(mode)
            kd_batch.fill_(-1)
            ms_b = timed(batched, reps)
            if not torch.equal(kd_batch, ref_k):
                raise RuntimeError(f"{tag} batch and per-image component counts differ")
            ms_g = graph_ms(batched, reps)
            status()
            out[tag] = {"ms": round(ms_b, 3), "graph_ms": round(ms_g, 3),
                        "gpx_s": round(px / ms_b / 1e6, 2), "gpx_s_graph": round(px / ms_g / 1e6, 2)}
        # a 64-image batch (the first 64 images) both ways, as a CUDA graph
        sub, sub_labs = imgs[:64], labs[:64]
        sub_px = sum(t.numel() for t in sub)
        k64 = torch.zeros(64, dtype=torch.int32, device=dev)
        small = {}
        for mode, tag in ((0, "tuned"), (2, "persistent"), (1, "three_launches")):
            lib.ccl_set_launch_mode(mode)

            def b64():
                ccl.label_batch(sub, connectivity=args.connectivity, outs=sub_labs, stream=stream, k_out=k64)

            b64()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                b64()
            ms = timed(g.replay, 20)
            if not torch.equal(k64, ref_k[:64]):
                raise RuntimeError("64-image batch component counts differ")
            small[tag] = {"graph_ms": round(ms, 4), "gpx_s": round(sub_px / ms / 1e6, 2)}
        lib.ccl_set_launch_mode(0)
        status()
    res.update({"per_image_ms": round(ms_single, 3), "gpx_s_per_image": round(px / ms_single / 1e6, 2),
                "batched_ms": out["tuned"]["ms"], "batched_graph_ms": out["tuned"]["graph_ms"],
                "gpx_s_batched": out["tuned"]["gpx_s"], "gpx_s_batched_graph": out["tuned"]["gpx_s_graph"],
                "speedup_batched_graph_vs_per_image": round(ms_single / out["tuned"]["graph_ms"], 2),
                "modes": out, "batch64": {"pixels": int(sub_px), **small},
                "how": "per-image: one ccl_label_async call per image; tuned: one ccl_label_batch call in the "
                       "launch form the tuning table gives its size class; persistent / three_launches: the same "
                       "call forced to one cooperative launch (ccl_set_launch_mode(2)) or three launches (1)"})
    return res


# ---- CPU oracle ---------------------------------------------------------------------------

def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample(host_imgs, rows):
    """The CPU legs' bounded sample: the first `rows` rows of every image of the workload
    (whole images when they are shorter)."""
    return [np.ascontiguousarray(im[:rows]) for im in host_imgs]


def time_leg(fn, sample, runs):
    """Median and p99 of `runs` timings of labelling every image of `sample` once."""
    secs = []
    for _ in range(runs):
        t0 = time.perf_counter()
        for im in sample:
            fn(im)
        secs.append(time.perf_counter() - t0)
    secs.sort()
    return statistics.median(secs), secs[min(len(secs) - 1, int(0.99 * len(secs)))]


def thread_counts(nthr):
    out, t = [], 1
    while t < nthr:
        out.append(t)
        t *= 2
    out.append(nthr)
    return out


def cpu_baseline(dev_imgs, args):
    """The oracle as it stands on the host's cores, on a bounded sample of the workload
    (the first rows of every image, about 10-30 s of CPU work in all): PARemSP (Algorithm
    7) at 1, 2, 4, ... and all threads, ARemSP (Algorithm 5, the paper's best sequential
    algorithm, Table II) and CCLRemSP (Algorithm 1) on one thread.  Each leg is the median
    of 3 runs over the sample (std::chrono-free: Python's perf_counter around the C call);
    the canonical renumbering of ARemSP / PARemSP is excluded (timed separately)."""
    import oracle

    orc = oracle.default()
    nthr = cpu_threads()
    conn = args.connectivity
    host = [t.cpu().numpy() for t in dev_imgs]
    rows = max(1, min(im.shape[0] for im in host) // 4) if host[0].size > (1 << 26) else host[0].shape[0]
    sample = cpu_sample(host, rows)
    px = sum(im.size for im in sample)
    runs = 3

    def leg(fn, cores, algorithm):
        med, p99 = time_leg(fn, sample, runs)
        return {"value": round(px / med / 1e9, 4), "cores": cores, "median_s": round(med, 4),
                "p99_s": round(p99, 4), "runs": runs, "algorithm": algorithm}

    desc = (f"the first {rows} rows of each of the {len(host)} image(s) of the workload "
            f"({px / 1e6:.1f} Mpx), each leg the median of {runs} runs")
    if conn != 8:  # PARemSP (Algorithm 7) is stated for 8-connectivity only
        c = leg(lambda im: orc.cclremsp(im, conn), 1, f"CCLRemSP (Algorithm 1), {conn}-connectivity")
        return {"value": c["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "algorithm": c["algorithm"], "sample": desc, "legs": {"cclremsp": c}}
    legs = {}
    for t in thread_counts(nthr):
        legs[f"paremsp_t{t}"] = leg(lambda im, t=t: orc.paremsp(im, t, remap=False), t,
                                    f"PARemSP (Algorithm 7) on {t} OpenMP thread(s)")
    legs["aremsp"] = leg(lambda im: orc.aremsp(im, remap=False), 1, "ARemSP (Algorithm 5), one thread")
    legs["cclremsp"] = leg(lambda im: orc.cclremsp(im), 1, "CCLRemSP (Algorithm 1), one thread")
    t0 = time.perf_counter()
    for im in sample:
        lab, k = orc.aremsp(im, remap=False)
        orc.canonicalize(lab, k)
    remap_s = time.perf_counter() - t0
    top = legs[f"paremsp_t{nthr}"]
    return {"value": top["value"], "unit": UNIT, "cores": nthr, "kind": "oracle",
            "algorithm": "PARemSP (Algorithm 7) on all host threads, canonical renumbering excluded",
            "sample": desc, "cpu_model": cpu_model(), "legs": legs,
            "speedup_paremsp_vs_aremsp": round(top["value"] / legs["aremsp"]["value"], 2),
            "aremsp_plus_renumbering_s": round(remap_s, 4)}


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo; Arm hosts list implementer and part)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    if "cpu part" in fields:
        return f"{os.uname().machine} (CPU implementer {fields.get('cpu implementer', '?')}, part {fields['cpu part']})"
    return os.uname().machine


def run_reference(args, rank, world):
    """The oracle as the reference arm: PARemSP (Algorithm 7) on the host's threads over
    the same images as our arm (identical bytes: the SHA-256s are in both lines), one image
    of the workload per step, round robin."""
    if rank != 0:
        return None
    if args.connectivity != 8:
        return {"impl": "reference", "unavailable": "PARemSP (Algorithm 7) is stated for 8-connectivity only"}
    import oracle

    orc = oracle.default()
    nthr = cpu_threads()
    pairs = workload_images(args.workload)
    host = [im for _, im in pairs]
    desc = {**WORKLOAD_DESC[args.workload], "inputs_sha256": {n: synth.sha256(im) for n, im in pairs}}
    for i in range(args.warmup):
        orc.paremsp(host[i % len(host)], nthr, remap=False)
    px, t0 = 0, time.perf_counter()
    for i in range(args.steps):
        im = host[i % len(host)]
        orc.paremsp(im, nthr, remap=False)
        px += im.size
    secs = time.perf_counter() - t0
    v = px / secs / 1e9
    return {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8->int32", "data": "synthetic", "impl": "reference",
            "config": {**desc, "parallelism": f"{nthr} OpenMP threads"},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": nthr, "kind": "oracle",
                             "sample": "one whole image of the workload per step, round robin"},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["big21568", "sweep8192", "small1024"], default="big21568")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the sweep8192 / small1024 extra keys")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--streams", type=int, default=3,
                    help="streams the images of a step alternate over (timed pass)")
    ap.add_argument("--global-ctas-per-sm", type=int, default=1,
                    help="cap on the global kernel's CTAs per SM during the timed pass "
                         "(ccl_set_global_ctas_per_sm; 0 = as many as fit)")
    ap.add_argument("--connectivity", type=int, choices=[8, 4], default=8,
                    help="8 (the paper's) or 4; the reference arm supports 8 only")
    ap.add_argument("--only", default=None, help="keep one image of the workload (profiling)")
    ap.add_argument("--side", type=int, default=None,
                    help="big21568 only: the same three images at a smaller side (profiling captures)")
    ap.add_argument("--batch-images", type=int, default=4096,
                    help="size of the uneven-batch comparison (0 skips it)")
    ap.add_argument("--no-served", dest="served", action="store_false", help="skip the serving measurement")
    ap.add_argument("--no-fused", dest="fused", action="store_false", help="skip the fused-binarisation measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
