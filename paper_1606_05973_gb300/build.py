"""Builds the CUDA library ``libccl.so`` (sm_103a) in-tree with nvcc.

``python -m paper_1606_05973_gb300.build`` or ``build()`` from Python.  The translation
units compile in parallel; the shared object lands in ``paper_1606_05973_gb300/_build``.
``debug=True`` builds ``libccl_debug.so`` with device-side index checks (CCL_DEBUG): an
out-of-range index sets a status bit and the access is skipped.
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SOURCES = ["ccl_kernels.cu", "ccl_api.cu", "ccl_static.cu", "ccl_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def lib_path(debug: bool = False) -> str:
    return os.path.join(OUT, "libccl_debug.so" if debug else "libccl.so")


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "ccl.h"))
    deps.append(os.path.abspath(__file__))
    deps.append(TUNING)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


TUNING = os.path.join(HERE, "tuning.json")
SHAPES = {"64x128": 0, "64x256": 1}


def tuning_source(path: str = TUNING) -> str:
    """The tuning table as C (the initialisers ccl_kernels.cu includes)."""
    with open(path) as f:
        t = json.load(f)
    lo, hi = (int(round(1024 * float(b))) for b in t["density_bounds"])
    rows = []
    for r in t["rows"]:
        shape = [SHAPES[x] for x in r["shape"]]
        assert len(shape) == 3 and int(r["ctas_per_sm"]) >= 1
        mx = -1 if r["max_px"] is None else int(r["max_px"])
        pers = 1 if r.get("persistent", True) else 0
        rows.append(f"    {{{mx}LL, {{{shape[0]}, {shape[1]}, {shape[2]}}}, {int(r['ctas_per_sm'])}, {pers}}},")
    assert rows and t["rows"][-1]["max_px"] is None, "the last row must have no bound"
    return "\n".join([
        "// written by paper_1606_05973_gb300/build.py from tuning.json; do not edit",
        "static const TuneRow kTuneRows[] = {", *rows, "};",
        f"static const int kTuneDensLo = {lo}, kTuneDensHi = {hi};",
        f"static const int kTuneProbeSamples = {int(t['probe_samples'])};",
        f"static const int64_t kTuneSingleFusedMaxPx = {int(t['single_fused_max_px'])}LL;",
        f"static const int64_t kTuneStreamsMinPx = {int(t.get('streams_min_px', -1))}LL;", ""])


def write_tuning_include() -> str:
    os.makedirs(OUT, exist_ok=True)
    path = os.path.join(OUT, "ccl_tuning.inc")
    src = tuning_source()
    if not os.path.exists(path) or open(path).read() != src:
        with open(path, "w") as f:
            f.write(src)
    return path


def build(debug: bool = False, force: bool = False, verbose: bool = False) -> str:
    target = lib_path(debug)
    write_tuning_include()
    if not force and not _stale(target):
        return target
    os.makedirs(OUT, exist_ok=True)
    tag = "dbg" if debug else "rel"
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
             "--expt-relaxed-constexpr", "-I", OUT, *ARCH]
    if debug:
        flags.append("-DCCL_DEBUG")
    if verbose:
        flags += ["-Xptxas", "-v"]
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, f"{os.path.splitext(src)[0]}.{tag}.o")
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = target + ".tmp"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    dbg = "--debug" in sys.argv
    print(build(debug=dbg, force="--force" in sys.argv, verbose="-v" in sys.argv))
