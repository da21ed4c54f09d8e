"""CPU oracle for connected-component labelling (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use this
package.  The GPU library never imports it and shares no code with it.

The C source ``ccl_oracle.c`` follows the paper's algorithms (CCLRemSP, Algorithms 1-4;
ARemSP, Algorithms 5-6; PARemSP, Algorithms 7-8) plus a flood fill from the definition.
It is compiled on demand with gcc into ``oracle/_build/``.

Every function returns ``(labels, K)``: ``labels`` is an int32 (H, W) array with
background 0 and components numbered 1..K in raster order of their first pixel.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libccl_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(src: str = _SRC, out: str = _SO, extra=()) -> str:
    """Compile a C oracle source into a shared object (plain gcc, OpenMP)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", out, src, *extra]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_oracle()
    return _SO


def load(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.oracle_cclremsp.argtypes = [p, i64, i64, i64, i32, p]
    lib.oracle_aremsp.argtypes = [p, i64, i64, i64, p, i32]
    lib.oracle_paremsp.argtypes = [p, i64, i64, i64, p, i32, i32]
    lib.oracle_bfs.argtypes = [p, i64, i64, i64, i32, p]
    lib.oracle_bfs_classes.argtypes = [p, i64, i64, i64, i32, p]
    lib.oracle_canonicalize.argtypes = [p, i64, i64]
    for f in (lib.oracle_cclremsp, lib.oracle_aremsp, lib.oracle_paremsp, lib.oracle_bfs,
              lib.oracle_bfs_classes, lib.oracle_canonicalize):
        f.restype = i64
    lib.oracle_max_threads.restype = i32
    lib.oracle_max_threads.argtypes = []
    return lib


def _get():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


class Oracle:
    """Binds one compiled oracle object (the default one, or a test variant)."""

    def __init__(self, lib: ctypes.CDLL):
        self.lib = lib

    @staticmethod
    def _prep(img: np.ndarray):
        img = np.asarray(img)
        if img.dtype != np.uint8 or img.ndim != 2:
            raise TypeError("image must be a 2-D uint8 array")
        if img.strides[1] != 1 or img.strides[0] < img.shape[1]:
            img = np.ascontiguousarray(img)
        h, w = img.shape
        pitch = img.strides[0] if h > 0 else w
        labels = np.zeros((h, w), dtype=np.int32)
        return img, h, w, pitch, labels

    @staticmethod
    def _check(k):
        if k < 0:
            raise RuntimeError(f"oracle error {k}")
        return int(k)

    def cclremsp(self, img, conn: int = 8):
        img, h, w, pitch, lab = self._prep(img)
        k = self.lib.oracle_cclremsp(img.ctypes.data, h, w, pitch, conn, lab.ctypes.data)
        return lab, self._check(k)

    def aremsp(self, img, remap: bool = True):
        img, h, w, pitch, lab = self._prep(img)
        k = self.lib.oracle_aremsp(img.ctypes.data, h, w, pitch, lab.ctypes.data, int(remap))
        return lab, self._check(k)

    def paremsp(self, img, threads: int = 0, remap: bool = True):
        img, h, w, pitch, lab = self._prep(img)
        t = threads if threads > 0 else self.lib.oracle_max_threads()
        k = self.lib.oracle_paremsp(img.ctypes.data, h, w, pitch, lab.ctypes.data, t, int(remap))
        return lab, self._check(k)

    def bfs(self, img, conn: int = 8):
        img, h, w, pitch, lab = self._prep(img)
        k = self.lib.oracle_bfs(img.ctypes.data, h, w, pitch, conn, lab.ctypes.data)
        return lab, self._check(k)

    def bfs_classes(self, img, conn: int = 8):
        img, h, w, pitch, lab = self._prep(img)
        k = self.lib.oracle_bfs_classes(img.ctypes.data, h, w, pitch, conn, lab.ctypes.data)
        return lab, self._check(k)

    def canonicalize(self, labels: np.ndarray, k: int):
        lab = np.ascontiguousarray(labels, dtype=np.int32).copy()
        kk = self.lib.oracle_canonicalize(lab.ctypes.data, lab.size, int(k))
        return lab, self._check(kk)

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())


def default() -> Oracle:
    return Oracle(_get())


def classes(img, conn: int = 8):
    """Multi-class labelling: neighbours connect when their bytes are equal and non-zero;
    canonical numbering (raster order of first pixels)."""
    return default().bfs_classes(img, conn)


def binarize(img, threshold: int) -> np.ndarray:
    """Fused binarisation's input, written out: object = byte > threshold (Section V
    binarises with im2bw(0.5), i.e. byte > 127.5 on 8-bit data: threshold 127)."""
    return (np.asarray(img, dtype=np.uint8) > int(threshold)).astype(np.uint8)


def cclremsp(img, conn: int = 8):
    """CCLRemSP (Algorithm 1): canonical labels of ``img`` under ``conn``-connectivity."""
    return default().cclremsp(img, conn)


def aremsp(img, remap: bool = True):
    """ARemSP (Algorithm 5), renumbered to the canonical order when ``remap``."""
    return default().aremsp(img, remap)


def paremsp(img, threads: int = 0, remap: bool = True):
    """PARemSP (Algorithm 7) on ``threads`` OpenMP threads (0 = all)."""
    return default().paremsp(img, threads, remap)


def bfs(img, conn: int = 8):
    """Flood fill from the definition, canonical numbering."""
    return default().bfs(img, conn)


def label(img, conn: int = 8):
    """The oracle's answer: CCLRemSP for 8- and 4-connectivity."""
    return cclremsp(img, conn)
