"""Builds and drives the host emulation of the GPU path (tests only).

``build(sanitize)`` compiles tests/emu/ccl_emu.cpp with g++ (optionally with
AddressSanitizer and UBSan); ``Emu(path).label(img, seed, shape)`` runs it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "ccl_emu.cpp")
CORE = os.path.join(HERE, "..", "..", "paper_1606_05973_gb300", "csrc", "ccl_core.cuh")

SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined"]


def asan_runtime() -> str | None:
    r = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True)
    p = r.stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def build(sanitize: bool = True) -> str:
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libccl_emu_san.so" if sanitize else "libccl_emu.so")
    newest = max(os.path.getmtime(SRC), os.path.getmtime(CORE))
    if os.path.exists(so) and os.path.getmtime(so) >= newest:
        return so
    # the global kernel's CTA size is reduced for the emulator (one OS thread per CUDA thread)
    cmd = ["g++", "-std=c++20", "-O1", "-g", "-DCCL_DEBUG", "-DCCL_GLOBAL_NT=64", "-shared", "-fPIC",
           "-o", so, SRC]
    if sanitize:
        cmd[1:1] = SAN
    subprocess.run(cmd, check=True)
    return so


class Emu:
    def __init__(self, path: str):
        self.lib = ctypes.CDLL(path)
        f = self.lib.emu_label
        f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                      ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p]
        f.restype = ctypes.c_int64
        fb = self.lib.emu_label_batch
        fb.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p]
        fb.restype = None
        ff = self.lib.emu_label_fused
        ff.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p,
                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        ff.restype = None
        self.lib.emu_set_threshold.argtypes = [ctypes.c_int32]
        self.lib.emu_gt_mask16.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        self.lib.emu_gt_mask16.restype = ctypes.c_uint32
        self.lib.emu_eq_nibble.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        self.lib.emu_eq_nibble.restype = ctypes.c_uint32

    def gt_mask16(self, src16: np.ndarray, threshold: int) -> int:
        """The load phase's test of 16 bytes: bit i set when byte i > threshold."""
        src16 = np.ascontiguousarray(src16, dtype=np.uint8)
        assert src16.size == 16
        return int(self.lib.emu_gt_mask16(src16.ctypes.data, int(threshold)))

    def label(self, img: np.ndarray, seed: int = 1, shape: int = 0, pitch: int | None = None, fill: int = 7,
              threshold: int = 0):
        import synth

        self.lib.emu_set_threshold(int(threshold))

        h, w = img.shape
        if pitch is None:
            src = np.ascontiguousarray(img)
            pitch = max(w, 1)
        else:
            src = synth.pad_pitch(img, pitch, fill)
        lab = np.full((h, w), -7, np.int32)
        st = np.zeros(1, np.int32)
        k = self.lib.emu_label(src.ctypes.data, h, w, pitch, lab.ctypes.data, seed, shape, st.ctypes.data)
        return lab, int(k), int(st[0])

    def label_batch(self, imgs, seed: int = 1, shape: int = 1):
        """Batched path on a list of non-empty images; returns (labels list, K list, status)."""
        n = len(imgs)
        srcs = [np.ascontiguousarray(im) for im in imgs]
        labs = [np.full(im.shape, -7, np.int32) for im in srcs]
        P = ctypes.c_void_p * n
        ip = P(*[im.ctypes.data for im in srcs])
        lp = P(*[lb.ctypes.data for lb in labs])
        H = np.array([im.shape[0] for im in srcs], np.int32)
        W = np.array([im.shape[1] for im in srcs], np.int32)
        pitch = np.array([im.shape[1] for im in srcs], np.int64)
        K = np.full(n, -1, np.int32)
        st = np.zeros(1, np.int32)
        self.lib.emu_label_batch(n, ip, H.ctypes.data, W.ctypes.data, pitch.ctypes.data, lp, K.ctypes.data,
                                 seed, shape, st.ctypes.data)
        return labs, [int(k) for k in K], int(st[0])

    def label_fused(self, imgs, seed: int = 1, pair: int = 0, pick=(0, 0, 0), lo: int = 0, hi: int = 0,
                    probe: int = 0, ctas: int = 3, threshold: int = 0):
        """Persistent single-launch path (fused_body) on a list of non-empty images; returns
        (labels list, K list, status)."""
        self.lib.emu_set_threshold(int(threshold))
        n = len(imgs)
        srcs = [np.ascontiguousarray(im) for im in imgs]
        labs = [np.full(im.shape, -7, np.int32) for im in srcs]
        P = ctypes.c_void_p * n
        ip = P(*[im.ctypes.data for im in srcs])
        lp = P(*[lb.ctypes.data for lb in labs])
        H = np.array([im.shape[0] for im in srcs], np.int32)
        W = np.array([im.shape[1] for im in srcs], np.int32)
        pitch = np.array([im.shape[1] for im in srcs], np.int64)
        K = np.full(n, -1, np.int32)
        st = np.zeros(1, np.int32)
        pk = np.array(pick, np.int32)
        self.lib.emu_label_fused(n, ip, H.ctypes.data, W.ctypes.data, pitch.ctypes.data, lp, K.ctypes.data,
                                 seed, pair, pk.ctypes.data, lo, hi, probe, ctas, st.ctypes.data)
        return labs, [int(k) for k in K], int(st[0])
