"""Helpers for GPU tests: run the library through its C ABI on numpy images."""
from __future__ import annotations

import ctypes

import numpy as np

import synth


def stream_handle():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def run_label(img: np.ndarray, lib=None, pitch: int | None = None, offset: int = 0,
              label_offset: int = 0, fill: int = 7, conn: int = 8):
    """Copy ``img`` to the device (rows of ``pitch`` bytes, padding bytes = ``fill``,
    starting ``offset`` bytes into the buffer), call ``ccl_label`` and return
    (status, labels, K, device status flags)."""
    import torch

    import paper_1606_05973_gb300 as ccl

    lib = lib or ccl.lib()
    h, w = img.shape
    pitch = pitch or max(w, 1)
    nbytes = offset + h * pitch + 16
    buf = torch.full((nbytes,), fill, dtype=torch.uint8, device="cuda")
    if h and w:
        host = synth.pad_pitch(np.ascontiguousarray(img), pitch, fill).reshape(-1)
        buf[offset:offset + h * pitch].copy_(torch.from_numpy(host))
    labels = torch.full((h * w + label_offset + 4,), -5, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(-1)
    s = stream_handle()
    rc = lib.ccl_label(ctypes.c_void_p(buf.data_ptr() + offset), h, w, pitch, conn,
                       ctypes.c_void_p(labels.data_ptr() + 4 * label_offset), ctypes.byref(k), s)
    flags = ctypes.c_int32(0)
    lib.ccl_device_status(s, ctypes.byref(flags))
    torch.cuda.synchronize()
    out = labels[label_offset:label_offset + h * w].view(h, w).cpu().numpy() if h * w else np.zeros((h, w), np.int32)
    return rc, out, k.value, flags.value


def mosaic_4x4_all():
    """Every 4x4 binary image (65536 of them) on a 256 x 256 grid, separated by one empty
    row and column, as one 1279 x 1279 image."""
    bits = np.arange(1 << 16, dtype=np.uint32)
    tiles = ((bits[:, None] >> np.arange(16, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    tiles = tiles.reshape(256, 256, 4, 4)
    big = np.zeros((256, 5, 256, 5), dtype=np.uint8)
    big[:, :4, :, :4] = tiles.transpose(0, 2, 1, 3)
    return np.ascontiguousarray(big.reshape(1280, 1280)[:1279, :1279])
