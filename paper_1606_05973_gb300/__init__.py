"""Python binding of ``libccl`` (GB300 connected-component labelling, PARemSP method).

This module only marshals arguments: every step of the labelling runs in the library's
CUDA kernels.  The C-ABI functions keep their C names (``ccl_label``, ``ccl_label_async``,
``ccl_label_host``, ``ccl_label_batch``, ...) and take plain integers for pointers and
streams.  ``label``/``label_batch``/``label_host`` are conveniences over torch tensors.

There is no CPU fallback: if the compiled library is missing the import of any entry
point raises ``CCLUnavailable``.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import build, lib_path

__all__ = [
    "CCLError", "CCLUnavailable", "load", "lib", "ccl_label", "ccl_label_async", "ccl_label_static", "ccl_label_static_status", "ccl_shutdown",
    "ccl_label_host", "ccl_label_batch", "ccl_workspace_bytes", "ccl_device_status", "ccl_release", "ccl_set_global_ctas_per_sm",
    "ccl_set_tile_policy",
    "ccl_profile_enable", "ccl_profile_reset", "ccl_profile_read", "ccl_status_string",
    "ccl_version", "label", "label_batch", "label_host", "kernel_times", "CCL_OK", "Server",
    "ccl_server_create", "ccl_server_submit", "ccl_server_wait", "ccl_server_get_stats",
    "ccl_server_reset_stats", "ccl_server_destroy",
]

CCL_OK = 0
STATUS_NAMES = {0: "CCL_OK", 1: "CCL_ERR_INVALID_ARGUMENT", 2: "CCL_ERR_UNSUPPORTED",
                3: "CCL_ERR_OUT_OF_MEMORY", 4: "CCL_ERR_CUDA", 5: "CCL_ERR_TIMEOUT",
                6: "CCL_ERR_BUSY", 7: "CCL_ERR_INTERNAL", 8: "CCL_ERR_TOO_LARGE"}


class CCLError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class CCLUnavailable(RuntimeError):
    pass


class ImageDesc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int64), ("labels", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_int64), ("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("connectivity", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("pixels", ctypes.c_int64), ("elapsed_s", ctypes.c_double),
                ("gpx_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("peak_inflight_bytes", ctypes.c_int64),
                ("peak_queue", ctypes.c_int32), ("peak_busy_lanes", ctypes.c_int32)]


class TuneRow(ctypes.Structure):
    _fields_ = [("max_px", ctypes.c_int64), ("shape", ctypes.c_int32 * 3), ("ctas_per_sm", ctypes.c_int32),
                ("persistent", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lock = threading.Lock()
_libs: dict = {}

_P, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "ccl_status_string": ([_I32], ctypes.c_char_p),
    "ccl_version": ([], _I32),
    "ccl_label": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_async": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_static": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_static_status": ([_P, _P], _I32),
    "ccl_label_host": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_host_async": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_batch": ([_P, _I32, _I32, _P, _P], _I32),
    "ccl_label_threshold": ([_P, _I32, _I32, _I64, _I32, _I32, _P, _P, _P], _I32),
    "ccl_label_batch_threshold": ([_P, _I32, _I32, _I32, _P, _P], _I32),
    "ccl_label_classes": ([_P, _I32, _I32, _I64, _I32, _P, _P, _P], _I32),
    "ccl_label_batch_classes": ([_P, _I32, _I32, _P, _P], _I32),
    "ccl_workspace_bytes": ([_I32, _I32, _P], _I32),
    "ccl_device_status": ([_P, _P], _I32),
    "ccl_release": ([], _I32),
    "ccl_shutdown": ([], _I32),
    "ccl_set_global_ctas_per_sm": ([_I32], _I32),
    "ccl_set_tile_policy": ([_I32], _I32),
    "ccl_set_launch_mode": ([_I32], _I32),
    "ccl_set_streams_min_px": ([_I64], _I32),
    "ccl_set_persistent_ctas_per_sm": ([_I32], _I32),
    "ccl_set_tuning": ([_P, _I32, _I32, _I32, _I32, _I64], _I32),
    "ccl_profile_enable": ([_I32], _I32),
    "ccl_profile_reset": ([], _I32),
    "ccl_profile_read": ([_P, _I32, _P], _I32),
    "ccl_server_create": ([_P, _P], _I32),
    "ccl_server_submit": ([_P, _P, _P], _I32),
    "ccl_server_wait": ([_P, ctypes.c_uint64, _P, _I32], _I32),
    "ccl_server_get_stats": ([_P, _P], _I32),
    "ccl_server_reset_stats": ([_P], _I32),
    "ccl_server_destroy": ([_P], _I32),
}


def load(debug: bool = False, path: str | None = None, allow_build: bool = True) -> ctypes.CDLL:
    """Load (building it first when missing) the compiled library."""
    key = path or ("debug" if debug else "release")
    with _lock:
        if key in _libs:
            return _libs[key]
        p = path or lib_path(debug)
        if not os.path.exists(p):
            if not allow_build:
                raise CCLUnavailable(f"compiled CUDA library not found at {p}")
            try:
                p = build(debug=debug)
            except Exception as e:  # noqa: BLE001 - surface the build failure loudly
                raise CCLUnavailable(f"cannot build the CUDA library: {e}") from e
        h = ctypes.CDLL(p)
        for name, (args, res) in _SIGS.items():
            f = getattr(h, name)
            f.argtypes = args
            f.restype = res
        _libs[key] = h
        return h


def lib() -> ctypes.CDLL:
    return load()


# ---- C-ABI entry points, same names and argument order as include/ccl.h ----------------

def ccl_status_string(status: int) -> str:
    return lib().ccl_status_string(status).decode()


def ccl_version() -> int:
    return lib().ccl_version()


def ccl_label(img, H, W, pitch_bytes, connectivity, labels, num_components, stream) -> int:
    return lib().ccl_label(img, H, W, pitch_bytes, connectivity, labels, num_components, stream)


def ccl_label_async(img, H, W, pitch_bytes, connectivity, labels, num_components_dev, stream) -> int:
    return lib().ccl_label_async(img, H, W, pitch_bytes, connectivity, labels, num_components_dev, stream)


def ccl_label_static(img, H, W, pitch_bytes, connectivity, labels, num_components_dev, stream) -> int:
    """ccl_label_async without any device allocation (fixed 16 MiB scratch in the library);
    for callers that may not allocate device memory."""
    return lib().ccl_label_static(img, H, W, pitch_bytes, connectivity, labels, num_components_dev, stream)


def ccl_label_static_status(stream, flags_ptr) -> int:
    """Read and clear the status word of ccl_label_static's fixed scratch (no allocation)."""
    return lib().ccl_label_static_status(stream, flags_ptr)


def ccl_label_host(img_host, H, W, pitch_bytes, connectivity, labels_host, num_components, stream) -> int:
    return lib().ccl_label_host(img_host, H, W, pitch_bytes, connectivity, labels_host, num_components, stream)


def ccl_label_host_async(img_host, H, W, pitch_bytes, connectivity, labels_host, num_components_host,
                         stream) -> int:
    return lib().ccl_label_host_async(img_host, H, W, pitch_bytes, connectivity, labels_host,
                                      num_components_host, stream)


def ccl_label_batch(imgs, n, connectivity, num_components_dev, stream) -> int:
    return lib().ccl_label_batch(imgs, n, connectivity, num_components_dev, stream)


def ccl_label_threshold(img, H, W, pitch_bytes, connectivity, threshold, labels, num_components, stream) -> int:
    return lib().ccl_label_threshold(img, H, W, pitch_bytes, connectivity, threshold, labels, num_components, stream)


def ccl_label_batch_threshold(imgs, n, connectivity, threshold, num_components_dev, stream) -> int:
    return lib().ccl_label_batch_threshold(imgs, n, connectivity, threshold, num_components_dev, stream)


def ccl_label_classes(img, H, W, pitch_bytes, connectivity, labels, num_components, stream) -> int:
    return lib().ccl_label_classes(img, H, W, pitch_bytes, connectivity, labels, num_components, stream)


def ccl_label_batch_classes(imgs, n, connectivity, num_components_dev, stream) -> int:
    return lib().ccl_label_batch_classes(imgs, n, connectivity, num_components_dev, stream)


def ccl_workspace_bytes(H, W, bytes_ptr) -> int:
    return lib().ccl_workspace_bytes(H, W, bytes_ptr)


def ccl_device_status(stream, flags_ptr) -> int:
    return lib().ccl_device_status(stream, flags_ptr)


def ccl_release() -> int:
    return lib().ccl_release()


def ccl_shutdown() -> int:
    return lib().ccl_shutdown()


def ccl_set_global_ctas_per_sm(n) -> int:
    return lib().ccl_set_global_ctas_per_sm(n)


def ccl_set_tile_policy(policy) -> int:
    return lib().ccl_set_tile_policy(policy)


def ccl_profile_enable(on) -> int:
    return lib().ccl_profile_enable(on)


def ccl_profile_reset() -> int:
    return lib().ccl_profile_reset()


def ccl_profile_read(out, max_entries, count_ptr) -> int:
    return lib().ccl_profile_read(out, max_entries, count_ptr)


def ccl_server_create(cfg, out_ptr) -> int:
    return lib().ccl_server_create(cfg, out_ptr)


def ccl_server_submit(srv, img_desc, id_ptr) -> int:
    return lib().ccl_server_submit(srv, img_desc, id_ptr)


def ccl_server_wait(srv, request_id, k_ptr, timeout_ms) -> int:
    return lib().ccl_server_wait(srv, request_id, k_ptr, timeout_ms)


def ccl_server_get_stats(srv, out) -> int:
    return lib().ccl_server_get_stats(srv, out)


def ccl_server_reset_stats(srv) -> int:
    return lib().ccl_server_reset_stats(srv)


def ccl_server_destroy(srv) -> int:
    return lib().ccl_server_destroy(srv)


class Server:
    """Continuous-batching server (ccl_server_*): submit device images, wait for K."""

    def __init__(self, mem_cap_bytes: int = 16 << 30, lanes: int = 3, max_batch: int = 64, max_pending: int = 0,
                 connectivity: int = 8):
        cfg = ServerConfig(mem_cap_bytes, lanes, max_batch, max_pending, connectivity)
        h = ctypes.c_void_p()
        _check(ccl_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ccl_server_create")
        self.h = h

    def submit(self, img, labels) -> int:
        """img: 2-D uint8 CUDA tensor (stride(1) == 1); labels: contiguous int32 (H, W)."""
        H, W = img.shape
        d = ImageDesc(img.data_ptr(), H, W, img.stride(0) if H > 0 else W, labels.data_ptr())
        rid = ctypes.c_uint64(0)
        _check(ccl_server_submit(self.h, ctypes.byref(d), ctypes.byref(rid)), "ccl_server_submit")
        return int(rid.value)

    def wait(self, request_id: int, timeout_ms: int = -1) -> int:
        k = ctypes.c_int32(-1)
        _check(ccl_server_wait(self.h, request_id, ctypes.byref(k), timeout_ms), "ccl_server_wait")
        return int(k.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(ccl_server_get_stats(self.h, ctypes.byref(st)), "ccl_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(ccl_server_reset_stats(self.h), "ccl_server_reset_stats")

    def close(self):
        if self.h:
            _check(ccl_server_destroy(self.h), "ccl_server_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- torch conveniences (marshalling only) ------------------------------------------------

def _check(rc: int, where: str):
    if rc != CCL_OK:
        raise CCLError(rc, where)


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def label(img, connectivity: int = 8, out=None, stream=None, sync: bool = True, threshold: int | None = None,
          classes: bool = False):
    """Label a 2-D uint8 CUDA tensor (rows may be padded: stride(1) must be 1).

    Returns ``(labels, K)`` with ``labels`` an int32 (H, W) CUDA tensor.  With ``sync=False``
    K is returned as a 1-element int32 CUDA tensor and nothing waits for the stream.  With
    ``threshold`` set, object pixels are bytes greater than it (ccl_label_threshold); with
    ``classes``, neighbours connect when their bytes are equal and non-zero
    (ccl_label_classes).
    """
    import torch

    if img.dtype != torch.uint8 or img.dim() != 2 or not img.is_cuda:
        raise TypeError("img must be a 2-D uint8 CUDA tensor")
    if img.stride(1) != 1:
        img = img.contiguous()
    H, W = img.shape
    pitch = img.stride(0) if H > 0 else W
    if out is None:
        out = torch.empty((H, W), dtype=torch.int32, device=img.device)
    elif out.dtype != torch.int32 or tuple(out.shape) != (H, W) or not out.is_contiguous():
        raise TypeError("out must be a contiguous int32 (H, W) tensor")
    s = _stream_ptr(stream)
    if classes:
        if not sync or threshold is not None:
            raise ValueError("classes labelling returns K on the host and takes no threshold")
        k = ctypes.c_int32(-1)
        _check(ccl_label_classes(img.data_ptr(), H, W, pitch, connectivity, out.data_ptr(), ctypes.byref(k), s),
               "ccl_label_classes")
        return out, int(k.value)
    if threshold is not None:
        if not sync:
            raise ValueError("threshold labelling returns K on the host (sync=True)")
        k = ctypes.c_int32(-1)
        _check(ccl_label_threshold(img.data_ptr(), H, W, pitch, connectivity, int(threshold), out.data_ptr(),
                                   ctypes.byref(k), s), "ccl_label_threshold")
        return out, int(k.value)
    if sync:
        k = ctypes.c_int32(-1)
        _check(ccl_label(img.data_ptr(), H, W, pitch, connectivity, out.data_ptr(), ctypes.byref(k), s),
               "ccl_label")
        return out, int(k.value)
    kd = torch.empty(1, dtype=torch.int32, device=img.device)
    _check(ccl_label_async(img.data_ptr(), H, W, pitch, connectivity, out.data_ptr(), kd.data_ptr(), s),
           "ccl_label_async")
    return out, kd


def label_batch(imgs, connectivity: int = 8, outs=None, stream=None, k_out=None, threshold: int | None = None,
                classes: bool = False):
    """Label a list of 2-D uint8 CUDA tensors in one call.  Returns (labels list, K tensor).
    With ``threshold`` set, object pixels are bytes greater than it."""
    import torch

    n = len(imgs)
    dev = imgs[0].device if n else torch.device("cuda")
    if outs is None:
        outs = [torch.empty(tuple(im.shape), dtype=torch.int32, device=dev) for im in imgs]
    descs = (ImageDesc * max(n, 1))()
    keep = []
    for i, im in enumerate(imgs):
        if im.stride(1) != 1:
            im = im.contiguous()
        keep.append(im)
        H, W = im.shape
        descs[i].img = im.data_ptr()
        descs[i].H = H
        descs[i].W = W
        descs[i].pitch_bytes = im.stride(0) if H > 0 else W
        descs[i].labels = outs[i].data_ptr()
    kd = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if k_out is None else k_out
    if classes:
        _check(ccl_label_batch_classes(descs, n, connectivity, kd.data_ptr(), _stream_ptr(stream)),
               "ccl_label_batch_classes")
    elif threshold is None:
        _check(ccl_label_batch(descs, n, connectivity, kd.data_ptr(), _stream_ptr(stream)), "ccl_label_batch")
    else:
        _check(ccl_label_batch_threshold(descs, n, connectivity, int(threshold), kd.data_ptr(), _stream_ptr(stream)),
               "ccl_label_batch_threshold")
    return outs, kd[:n]


def label_host(img, connectivity: int = 8, out=None, stream=None):
    """Label a HOST image (numpy uint8 array or CPU uint8 tensor; pinned memory is
    fastest).  Returns ``(labels, K)`` with labels on the host (same kind as ``out`` or a
    numpy array)."""
    import numpy as np

    if hasattr(img, "data_ptr"):
        ptr, (H, W), pitch = img.data_ptr(), tuple(img.shape), img.stride(0)
    else:
        img = np.asarray(img)
        if img.dtype != np.uint8 or img.ndim != 2 or img.strides[1] != 1:
            img = np.ascontiguousarray(img, dtype=np.uint8)
        ptr, (H, W), pitch = img.ctypes.data, img.shape, img.strides[0]
    if out is None:
        out = np.empty((H, W), dtype=np.int32)
    optr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    k = ctypes.c_int32(-1)
    _check(ccl_label_host(ptr, H, W, pitch if H > 0 else W, connectivity, optr, ctypes.byref(k),
                          _stream_ptr(stream)), "ccl_label_host")
    return out, int(k.value)


def kernel_times() -> dict:
    """{kernel name: (launches, total ms)} since the last ccl_profile_reset()."""
    buf = (KernelTime * 32)()
    n = ctypes.c_int32(0)
    _check(ccl_profile_read(buf, 32, ctypes.byref(n)), "ccl_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, 32))}
