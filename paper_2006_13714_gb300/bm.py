"""Thin ctypes binding over the C ABI in ``include/bm.h`` (argument marshalling only).

The low-level functions carry the C names and take raw pointers (ints);
``Context`` wraps them for torch tensors.  Every step of block matching
runs in the CUDA library; if the library cannot be loaded this module
raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build_ext

BM_U8, BM_F32 = 0, 1
BM_OK = 0
BM_ERR_INVALID, BM_ERR_UNSUPPORTED, BM_ERR_OOM, BM_ERR_CUDA = -1, -2, -3, -4
BM_ERR_TIMEOUT, BM_ERR_BUSY, BM_ERR_NOT_FOUND, BM_ERR_TOO_LARGE = -5, -6, -7, -8
BM_STATIC_SCRATCH_BYTES = 16 << 20
BM_ALGO_AUTO, BM_ALGO_SELFCONV_TC, BM_ALGO_DIRECT = 0, 1, 2

INT32_MAX = 2**31 - 1

_lock = threading.Lock()
_lib = None


class BMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bm error {code}: {msg}")
        self.code = code


class bm_request(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("C", ctypes.c_int), ("dtype", ctypes.c_int), ("patch", ctypes.c_int),
                ("window", ctypes.c_int), ("stride", ctypes.c_int), ("K", ctypes.c_int),
                ("out_idx", ctypes.c_void_p), ("out_dist", ctypes.c_void_p)]


class bm_stats(ctypes.Structure):
    _fields_ = [("matches", ctypes.c_uint64), ("refs", ctypes.c_uint64),
                ("rerank_overflow", ctypes.c_uint64), ("fp64_rechecks", ctypes.c_uint64),
                ("bound_violations", ctypes.c_uint64), ("tc_jobs", ctypes.c_uint64)]


NUM_STAGES = 5
STAGES = ("planes", "box", "tc", "rerank", "direct")


class bm_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * NUM_STAGES), ("ms", ctypes.c_double * NUM_STAGES)]


def library_path() -> str:
    return build_ext.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_ext.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA block-matching library not built: {path}")
            build_ext.build()
        lib = ctypes.CDLL(path)
        vp, ci, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        pi = ctypes.POINTER(ctypes.c_int)
        sig = {
            "bm_create": ([ctypes.POINTER(vp), ci, sz, ctypes.c_char_p], ci),
            "bm_destroy": ([vp], None),
            "bm_last_error": ([vp], ctypes.c_char_p),
            "bm_num_refs": ([ci, ci, ci, ci, pi, pi], ci),
            "bm_match": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_match_direct": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_match_host": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp], ci),
            "bm_match_batch": ([vp, ctypes.POINTER(bm_request), ci, vp], ci),
            "bm_match_host_batch": ([vp, ctypes.POINTER(bm_request), ci], ci),
            "bm_set_algo": ([vp, ci], ci),
            "bm_submit": ([vp, ctypes.POINTER(bm_request), ctypes.POINTER(ctypes.c_uint64)], ci),
            "bm_poll": ([vp, ctypes.c_uint64, pi, pi], ci),
            "bm_get_stats": ([vp, ctypes.POINTER(bm_stats)], ci),
            "bm_set_timing": ([vp, ci], ci),
            "bm_get_timing": ([vp, ctypes.POINTER(bm_timing), ci], ci),
            "bm_static_scratch_bytes": ([ci, ci, ci, ci, ci, ci, ci, ci], sz),
            "bm_window_split": ([ci, ci, ci, ci, ci, ci, ci, ci], ci),
            "bm_workspace_bytes": ([ci, ci, ci, ci, ci, ci, ci, ci], sz),
            "bm_match_static": ([vp, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_static_init": ([], ci),
            "bm_static_check": ([vp], ci),
            "bm_static_set_fault_injection": ([ci], ci),
            "bm_gather_groups": ([vp, vp, ci, ci, ci, ci, ci, vp, ci, ci, ci, vp, vp], ci),
            "bm_aggregate": ([vp, vp, vp, vp, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_nlm": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ctypes.c_float, vp, vp, vp], ci),
            "bm_match_ncc": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_match_3d": ([vp, vp, ci, ci, ci, ci, ci, ci, ci, ci, ci, vp, vp, vp], ci),
            "bm_check": ([vp, vp], ci),
            "bm_set_fault_injection": ([vp, ci], ci),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


# ---- low-level functions with the C names ----

def bm_create(device: int = 0, mem_budget_bytes: int = 0, tune_cache: str | None = None) -> int:
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.bm_create(ctypes.byref(out), device, mem_budget_bytes,
                       tune_cache.encode() if tune_cache else None)
    if rc != BM_OK:
        raise BMError(rc, lib.bm_last_error(None).decode())
    return out.value


def bm_destroy(ctx: int) -> None:
    load().bm_destroy(ctx)


def bm_last_error(ctx: int | None = None) -> str:
    return load().bm_last_error(ctx).decode()


def bm_num_refs(H: int, W: int, patch: int, stride: int) -> tuple[int, int]:
    ry, rx = ctypes.c_int(), ctypes.c_int()
    rc = load().bm_num_refs(H, W, patch, stride, ctypes.byref(ry), ctypes.byref(rx))
    if rc != BM_OK:
        raise BMError(rc, bm_last_error())
    return ry.value, rx.value


def bm_match(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist, stream) -> int:
    return load().bm_match(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx,
                           out_dist, stream)


def bm_match_direct(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist,
                    stream) -> int:
    return load().bm_match_direct(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx,
                                  out_dist, stream)


def bm_workspace_bytes(H, W, C, dtype, patch, window, stride, K) -> int:
    return load().bm_workspace_bytes(H, W, C, dtype, patch, window, stride, K)


def bm_window_split(H, W, C, dtype, patch, window, stride, K) -> int:
    return load().bm_window_split(H, W, C, dtype, patch, window, stride, K)


def bm_static_scratch_bytes(H, W, C, dtype, patch, window, stride, K) -> int:
    return load().bm_static_scratch_bytes(H, W, C, dtype, patch, window, stride, K)


def bm_match_static(img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist,
                    stream) -> int:
    """No-allocation matcher (fixed device scratch shared by all calls; see bm.h)."""
    return load().bm_match_static(img, H, W, C, dtype, patch, window, stride, K, out_idx,
                                  out_dist, stream)


def bm_static_init() -> int:
    return load().bm_static_init()


def bm_static_check(stream) -> int:
    return load().bm_static_check(stream)


def bm_static_set_fault_injection(mode) -> int:
    return load().bm_static_set_fault_injection(mode)


def bm_gather_groups(ctx, img, H, W, C, dtype, patch, idx, n_ry, n_rx, K, out_groups,
                     stream) -> int:
    return load().bm_gather_groups(ctx, img, H, W, C, dtype, patch, idx, n_ry, n_rx, K,
                                   out_groups, stream)


def bm_aggregate(ctx, groups, idx, weights, n_ry, n_rx, K, H, W, C, patch, out_img, out_weight,
                 stream) -> int:
    return load().bm_aggregate(ctx, groups, idx, weights, n_ry, n_rx, K, H, W, C, patch,
                               out_img, out_weight, stream)


def bm_check(ctx, stream) -> int:
    return load().bm_check(ctx, stream)


def bm_set_fault_injection(ctx, mode: int) -> int:
    return load().bm_set_fault_injection(ctx, mode)


def bm_match_3d(ctx, img, H, W, C, dtype, patch, depth, window, stride, K, out_idx, out_dist,
                stream) -> int:
    return load().bm_match_3d(ctx, img, H, W, C, dtype, patch, depth, window, stride, K, out_idx,
                              out_dist, stream)


def bm_match_ncc(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx, out_score,
                 stream) -> int:
    return load().bm_match_ncc(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx,
                               out_score, stream)


def bm_nlm(ctx, img, H, W, C, dtype, patch, window, stride, b, out_est, out_theta, stream) -> int:
    return load().bm_nlm(ctx, img, H, W, C, dtype, patch, window, stride, b, out_est, out_theta,
                         stream)


def bm_match_host(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx, out_dist) -> int:
    return load().bm_match_host(ctx, img, H, W, C, dtype, patch, window, stride, K, out_idx,
                                out_dist)


def bm_match_host_batch(ctx, reqs, n) -> int:
    return load().bm_match_host_batch(ctx, reqs, n)


def bm_match_batch(ctx, reqs, n, stream) -> int:
    return load().bm_match_batch(ctx, reqs, n, stream)


def bm_set_algo(ctx, algo) -> int:
    return load().bm_set_algo(ctx, algo)


def bm_submit(ctx, req) -> tuple[int, int]:
    t = ctypes.c_uint64()
    rc = load().bm_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    return rc, t.value


def bm_poll(ctx, ticket) -> tuple[int, int, int]:
    done, status = ctypes.c_int(), ctypes.c_int()
    rc = load().bm_poll(ctx, ticket, ctypes.byref(done), ctypes.byref(status))
    return rc, done.value, status.value


def bm_get_stats(ctx) -> dict:
    s = bm_stats()
    rc = load().bm_get_stats(ctx, ctypes.byref(s))
    if rc != BM_OK:
        raise BMError(rc, bm_last_error(ctx))
    return {k: int(getattr(s, k)) for k, _ in bm_stats._fields_}


def bm_set_timing(ctx, enable: int) -> int:
    return load().bm_set_timing(ctx, enable)


def bm_get_timing(ctx, reset: int = 0) -> dict:
    t = bm_timing()
    rc = load().bm_get_timing(ctx, ctypes.byref(t), reset)
    if rc != BM_OK:
        raise BMError(rc, bm_last_error(ctx))
    return {name: {"launches": int(t.launches[i]), "ms": float(t.ms[i])}
            for i, name in enumerate(STAGES)}


# ---- torch convenience wrapper ----

def _dtype_code(t):
    import torch
    if t.dtype == torch.uint8:
        return BM_U8
    if t.dtype == torch.float32:
        return BM_F32
    raise TypeError("image must be uint8 or float32")


def _hwc(img):
    if img.dim() == 2:
        return img.shape[0], img.shape[1], 1
    if img.dim() == 3:
        return img.shape[0], img.shape[1], img.shape[2]
    raise ValueError("image must be H x W or H x W x C")


class Context:
    """A library context on one CUDA device; tensors are torch CUDA tensors."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, tune_cache: str | None = None):
        self.device = device
        self.handle = bm_create(device, mem_budget_bytes, tune_cache)

    def close(self):
        if self.handle:
            bm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != BM_OK:
            raise BMError(rc, bm_last_error(self.handle))

    def set_algo(self, algo: int):
        self._check(bm_set_algo(self.handle, algo))

    def outputs(self, img, patch, stride, K):
        import torch
        H, W, _ = _hwc(img)
        ry, rx = bm_num_refs(H, W, patch, stride)
        idx = torch.empty((ry * rx, K), dtype=torch.int32, device=img.device)
        dist = torch.empty((ry * rx, K), dtype=torch.int32 if img.dtype == torch.uint8
                           else torch.float32, device=img.device)
        return idx, dist

    def _run(self, fn, img, patch, window, stride, K, out=None, stream=None):
        import torch
        if not img.is_cuda or not img.is_contiguous():
            raise ValueError("image must be a contiguous CUDA tensor")
        H, W, C = _hwc(img)
        idx, dist = out if out is not None else self.outputs(img, patch, stride, K)
        st = stream if stream is not None else torch.cuda.current_stream(img.device)
        rc = fn(self.handle, img.data_ptr(), H, W, C, _dtype_code(img), patch, window, stride, K,
                idx.data_ptr(), dist.data_ptr(), st.cuda_stream)
        self._check(rc)
        return idx, dist

    def match(self, img, patch, window, stride, K, out=None, stream=None):
        """Self-Convolution block matching; returns (idx int32 [nR,K], dist [nR,K])."""
        return self._run(bm_match, img, patch, window, stride, K, out, stream)

    def match_direct(self, img, patch, window, stride, K, out=None, stream=None):
        """Plain FP32 CUDA-core direct-distance block matching (baseline)."""
        return self._run(bm_match_direct, img, patch, window, stride, K, out, stream)

    def match_host(self, img_np, patch, window, stride, K, out=None):
        """Host (numpy) buffers in and out; synchronous."""
        import numpy as np
        a = np.ascontiguousarray(img_np)
        if a.ndim == 2:
            a = a[:, :, None]
        H, W, C = a.shape
        dt = BM_U8 if a.dtype == np.uint8 else BM_F32
        ry, rx = bm_num_refs(H, W, patch, stride)
        if out is None:
            idx = np.empty((ry * rx, K), np.int32)
            dist = np.empty((ry * rx, K), np.int32 if dt == BM_U8 else np.float32)
        else:
            idx, dist = out
        rc = bm_match_host(self.handle, a.ctypes.data, H, W, C, dt, patch, window, stride, K,
                           idx.ctypes.data, dist.ctypes.data)
        self._check(rc)
        return idx, dist

    @staticmethod
    def request(img, patch, window, stride, K, idx, dist) -> bm_request:
        H, W, C = _hwc(img)
        return bm_request(img.data_ptr(), H, W, C, _dtype_code(img), patch, window, stride, K,
                          idx.data_ptr(), dist.data_ptr())

    def match_batch(self, reqs, stream=None):
        import torch
        arr = (bm_request * len(reqs))(*reqs)
        st = stream if stream is not None else torch.cuda.current_stream()
        self._check(bm_match_batch(self.handle, arr, len(reqs), st.cuda_stream))

    def submit(self, req: bm_request) -> int:
        rc, t = bm_submit(self.handle, req)
        self._check(rc)
        return t

    def poll(self, ticket: int):
        rc, done, status = bm_poll(self.handle, ticket)
        self._check(rc)
        return bool(done), status

    def gather_groups(self, img, patch, idx, n_ry, n_rx, out=None, stream=None):
        """Patch groups [n_ry*n_rx, K, patch*patch*C] (img's dtype) of the matches idx."""
        import torch
        if not img.is_cuda or not img.is_contiguous() or not idx.is_contiguous():
            raise ValueError("image and idx must be contiguous CUDA tensors")
        H, W, C = _hwc(img)
        K = idx.shape[-1]
        if out is None:
            out = torch.empty((n_ry * n_rx, K, patch * patch * C), dtype=img.dtype,
                              device=img.device)
        st = stream if stream is not None else torch.cuda.current_stream(img.device)
        self._check(bm_gather_groups(self.handle, img.data_ptr(), H, W, C, _dtype_code(img), patch,
                                     idx.data_ptr(), n_ry, n_rx, K, out.data_ptr(),
                                     st.cuda_stream))
        return out

    def aggregate(self, groups, idx, H, W, C, patch, n_ry, n_rx, weights=None, out=None,
                  stream=None):
        """Reconstruction: (image [H, W, C] float32, weight map [H, W] float32)."""
        import torch
        if groups.dtype != torch.float32 or not groups.is_contiguous() or not idx.is_contiguous():
            raise ValueError("groups must be contiguous float32, idx contiguous int32")
        K = idx.shape[-1]
        if out is None:
            out = (torch.empty((H, W, C), dtype=torch.float32, device=groups.device),
                   torch.empty((H, W), dtype=torch.float32, device=groups.device))
        st = stream if stream is not None else torch.cuda.current_stream(groups.device)
        wp = weights.data_ptr() if weights is not None else None
        self._check(bm_aggregate(self.handle, groups.data_ptr(), idx.data_ptr(), wp, n_ry, n_rx,
                                 K, H, W, C, patch, out[0].data_ptr(), out[1].data_ptr(),
                                 st.cuda_stream))
        return out

    def match_3d(self, img, patch, depth, window, stride, K, out=None, stream=None):
        """3-D block matching across channels: (idx [nR*(C-depth+1), K], dist), nearest first."""
        import torch
        if not img.is_cuda or not img.is_contiguous():
            raise ValueError("image must be a contiguous CUDA tensor")
        H, W, C = _hwc(img)
        ry, rx = bm_num_refs(H, W, patch, stride)
        n = ry * rx * (C - depth + 1)
        if out is None:
            out = (torch.empty((n, K), dtype=torch.int32, device=img.device),
                   torch.empty((n, K), dtype=torch.int32 if img.dtype == torch.uint8
                               else torch.float32, device=img.device))
        st = stream if stream is not None else torch.cuda.current_stream(img.device)
        self._check(bm_match_3d(self.handle, img.data_ptr(), H, W, C, _dtype_code(img), patch,
                                depth, window, stride, K, out[0].data_ptr(), out[1].data_ptr(),
                                st.cuda_stream))
        return out

    def match_ncc(self, img, patch, window, stride, K, out=None, stream=None):
        """NCC block matching: (idx int32 [nR, K], score float32 [nR, K]), best first."""
        import torch
        if not img.is_cuda or not img.is_contiguous():
            raise ValueError("image must be a contiguous CUDA tensor")
        H, W, C = _hwc(img)
        ry, rx = bm_num_refs(H, W, patch, stride)
        if out is None:
            out = (torch.empty((ry * rx, K), dtype=torch.int32, device=img.device),
                   torch.empty((ry * rx, K), dtype=torch.float32, device=img.device))
        st = stream if stream is not None else torch.cuda.current_stream(img.device)
        self._check(bm_match_ncc(self.handle, img.data_ptr(), H, W, C, _dtype_code(img), patch,
                                 window, stride, K, out[0].data_ptr(), out[1].data_ptr(),
                                 st.cuda_stream))
        return out

    def nlm(self, img, patch, window, stride, b, out=None, stream=None):
        """Non-local means: (estimates [nR, patch*patch*C] float32, Theta [nR] float32)."""
        import torch
        if not img.is_cuda or not img.is_contiguous():
            raise ValueError("image must be a contiguous CUDA tensor")
        H, W, C = _hwc(img)
        ry, rx = bm_num_refs(H, W, patch, stride)
        if out is None:
            out = (torch.empty((ry * rx, patch * patch * C), dtype=torch.float32, device=img.device),
                   torch.empty((ry * rx,), dtype=torch.float32, device=img.device))
        st = stream if stream is not None else torch.cuda.current_stream(img.device)
        tp = out[1].data_ptr() if out[1] is not None else None
        self._check(bm_nlm(self.handle, img.data_ptr(), H, W, C, _dtype_code(img), patch, window,
                           stride, float(b), out[0].data_ptr(), tp, st.cuda_stream))
        return out

    def stats(self) -> dict:
        return bm_get_stats(self.handle)

    def set_timing(self, enable: bool):
        self._check(bm_set_timing(self.handle, 1 if enable else 0))

    def timing(self, reset: bool = False) -> dict:
        return bm_get_timing(self.handle, 1 if reset else 0)
