"""ctypes wrapper around the plain-C block-matching oracle (``bm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product library.

The oracle evaluates the Euclidean block-matching problem of §III-A
(Eq. equ:bm) directly, in int64 for uint8 images and in IEEE double for
float32 images, restricted to the clipped search window (footnote to
Eq. eq:unifySelfConv, §III-B) and summed over channels (§IV, Eq.
equ:self-convMM).  ``method="selfconv"`` evaluates the same distances
through Lemma 2 (§III-B) instead, with the box-sum norms and the
Self-Convolution cross term of Eq. eq:selfConv computed separately.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libbm_oracle.so")
_lock = threading.Lock()
_lib = None

SENTINEL_U8 = np.int64(2**31 - 1)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no host-specific flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        ci = ctypes.c_int
        for name, dptr in (("bmo_match_u8", i64p), ("bmo_selfconv_u8", i64p),
                           ("bmo_match_f32", f64p), ("bmo_selfconv_f32", f64p)):
            fn = getattr(lib, name)
            fn.argtypes = [vp, ci, ci, ci, ci, ci, ci, ci, i32p, ci, i32p, dptr, ci]
            fn.restype = ci
        lib.bmo_pair_u8.argtypes = [vp, ci, ci, ci, ci, ci, ci, ci, ci, i64p]
        lib.bmo_pair_u8.restype = ci
        lib.bmo_pair_f32.argtypes = [vp, ci, ci, ci, ci, ci, ci, ci, ci, f64p]
        lib.bmo_pair_f32.restype = ci
        lib.bmo_num_refs.argtypes = [ci, ci, ci, ci, i32p, i32p]
        lib.bmo_num_refs.restype = ci
        lib.bmo_max_threads.argtypes = []
        lib.bmo_max_threads.restype = ci
        _lib = lib
        return lib


def max_threads() -> int:
    return int(_load().bmo_max_threads())


def num_refs(H: int, W: int, patch: int, stride: int) -> tuple[int, int]:
    ry = ctypes.c_int32()
    rx = ctypes.c_int32()
    rc = _load().bmo_num_refs(H, W, patch, stride, ctypes.byref(ry), ctypes.byref(rx))
    if rc != 0:
        raise ValueError("invalid geometry")
    return ry.value, rx.value


def _as_hwc(img: np.ndarray) -> np.ndarray:
    if img.ndim == 2:
        img = img[:, :, None]
    if img.ndim != 3:
        raise ValueError("image must be H x W or H x W x C")
    if img.dtype not in (np.uint8, np.float32):
        raise TypeError("image dtype must be uint8 or float32")
    return np.ascontiguousarray(img)


def match(img: np.ndarray, patch: int, window: int, stride: int, K: int,
          refs=None, threads: int = 1, method: str = "direct"):
    """Exact K-nearest block matching.

    Returns ``(idx, dist)``: ``idx`` int32 [n_refs, K] holding row-major
    candidate offsets y*W + x (or -1), ``dist`` int64 (uint8 input, sentinel
    2**31-1) or float64 (float32 input, sentinel +inf) [n_refs, K].
    ``refs`` optionally restricts the computation to these row-major
    reference indices (output rows follow that list).
    """
    img = _as_hwc(img)
    H, W, C = img.shape
    lib = _load()
    ry, rx = num_refs(H, W, patch, stride)
    if refs is None:
        n = ry * rx
        refs_arr = None
        refs_ptr = None
    else:
        refs_arr = np.ascontiguousarray(np.asarray(refs, dtype=np.int32))
        n = int(refs_arr.size)
        refs_ptr = refs_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    idx = np.empty((n, K), dtype=np.int32)
    is_int = img.dtype == np.uint8
    dist = np.empty((n, K), dtype=np.int64 if is_int else np.float64)
    name = {("direct", True): "bmo_match_u8", ("direct", False): "bmo_match_f32",
            ("selfconv", True): "bmo_selfconv_u8", ("selfconv", False): "bmo_selfconv_f32"}[
        (method, is_int)]
    dptr = dist.ctypes.data_as(ctypes.POINTER(ctypes.c_int64 if is_int else ctypes.c_double))
    rc = getattr(lib, name)(img.ctypes.data, H, W, C, patch, window, stride, K,
                            refs_ptr, n, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            dptr, int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return idx, dist


def pair_distance(img: np.ndarray, patch: int, ref_yx, cand_yx):
    """Distance of one explicit pair by the definition (int for uint8, float for float32)."""
    img = _as_hwc(img)
    H, W, C = img.shape
    lib = _load()
    if img.dtype == np.uint8:
        out = ctypes.c_int64()
        rc = lib.bmo_pair_u8(img.ctypes.data, H, W, C, patch, int(ref_yx[0]), int(ref_yx[1]),
                             int(cand_yx[0]), int(cand_yx[1]), ctypes.byref(out))
    else:
        out = ctypes.c_double()
        rc = lib.bmo_pair_f32(img.ctypes.data, H, W, C, patch, int(ref_yx[0]), int(ref_yx[1]),
                              int(cand_yx[0]), int(cand_yx[1]), ctypes.byref(out))
    if rc != 0:
        raise ValueError("pair outside the image")
    return out.value
