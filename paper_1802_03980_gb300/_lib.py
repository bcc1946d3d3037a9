"""ctypes binding of libkftrack.so: the C ABI of include/kf_track.h, same names.

Argument marshalling only. Every step of the tracking path runs in the CUDA
library; if the library is missing this module raises at import time instead
of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("KF_TRACK_LIB") or os.path.join(HERE, "libkftrack.so")

KF_MAX_LEVELS = 4
KF_TRACE_MAX = 64

KF_OK = 0
KF_NOT_CONVERGED = 1
KF_ERR_INVALID_ARG = -1
KF_ERR_CUDA = -2
KF_ERR_OOM = -3
KF_ERR_NO_FRAME = -4
KF_ERR_NO_MODEL = -5
KF_ERR_TOO_FEW_INLIERS = -6
KF_ERR_DEGENERATE = -7
KF_ERR_TIMEOUT = -8
KF_ERR_INTERNAL = -9
KF_ERR_SCRATCH_LIMIT = -10

KF_USE_PRIOR = 1
KF_USE_FILTER = 2
KF_USE_CONVERGENCE = 4
KF_SINGLE_PASS = 8
KF_LAUNCH_PER_ITERATION = 16
KF_PRIOR_ANCHORED = 32
KF_FP32 = 0
KF_FP16 = 1
KF_NORMALS_CROSS = 0
KF_NORMALS_INTEGRAL = 1
KF_FRAME_HOST, KF_FRAME_DEVICE, KF_FRAME_HOST_COPY_ENGINE = 0, 1, 2
KF_LAMBDA_CONST, KF_LAMBDA_C_SQRT_N, KF_LAMBDA_C_N, KF_LAMBDA_C_N2, KF_LAMBDA_C_LOG_N = range(5)


class kf_intrinsics(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]


class kf_params(C.Structure):
    _fields_ = [("levels", C.c_int), ("max_iters", C.c_int * KF_MAX_LEVELS), ("hist_bins", C.c_int),
                ("d_max", C.c_double), ("band_kappa", C.c_double), ("cos_angle_min", C.c_double),
                ("conv_window", C.c_int), ("lambda_mode", C.c_int), ("lambda_c", C.c_double),
                ("n_min", C.c_int), ("precision", C.c_int), ("flags", C.c_uint),
                ("bilateral_sigma_s", C.c_double), ("bilateral_sigma_r", C.c_double),
                ("bilateral_radius", C.c_int), ("normal_mode", C.c_int),
                ("ii_radius_a", C.c_double), ("ii_radius_b", C.c_double),
                ("ii_depth_change", C.c_double), ("ii_radius_max", C.c_int),
                ("shoot_radius", C.c_int)]


class kf_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int * KF_MAX_LEVELS), ("total_iters", C.c_int),
                ("inliers", C.c_int), ("valid_pairs", C.c_int),
                ("median_bin", C.c_int * KF_MAX_LEVELS), ("rms_residual", C.c_double)]


class kf_iter_record(C.Structure):
    _fields_ = [("level", C.c_int), ("iter", C.c_int), ("N", C.c_int), ("kmed", C.c_int),
                ("klo", C.c_int), ("khi", C.c_int), ("n", C.c_int), ("solve_ns", C.c_int),
                ("passes", C.c_int), ("w0", C.c_int), ("w1", C.c_int), ("pad", C.c_int),
                ("lambda_", C.c_double), ("x", C.c_double * 6)]


class kf_volume_params(C.Structure):
    _fields_ = [("res", C.c_int), ("side", C.c_float), ("origin", C.c_float * 3), ("mu", C.c_float),
                ("w_max", C.c_float)]


class kf_profile(C.Structure):
    _fields_ = [("frontend_ms", C.c_double), ("assoc_ms", C.c_double), ("reduce_ms", C.c_double),
                ("fused_ms", C.c_double), ("align_ms", C.c_double),
                ("frontend_calls", C.c_longlong), ("assoc_launches", C.c_longlong),
                ("reduce_launches", C.c_longlong), ("fused_launches", C.c_longlong),
                ("graph_launches", C.c_longlong), ("pixel_iters", C.c_longlong),
                ("alignments", C.c_longlong), ("sched_ms", C.c_double),
                ("sched_launches", C.c_longlong)]


EXPORTS = ["kf_default_params", "kf_track_create", "kf_track_destroy", "kf_set_frame",
           "kf_set_frame_batch", "kf_set_model", "kf_align", "kf_align_batch", "kf_last_error",
           "kf_debug_frame_level", "kf_debug_model_level", "kf_debug_associate",
           "kf_debug_reduce", "kf_debug_trace", "kf_profile_enable", "kf_profile_read",
           "kf_reduce_noalloc", "kf_debug_wait_timeout", "kf_volume_default_params",
           "kf_volume_create", "kf_volume_destroy", "kf_volume_last_error", "kf_volume_reset",
           "kf_volume_integrate", "kf_volume_raycast", "kf_volume_read"]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1802_03980_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D, VP = C.POINTER, C.c_int, C.c_double, C.c_void_p
    sig = {
        "kf_default_params": (I, [P(kf_params)]),
        "kf_track_create": (I, [P(kf_params), I, I, VP, P(VP)]),
        "kf_track_destroy": (None, [VP]),
        "kf_set_frame": (I, [VP, VP, P(kf_intrinsics), I]),
        "kf_set_frame_batch": (I, [P(VP), I, P(VP), P(kf_intrinsics), I]),
        "kf_set_model": (I, [VP, VP, VP, P(D), P(kf_intrinsics), I]),
        "kf_align": (I, [VP, P(D), P(D), D, P(D), P(kf_result)]),
        "kf_align_batch": (I, [P(VP), I, P(D), P(D), P(D), P(D), P(kf_result)]),
        "kf_last_error": (C.c_char_p, [VP]),
        "kf_debug_frame_level": (I, [VP, I, VP, VP, VP, P(I)]),
        "kf_debug_model_level": (I, [VP, I, VP, VP, P(I)]),
        "kf_debug_associate": (I, [VP, I, P(D), VP, VP, VP]),
        "kf_debug_reduce": (I, [VP, I, P(D), I, I, P(D)]),
        "kf_debug_trace": (I, [VP, P(kf_iter_record), I, P(I)]),
        "kf_profile_enable": (I, [VP, I]),
        "kf_profile_read": (I, [VP, P(kf_profile)]),
        "kf_reduce_noalloc": (I, [VP, I, I, VP, VP, P(kf_intrinsics), P(D), P(D), D, I, I, I, VP, VP]),
        "kf_debug_wait_timeout": (I, [VP, D]),
        "kf_volume_default_params": (I, [P(kf_volume_params)]),
        "kf_volume_create": (I, [P(kf_volume_params), VP, P(VP)]),
        "kf_volume_destroy": (None, [VP]),
        "kf_volume_last_error": (C.c_char_p, [VP]),
        "kf_volume_reset": (I, [VP]),
        "kf_volume_integrate": (I, [VP, VP, P(kf_intrinsics), P(D), I]),
        "kf_volume_raycast": (I, [VP, P(kf_intrinsics), P(D), C.c_float, C.c_float, C.c_float, VP, VP, I]),
        "kf_volume_read": (I, [VP, VP, VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# kf_intrinsics as a numpy record (same layout), so that a batch's intrinsics
# marshal without building one ctypes object per pair
_INTR_DT = np.dtype([("width", "<i4"), ("height", "<i4"), ("fx", "<f8"), ("fy", "<f8"),
                     ("cx", "<f8"), ("cy", "<f8")], align=True)
_ptr_cache: dict = {}


def _intr_array(Ks) -> np.ndarray:
    if isinstance(Ks, np.ndarray) and Ks.dtype == _INTR_DT:
        return np.ascontiguousarray(Ks)
    k0 = Ks[0]
    if not isinstance(k0, kf_intrinsics) and all(K is k0 or K == k0 for K in Ks):
        return np.array([tuple(k0)], _INTR_DT).repeat(len(Ks))  # one camera for the batch
    rows = [(K.width, K.height, K.fx, K.fy, K.cx, K.cy) if isinstance(K, kf_intrinsics) else tuple(K)
            for K in Ks]
    return np.array(rows, _INTR_DT)


def _tracker_array(ts):
    """ctypes array of tracker handles, cached for a repeated tracker list."""
    key = tuple(t.value for t in ts)
    arr = _ptr_cache.get(key)
    if arr is None:
        if len(_ptr_cache) > 64:
            _ptr_cache.clear()
        arr = (C.c_void_p * len(key))(*key)
        _ptr_cache[key] = arr
    return arr


def _intr(K) -> kf_intrinsics:
    if isinstance(K, kf_intrinsics):
        return K
    w, h, fx, fy, cx, cy = K
    return kf_intrinsics(int(w), int(h), float(fx), float(fy), float(cx), float(cy))


class KFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"kf status {status}: {msg}")
        self.status = status


# ---- functions with the ABI's names -----------------------------------------
def kf_default_params() -> kf_params:
    p = kf_params()
    _lib.kf_default_params(C.byref(p))
    return p


def kf_track_create(params: kf_params, max_w: int, max_h: int, cuda_stream: int = 0):
    h = C.c_void_p()
    st = _lib.kf_track_create(C.byref(params), max_w, max_h, C.c_void_p(cuda_stream), C.byref(h))
    if st != KF_OK:
        raise KFError(st, "kf_track_create failed")
    return h


def kf_track_destroy(t):
    _lib.kf_track_destroy(t)


def kf_last_error(t) -> str:
    return _lib.kf_last_error(t).decode()


def _check(t, st, ok=(KF_OK, KF_NOT_CONVERGED)):
    if st not in ok:
        raise KFError(st, kf_last_error(t))
    return st


def kf_set_frame(t, depth_ptr: int, K, is_device_ptr) -> int:
    Ki = _intr(K)
    return _check(t, _lib.kf_set_frame(t, C.c_void_p(depth_ptr), C.byref(Ki), int(is_device_ptr)))


def kf_set_frame_batch(ts, depth_ptrs, Ks, is_device_ptr) -> int:
    n = len(ts)
    arr_t = _tracker_array(ts)
    arr_d = np.asarray(depth_ptrs, np.uintp)
    arr_k = _intr_array(Ks)
    if arr_d.shape != (n,) or arr_k.shape != (n,):
        raise ValueError("one depth pointer and one intrinsics entry per tracker")
    return _check(ts[0], _lib.kf_set_frame_batch(arr_t, n, arr_d.ctypes.data_as(C.POINTER(C.c_void_p)),
                                                 arr_k.ctypes.data_as(C.POINTER(kf_intrinsics)),
                                                 int(is_device_ptr)))


def kf_set_model(t, vertex_ptr: int, normal_ptr: int, model_pose, K, is_device_ptr: bool) -> int:
    pose = np.ascontiguousarray(model_pose, np.float64).reshape(16)
    Ki = _intr(K)
    return _check(t, _lib.kf_set_model(t, C.c_void_p(vertex_ptr), C.c_void_p(normal_ptr),
                                       _dptr(pose), C.byref(Ki), int(is_device_ptr)))


def kf_align(t, prior_R, init_pose, lam: float):
    """Returns (status, pose 4x4, kf_result). Errors other than the alignment's
    own statuses (too few inliers, degenerate, not converged) raise."""
    init = np.ascontiguousarray(init_pose, np.float64).reshape(16)
    pr = None if prior_R is None else np.ascontiguousarray(prior_R, np.float64).reshape(9)
    out = np.zeros(16, np.float64)
    res = kf_result()
    st = _lib.kf_align(t, None if pr is None else _dptr(pr), _dptr(init), float(lam), _dptr(out),
                       C.byref(res))
    _check(t, st, (KF_OK, KF_NOT_CONVERGED, KF_ERR_TOO_FEW_INLIERS, KF_ERR_DEGENERATE))
    return st, out.reshape(4, 4), res


def kf_align_batch(ts, prior_R, init_pose, lam):
    n = len(ts)
    arr_t = _tracker_array(ts)
    init = np.ascontiguousarray(init_pose, np.float64).reshape(n * 16)
    pr = None if prior_R is None else np.ascontiguousarray(prior_R, np.float64).reshape(n * 9)
    lm = np.ascontiguousarray(lam, np.float64).reshape(n)
    out = np.zeros(n * 16, np.float64)
    res = (kf_result * n)()
    st = _lib.kf_align_batch(arr_t, n, None if pr is None else _dptr(pr), _dptr(init), _dptr(lm),
                             _dptr(out), res)
    _check(ts[0], st, (KF_OK, KF_NOT_CONVERGED, KF_ERR_TOO_FEW_INLIERS, KF_ERR_DEGENERATE))
    return st, out.reshape(n, 4, 4), list(res)


def kf_debug_frame_level(t, level: int):
    dims = (C.c_int * 2)()
    _check(t, _lib.kf_debug_frame_level(t, level, None, None, None, dims))
    w, h = dims[0], dims[1]
    D = np.zeros((h, w), np.float32)
    V = np.zeros((h, w, 3), np.float32)
    N = np.zeros((h, w, 3), np.float32)
    _check(t, _lib.kf_debug_frame_level(t, level, D.ctypes.data, V.ctypes.data, N.ctypes.data, dims))
    return D, V, N


def kf_debug_model_level(t, level: int):
    dims = (C.c_int * 2)()
    _check(t, _lib.kf_debug_model_level(t, level, None, None, dims))
    w, h = dims[0], dims[1]
    V = np.zeros((h, w, 3), np.float32)
    N = np.zeros((h, w, 3), np.float32)
    _check(t, _lib.kf_debug_model_level(t, level, V.ctypes.data, N.ctypes.data, dims))
    return V, N


def kf_debug_associate(t, level: int, pose, shape, bins: int):
    h, w = shape
    pose = np.ascontiguousarray(pose, np.float64).reshape(16)
    idx = np.zeros((h, w), np.int32)
    b = np.zeros((h, w), np.int32)
    hist = np.zeros(bins, np.uint32)
    _check(t, _lib.kf_debug_associate(t, level, _dptr(pose), idx.ctypes.data, b.ctypes.data,
                                      hist.ctypes.data))
    return idx, b, hist


def kf_debug_reduce(t, level: int, pose, klo: int, khi: int) -> np.ndarray:
    pose = np.ascontiguousarray(pose, np.float64).reshape(16)
    sums = np.zeros(29, np.float64)
    _check(t, _lib.kf_debug_reduce(t, level, _dptr(pose), klo, khi, _dptr(sums)))
    return sums


def kf_debug_trace(t):
    rec = (kf_iter_record * KF_TRACE_MAX)()
    cnt = C.c_int()
    _check(t, _lib.kf_debug_trace(t, rec, KF_TRACE_MAX, C.byref(cnt)))
    return list(rec)[: cnt.value]


def kf_debug_wait_timeout(t, wait_ms: float) -> int:
    """Status of an empty scheduled launch whose bounded waits run out
    (KF_ERR_TIMEOUT expected); raises on any other error."""
    return _check(t, _lib.kf_debug_wait_timeout(t, float(wait_ms)), ok=(KF_ERR_TIMEOUT,))


def kf_profile_enable(t, on: bool = True) -> int:
    return _check(t, _lib.kf_profile_enable(t, int(on)))


def kf_profile_read(t) -> kf_profile:
    pr = kf_profile()
    _check(t, _lib.kf_profile_read(t, C.byref(pr)))
    return pr


def kf_reduce_noalloc(frame_vertex_ptr: int, width: int, height: int, model_vertex_ptr: int,
                      model_normal_ptr: int, model_K, pose, model_pose, d_max: float,
                      hist_bins: int, klo: int, khi: int, sums_ptr: int, cuda_stream: int = 0) -> int:
    """Device pointers in, 29 double sums written to device memory at sums_ptr.
    Returns the status (no tracker exists to hold an error message)."""
    Ki = _intr(model_K)
    pz = np.ascontiguousarray(pose, np.float64).reshape(16)
    mz = np.ascontiguousarray(model_pose, np.float64).reshape(16)
    return _lib.kf_reduce_noalloc(C.c_void_p(frame_vertex_ptr), width, height,
                                  C.c_void_p(model_vertex_ptr), C.c_void_p(model_normal_ptr),
                                  C.byref(Ki), _dptr(pz), _dptr(mz), float(d_max), hist_bins,
                                  klo, khi, C.c_void_p(sums_ptr), C.c_void_p(cuda_stream))


# ---- model producer (TSDF volume + raycast) --------------------------------
def _vcheck(v, st):
    if st != KF_OK:
        raise KFError(st, (_lib.kf_volume_last_error(v) or b"").decode())
    return st


def kf_volume_default_params() -> kf_volume_params:
    p = kf_volume_params()
    _lib.kf_volume_default_params(C.byref(p))
    return p


def kf_volume_create(p: kf_volume_params, stream: int = 0):
    v = C.c_void_p()
    st = _lib.kf_volume_create(C.byref(p), C.c_void_p(stream), C.byref(v))
    if st != KF_OK:
        raise KFError(st, "kf_volume_create failed")
    return v


def kf_volume_destroy(v) -> None:
    _lib.kf_volume_destroy(v)


def kf_volume_reset(v) -> int:
    return _vcheck(v, _lib.kf_volume_reset(v))


def kf_volume_integrate(v, depth_ptr: int, K, pose, is_device_ptr: bool) -> int:
    Ki = _intr(K)
    T = np.ascontiguousarray(pose, np.float64).reshape(16)
    return _vcheck(v, _lib.kf_volume_integrate(v, C.c_void_p(depth_ptr), C.byref(Ki), _dptr(T),
                                               int(is_device_ptr)))


def kf_volume_raycast(v, K, pose, z_near: float, z_far: float, dz: float,
                      vertex_ptr: int = 0, normal_ptr: int = 0, is_device_ptr: bool = False):
    """With device pointers the maps are written there; else host arrays
    (H, W, 3) are returned."""
    Ki = _intr(K)
    T = np.ascontiguousarray(pose, np.float64).reshape(16)
    if is_device_ptr:
        _vcheck(v, _lib.kf_volume_raycast(v, C.byref(Ki), _dptr(T), z_near, z_far, dz,
                                          C.c_void_p(vertex_ptr), C.c_void_p(normal_ptr), 1))
        return None
    V = np.zeros((Ki.height, Ki.width, 3), np.float32)
    N = np.zeros((Ki.height, Ki.width, 3), np.float32)
    _vcheck(v, _lib.kf_volume_raycast(v, C.byref(Ki), _dptr(T), z_near, z_far, dz,
                                      V.ctypes.data_as(C.c_void_p), N.ctypes.data_as(C.c_void_p), 0))
    return V, N


def kf_volume_read(v, res: int):
    F = np.zeros((res, res, res), np.float32)
    W = np.zeros((res, res, res), np.float32)
    _vcheck(v, _lib.kf_volume_read(v, F.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p)))
    return F, W


def kf_volume_last_error(v) -> str:
    return (_lib.kf_volume_last_error(v) or b"").decode()
