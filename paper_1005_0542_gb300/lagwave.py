"""Thin ctypes binding of liblagwave.so (the C ABI declared in include/lagwave.h).

Functions keep the C names; arguments are marshalled only (every step of the computation runs
in the library's CUDA kernels).  Device arrays are passed as integers (``tensor.data_ptr()``);
host arrays as float64 / int numpy arrays.  Importing this module loads the library and raises
``RuntimeError`` if it has not been built (``python -m paper_1005_0542_gb300.build``); there is
no fallback implementation.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblagwave.so")

LAG_OK, LAG_EINVAL, LAG_ENOMEM, LAG_ENOTCONV = 0, -1, -2, -3
LAG_ENUMERIC, LAG_ECUDA, LAG_EAGAIN, LAG_ETIMEDOUT, LAG_ECANCELED = -4, -5, -6, -7, -8
LAG_FP64, LAG_MIXED = 0, 1
LAG_WAVELET_RICKER, LAG_WAVELET_PAPER = 0, 1
LAG_GEMM_SIMT, LAG_GEMM_SPLIT_BF16, LAG_GEMM_SLICE_TILES, LAG_GEMM_SLICE_STREAMK, LAG_GEMM_SLICE_PAIRS = 0, 1, 2, 3, 4
LAG_GEMM_SLICE_CLUSTER = 5


class lag_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dz", C.c_double), ("free_surface", C.c_int),
                ("cylindrical", C.c_int)]


class lag_laguerre(C.Structure):
    _fields_ = [("h", C.c_double), ("alpha", C.c_int), ("n_harm", C.c_int)]


class lag_solver(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("restart_k", C.c_int), ("prec", C.c_int),
                ("partitions", C.c_int), ("tune", C.c_int), ("layered", C.c_int)]


class lag_point(C.Structure):
    _fields_ = [("ix", C.c_int), ("iz", C.c_int)]


class lag_wavelet(C.Structure):
    _fields_ = [("f0", C.c_double), ("t0", C.c_double), ("gamma", C.c_double), ("kind", C.c_int)]


class lag_stats(C.Structure):
    _fields_ = [("iters", C.POINTER(C.c_int)), ("relres", C.POINTER(C.c_double)),
                ("total_iters", C.c_longlong), ("seconds", C.c_double)]


class lag_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("grid", lag_grid), ("c_host", C.POINTER(C.c_double)),
                ("vs_host", C.POINTER(C.c_double)), ("rho_host", C.POINTER(C.c_double)),
                ("lag", lag_laguerre), ("solver", lag_solver), ("wavelet", lag_wavelet),
                ("nsrc", C.c_int), ("src", C.POINTER(lag_point)), ("nrcv", C.c_int),
                ("rcv", C.POINTER(lag_point)), ("nt", C.c_int), ("t_out_host", C.POINTER(C.c_double))]


class lag_result(C.Structure):
    _fields_ = [("status", C.c_int), ("traces_host", C.POINTER(C.c_double)), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("total_iters", C.c_longlong),
                ("device_bytes", C.c_size_t), ("harmonics_done", C.c_int)]


VP = C.c_void_p
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
I = C.c_int
D = C.c_double

# name -> (restype, argtypes)
_PROTOS = {
    "lag_strerror": (C.c_char_p, [I]),
    "lag_last_error": (C.c_char_p, [VP]),
    "lag_version": (I, []),
    "lag_create": (I, [C.POINTER(VP), I, C.c_size_t, VP]),
    "lag_destroy": (None, [VP]),
    "lag_synchronize": (I, [VP]),
    "lag_bytes_in_use": (C.c_size_t, [VP]),
    "lag_kernel_launches": (C.c_longlong, [VP]),
    "lag_profile_enable": (I, [VP, I]),
    "lag_profile_read": (I, [VP, I, C.POINTER(C.c_longlong), PD]),
    "lag_profile_num_classes": (I, []),
    "lag_profile_class_name": (C.c_char_p, [I]),
    "lag_precond_create": (I, [VP, C.POINTER(lag_grid), D, D, D, I, C.POINTER(VP)]),
    "lag_precond_create_sep": (I, [VP, C.POINTER(lag_grid), D, D, D, I, I, C.POINTER(VP)]),
    "lag_precond_create_layered": (I, [VP, C.POINTER(lag_grid), PD, PD, PD, I, I, C.POINTER(VP)]),
    "lag_precond_is_layered": (I, [VP]),
    "lag_precond_create_cyl": (I, [VP, C.POINTER(lag_grid), D, D, D, D, I, I, C.POINTER(VP)]),
    "lag_precond_destroy": (None, [VP]),
    "lag_precond_apply": (I, [VP, VP, VP, I]),
    "lag_precond_dst": (I, [VP, VP, VP, I]),
    "lag_precond_dst_inverse": (I, [VP, VP, VP, I]),
    "lag_precond_dst_f32": (I, [VP, VP, VP, I]),
    "lag_precond_tridiag": (I, [VP, VP, VP, I]),
    "lag_precond_tridiag_f32": (I, [VP, VP, VP, I]),
    "lag_precond_apply_static": (I, [VP, VP, VP, I]),
    "lag_precond_static_capacity": (C.c_size_t, []),
    "lag_precond_info": (I, [VP, PI, PI, PI]),
    "lag_precond_autotune": (I, [VP, I, PI, PI, PI, PD]),
    "lag_precond_set_layout": (I, [VP, I, I]),
    "lag_precond_uses_tensor_cores": (I, [VP]),
    "lag_precond_dst_gemm": (I, [VP, I]),
    "lag_precond_set_dst_products": (I, [VP, I]),
    "lag_medium_create_acoustic": (I, [VP, C.POINTER(lag_grid), PD, PD, D, C.POINTER(VP)]),
    "lag_medium_create_elastic": (I, [VP, C.POINTER(lag_grid), PD, PD, PD, D, C.POINTER(VP)]),
    "lag_medium_destroy": (None, [VP]),
    "lag_medium_midranges": (I, [VP, PD]),
    "lag_apply_operator": (I, [VP, VP, VP, I]),
    "lag_solve_system": (I, [VP, VP, VP, VP, VP, I, C.POINTER(lag_solver), PI, PD]),
    "lag_source_coeffs": (I, [VP, C.POINTER(lag_laguerre), C.POINTER(lag_wavelet), PD]),
    "lag_laguerre_table": (I, [VP, C.POINTER(lag_laguerre), I, PD, PD]),
    "lag_shot_create": (I, [VP, C.POINTER(lag_grid), PD, PD, PD, C.POINTER(lag_laguerre), C.POINTER(lag_solver),
                            C.POINTER(lag_wavelet), I, C.POINTER(lag_point), I, C.POINTER(lag_point), I, PD,
                            C.POINTER(VP)]),
    "lag_shot_destroy": (None, [VP]),
    "lag_shot_step": (I, [VP, I]),
    "lag_shot_pump": (I, [VP, PI]),
    "lag_shot_harmonic": (I, [VP]),
    "lag_shot_stream": (VP, [VP]),
    "lag_shot_traces": (I, [VP, PD]),
    "lag_shot_receiver_harmonics": (I, [VP, PD]),
    "lag_shot_field": (VP, [VP]),
    "lag_shot_copy_field": (I, [VP, VP]),
    "lag_shot_stats": (I, [VP, C.POINTER(lag_stats)]),
    "lag_precond_status": (I, [VP]),
    "lag_dst_f64_slice_products": (I, [I]),
    "lag_shot_checkpoint_size": (C.c_size_t, [VP]),
    "lag_shot_checkpoint": (I, [VP, VP, C.c_size_t]),
    "lag_shot_restore": (I, [VP, VP, C.c_size_t]),
    "lag_selftest_wait_timeout": (I, [VP, C.c_longlong]),
    "lag_solve_acoustic": (I, [VP, C.POINTER(lag_grid), PD, PD, C.POINTER(lag_laguerre), C.POINTER(lag_solver),
                               C.POINTER(lag_wavelet), I, C.POINTER(lag_point), I, C.POINTER(lag_point), I, PD, PD,
                               C.POINTER(lag_stats)]),
    "lag_solve_elastic": (I, [VP, C.POINTER(lag_grid), PD, PD, PD, C.POINTER(lag_laguerre), C.POINTER(lag_solver),
                              C.POINTER(lag_wavelet), I, C.POINTER(lag_point), I, C.POINTER(lag_point), I, PD, PD,
                              C.POINTER(lag_stats)]),
    "lag_serve_start": (I, [VP, I]),
    "lag_serve_stop": (I, [VP]),
    "lag_serve_submit": (I, [VP, C.POINTER(lag_request), C.POINTER(C.c_uint64)]),
    "lag_serve_poll": (I, [VP, C.c_uint64, C.POINTER(lag_result)]),
    "lag_serve_cancel": (I, [VP, C.c_uint64]),
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1005_0542_gb300.build` "
                           "(there is no fallback implementation)")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = load()
globals().update({name: getattr(lib, name) for name in _PROTOS})


class LagError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib.lag_strerror(status).decode()} ({status}): {msg}")
        self.status = status


def check(status, ctx=None, ok=(LAG_OK,)):
    """Raise LagError unless ``status`` is in ``ok``; returns the status."""
    if status not in ok:
        msg = lib.lag_last_error(ctx).decode() if ctx is not None else lib.lag_last_error(None).decode()
        raise LagError(status, msg)
    return status


# ---------------------------------------------------------------------------- marshalling helpers
def f64(a):
    """float64, C-contiguous copy/view and its double* pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(PD)


def points(pts):
    arr = (lag_point * max(1, len(pts)))()
    for i, (ix, iz) in enumerate(pts):
        arr[i].ix, arr[i].iz = int(ix), int(iz)
    return arr


def grid(nx, nz, dx, dz, free_surface=False, cylindrical=False):
    """Cartesian grid, or with cylindrical=True the axisymmetric (r, z) grid of nx radii and nz
    depths (fields [nx][nz], depth fastest; a free surface on top by construction)."""
    if cylindrical:
        free_surface = True
    return lag_grid(int(nx), int(nz), float(dx), float(dz), 1 if free_surface else 0, 1 if cylindrical else 0)


def solver(tol=1e-10, max_iter=2000, restart_k=20, prec=LAG_FP64, partitions=0, tune=0, layered=0):
    return lag_solver(float(tol), int(max_iter), int(restart_k), int(prec), int(partitions), int(tune),
                      int(layered))


def laguerre(h, alpha, n_harm):
    return lag_laguerre(float(h), int(alpha), int(n_harm))


def wavelet(f0, t0, gamma=4.0, kind=LAG_WAVELET_RICKER):
    return lag_wavelet(float(f0), float(t0), float(gamma), int(kind))


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream (torch's default stream, handle 0)


def create(device=0, budget=0, stream=None):
    """lag_create; ``stream`` is a cudaStream_t as an int (0 = the legacy default stream),
    or None for a stream of the library's own."""
    ctx = VP()
    if stream is not None and int(stream) == 0:
        stream = CUDA_STREAM_LEGACY
    check(lib.lag_create(C.byref(ctx), int(device), int(budget), VP(stream) if stream is not None else None))
    return ctx
