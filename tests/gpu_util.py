"""Helpers of the GPU parity tests: device arrays through torch, C-ABI objects."""
import ctypes as C

import numpy as np

from paper_1005_0542_gb300 import lagwave as L


def torch():
    import torch as t
    return t


def make_ctx():
    """A context whose stream is torch's current stream, so that library work is ordered after
    the torch kernels that produced its inputs."""
    t = torch()
    return L.create(0, stream=t.cuda.current_stream().cuda_stream)


def dev(a, dtype=None):
    t = torch()
    a = np.ascontiguousarray(a)
    x = t.from_numpy(a).cuda()
    return x if dtype is None else x.to(dtype)


def empty(shape, dtype=None):
    t = torch()
    return t.empty(shape, dtype=dtype or t.float64, device="cuda")


def ptr(x):
    return C.c_void_p(x.data_ptr())


def host(x):
    torch().cuda.synchronize()
    return x.detach().cpu().numpy()


def rel(a, b):
    """max |a - b| / max |b| (b the oracle)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (s if s > 0 else 1.0))


def plan(ctx, nx, nz, dx, dz, ax, az, d, prec=L.LAG_FP64, partitions=0, free_surface=False):
    p = C.c_void_p()
    g = L.grid(nx, nz, dx, dz, free_surface)
    L.check(L.lag_precond_create_sep(ctx, C.byref(g), ax, az, d, prec, partitions, C.byref(p)), ctx)
    return p


def plan_info(p):
    P, Lp, mt = C.c_int(), C.c_int(), C.c_int()
    L.check(L.lag_precond_info(p, C.byref(P), C.byref(Lp), C.byref(mt)))
    return P.value, Lp.value, mt.value


def medium(ctx, nx, nz, dx, dz, c, rho, h, vs=None, free_surface=False):
    m = C.c_void_p()
    g = L.grid(nx, nz, dx, dz, free_surface)
    c_, pc = L.f64(c)
    r_, pr = L.f64(rho)
    if vs is None:
        L.check(L.lag_medium_create_acoustic(ctx, C.byref(g), pc, pr, h, C.byref(m)), ctx)
    else:
        v_, pv = L.f64(vs)
        L.check(L.lag_medium_create_elastic(ctx, C.byref(g), pc, pv, pr, h, C.byref(m)), ctx)
    return m
