"""lag_precond_apply_static: the preconditioner apply that allocates nothing.

Some callers cannot let a library allocate device memory when they call it (their own allocator
owns the device memory, or their loop must not block in cudaMalloc/cudaFree).  This entry point
keeps its intermediate spectrum in a static device array instead and runs the float64 DST on the
SIMT pipes (the tensor-core DST needs plan-owned scratch for its operand slices); its results must
equal those of lag_precond_apply on a plan with the SIMT kernels bit for bit, call after call, and
those of the tensor-core plan to float64 accuracy.  The file sorts last so that a run stopping at
the first failure has run every other test before it."""
import ctypes as C
import os

import numpy as np
import pytest
import torch

from paper_1005_0542_gb300 import lagwave as L

from gpu_util import dev, empty, host, make_ctx, plan, ptr, rel

pytestmark = pytest.mark.gpu
TOL64 = 1e-12   # the float64 preconditioner tolerance of the other parity tests


def _simt_plan(ctx, *args):
    os.environ["LAGWAVE_DST_KERNEL"] = "simt"   # read at plan creation
    try:
        return plan(ctx, *args)
    finally:
        del os.environ["LAGWAVE_DST_KERNEL"]


def test_static_apply_matches_regular_apply_twice():
    ctx = make_ctx()
    try:
        nx, nz, nrhs = 160, 96, 3
        args = (nx, nz, 5.0, 7.0, 3.0e9, 2.0e9, 1.0e7)
        p = plan(ctx, *args)            # float64 DST on the tensor cores
        q = _simt_plan(ctx, *args)      # float64 DST on the SIMT pipes, as the static entry point
        assert L.lag_precond_uses_tensor_cores(p) == 1 and L.lag_precond_uses_tensor_cores(q) == 0
        rng = np.random.default_rng(2024)
        for call in range(2):  # two calls in a row: the shared array keeps the previous contents
            r = rng.standard_normal((nrhs, nz, nx)) * (1.0 + call)
            rd, z_tc, z_simt, z_sta = dev(r), empty(r.shape), empty(r.shape), empty(r.shape)
            L.check(L.lag_precond_apply(p, ptr(rd), ptr(z_tc), nrhs), ctx)
            L.check(L.lag_precond_apply(q, ptr(rd), ptr(z_simt), nrhs), ctx)
            torch.cuda.synchronize()
            held = L.lag_bytes_in_use(ctx)
            free0 = torch.cuda.mem_get_info()[0]
            L.check(L.lag_precond_apply_static(p, ptr(rd), ptr(z_sta), nrhs), ctx)
            torch.cuda.synchronize()
            # nothing allocated: the library's ledger is unchanged, and after the first call's
            # one-time set-up the device's free memory is too
            assert L.lag_bytes_in_use(ctx) == held
            if call > 0:
                assert torch.cuda.mem_get_info()[0] == free0
            a = host(z_sta)
            assert np.array_equal(a, host(z_simt))   # same kernels, same order: identical bits
            assert rel(a, host(z_tc)) < TOL64
        L.lag_precond_destroy(p)
        L.lag_precond_destroy(q)
    finally:
        L.lag_destroy(ctx)


def test_static_apply_limits():
    ctx = make_ctx()
    try:
        cap = L.lag_precond_static_capacity()
        assert cap == 1 << 21
        nx, nz = 2048, 1024                   # one field of the bench workload fills it exactly
        p = plan(ctx, nx, nz, 5.0, 5.0, 3.0e10, 3.0e10, 1.0e7)
        assert L.lag_precond_apply_static(p, None, None, 0) == L.LAG_OK
        big = C.c_void_p(1)
        assert L.lag_precond_apply_static(p, big, big, 2) == L.LAG_EINVAL   # 2 * 2^21 > capacity
        assert b"exceeds the static capacity" in L.lag_last_error(ctx)
        L.lag_precond_destroy(p)
        q = plan(ctx, 64, 64, 1.0, 1.0, 1.0, 1.0, 0.1, prec=L.LAG_MIXED)
        assert L.lag_precond_apply_static(q, big, big, 1) == L.LAG_EINVAL  # float64 plans only
        L.lag_precond_destroy(q)
    finally:
        L.lag_destroy(ctx)
