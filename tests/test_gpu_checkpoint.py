"""Checkpoint / resume of a shot, and failure detection through a bounded device wait.

A shot interrupted after harmonic k, written to host memory and resumed in a new shot (as after a
process restart), gives traces, receiver harmonics and iteration counts equal bit for bit to the
uninterrupted run: the state between harmonics is exactly m, the history sums T and S of Eq. 9,
the receiver values so far and the statistics.  The failure test makes a device wait run out on
purpose (a barrier nothing arrives on) and checks that the error comes back as a status with the
context still usable; nothing faults or hangs the GPU.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


def _create(ctx, s, prec, elastic=False):
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=1e-11, prec=prec, restart_k=s.restart)
    w = L.wavelet(s.f0, s.t0)
    keep = [L.f64(s.c), L.f64(s.rho), L.f64(s.t_out)]
    pv = None
    if elastic:
        keep.append(L.f64(s.vs))
        pv = keep[-1][1]
    sh = C.c_void_p()
    L.check(L.lag_shot_create(ctx, C.byref(g), keep[0][1], pv, keep[1][1], C.byref(lag), C.byref(sv), C.byref(w),
                              len(s.sources), L.points(s.sources), len(s.receivers), L.points(s.receivers),
                              s.t_out.size, keep[2][1], C.byref(sh)), ctx)
    return sh


def _outputs(ctx, sh, s, ncomp):
    traces = np.zeros((len(s.sources), ncomp, len(s.receivers), s.t_out.size))
    rr = np.zeros((s.n_harm, len(s.sources), ncomp, len(s.receivers)))
    its = np.zeros((len(s.sources), s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    L.check(L.lag_shot_traces(sh, traces.ctypes.data_as(L.PD)), ctx)
    L.check(L.lag_shot_receiver_harmonics(sh, rr.ctypes.data_as(L.PD)), ctx)
    L.check(L.lag_shot_stats(sh, C.byref(st)), ctx)
    return traces, rr, its, st.total_iters


@pytest.mark.parametrize("prec,elastic", [(L.LAG_FP64, False), (L.LAG_MIXED, False), (L.LAG_FP64, True)])
def test_resume_equals_uninterrupted(ctx, prec, elastic):
    if elastic:
        s = inputs.elastic_layered(nx=40, nz=24, hx=2.5, n_harm=8, nsrc=2)
        s.receivers = s.receivers[:6]
    else:
        s = inputs.random_layered(nx=96, nz=72, hx=12.0, n_harm=12, sources=[(10, 3), (60, 40)], f0=12.0)
        s.receivers = s.receivers[:12]
    ncomp = 2 if elastic else 1
    ref = _create(ctx, s, prec, elastic)
    L.check(L.lag_shot_step(ref, s.n_harm), ctx)
    want = _outputs(ctx, ref, s, ncomp)
    L.lag_shot_destroy(ref)

    k = 5
    a = _create(ctx, s, prec, elastic)
    L.check(L.lag_shot_step(a, k), ctx)
    nbytes = L.lag_shot_checkpoint_size(a)
    assert nbytes > 0
    buf = (C.c_ubyte * nbytes)()
    L.check(L.lag_shot_checkpoint(a, buf, nbytes), ctx)
    L.lag_shot_destroy(a)

    b = _create(ctx, s, prec, elastic)
    L.check(L.lag_shot_restore(b, buf, nbytes), ctx)
    assert L.lag_shot_harmonic(b) == k
    L.check(L.lag_shot_step(b, s.n_harm), ctx)
    got = _outputs(ctx, b, s, ncomp)
    L.lag_shot_destroy(b)
    for w_, g_ in zip(want[:3], got[:3]):
        assert np.array_equal(w_, g_)
    assert want[3] == got[3]
    assert rel_l2(got[0], want[0]) == 0.0


def test_restore_rejects_mismatch(ctx):
    s = inputs.random_layered(nx=64, nz=48, hx=12.0, n_harm=6, sources=[(10, 3)], f0=12.0)
    s.receivers = s.receivers[:4]
    a = _create(ctx, s, L.LAG_FP64)
    L.check(L.lag_shot_step(a, 2), ctx)
    nbytes = L.lag_shot_checkpoint_size(a)
    buf = (C.c_ubyte * nbytes)()
    assert L.lag_shot_checkpoint(a, buf, nbytes - 1) == L.LAG_EINVAL   # buffer too small
    L.check(L.lag_shot_checkpoint(a, buf, nbytes), ctx)
    s2 = inputs.random_layered(nx=64, nz=40, hx=12.0, n_harm=6, sources=[(10, 3)], f0=12.0)
    s2.receivers = s2.receivers[:4]
    b = _create(ctx, s2, L.LAG_FP64)                                    # other grid
    assert L.lag_shot_restore(b, buf, nbytes) == L.LAG_EINVAL
    bad = bytearray(buf)
    bad[0] ^= 0xFF                                                      # not a checkpoint
    badbuf = (C.c_ubyte * nbytes).from_buffer(bad)
    assert L.lag_shot_restore(a, badbuf, nbytes) == L.LAG_EINVAL
    L.check(L.lag_shot_step(a, 1), ctx)                                 # the shot is still usable
    assert L.lag_shot_harmonic(a) == 3
    L.lag_shot_destroy(a)
    L.lag_shot_destroy(b)


def test_bounded_wait_reports_timeout(ctx):
    # a wait that nothing ends gives up after its poll limit and returns a status
    assert L.lag_selftest_wait_timeout(ctx, 2000) == L.LAG_ETIMEDOUT
    assert b"bounded device wait" in L.lag_last_error(ctx)
    assert L.lag_selftest_wait_timeout(ctx, 0) == L.LAG_EINVAL
    # the context keeps working afterwards: a solve on it still succeeds
    s = inputs.random_layered(nx=48, nz=32, hx=12.0, n_harm=3, sources=[(10, 3)], f0=12.0)
    s.receivers = s.receivers[:3]
    sh = _create(ctx, s, L.LAG_FP64)
    L.check(L.lag_shot_step(sh, 3), ctx)
    assert L.lag_shot_harmonic(sh) == 3
    L.lag_shot_destroy(sh)


def test_precond_status_clean_after_applies(ctx):
    # the tensor-core DST's error word stays clear over ordinary applies
    from gpu_util import dev, empty, plan, ptr
    nz, nx = 64, 96
    p = plan(ctx, nx, nz, 5.0, 5.0, 2.0, 2.0, 0.5, prec=L.LAG_MIXED)
    r = dev(np.random.default_rng(5).standard_normal((3, nz, nx)))
    z = empty((3, nz, nx))
    for _ in range(3):
        L.check(L.lag_precond_apply(p, ptr(r), ptr(z), 3), ctx)
    assert L.lag_precond_status(p) == L.LAG_OK
    assert L.lag_precond_status(None) == L.LAG_EINVAL
    L.lag_precond_destroy(p)
