"""Serving loop: continuous batching of shots, admission by HBM budget, per-request faults.

Faults are made on the host (an input with a NaN, a cancelled request, a budget too small);
nothing here faults or stalls the GPU."""
import ctypes as C
import time

import numpy as np
import pytest

from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

pytestmark = pytest.mark.gpu


def _request(s, elastic=False, prec=L.LAG_FP64, keep=None):
    keep = [] if keep is None else keep
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    src, rcv = L.points(s.sources), L.points(s.receivers)
    keep += [c_, r_, t_, src, rcv]
    req = L.lag_request()
    req.kind = 1 if elastic else 0
    req.grid = L.grid(s.nx, s.nz, s.hx, s.hz)
    req.c_host, req.rho_host = pc, pr
    if elastic:
        v_, pv = L.f64(s.vs)
        keep.append(v_)
        req.vs_host = pv
    req.lag = L.laguerre(s.h, s.alpha, s.n_harm)
    req.solver = L.solver(tol=1e-10, prec=prec, restart_k=s.restart)
    req.wavelet = L.wavelet(s.f0, s.t0)
    req.nsrc, req.src = len(s.sources), C.cast(src, C.POINTER(L.lag_point))
    req.nrcv, req.rcv = len(s.receivers), C.cast(rcv, C.POINTER(L.lag_point))
    req.nt, req.t_out_host = s.t_out.size, pt
    return req, keep


def _alone(ctx, s, elastic=False, prec=L.LAG_FP64):
    ncomp = 2 if elastic else 1
    tr = np.zeros((len(s.sources), ncomp, len(s.receivers), s.t_out.size))
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=1e-10, prec=prec, restart_k=s.restart)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    if elastic:
        v_, pv = L.f64(s.vs)
        rc = L.lag_solve_elastic(ctx, C.byref(g), pc, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), len(s.sources),
                                 L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                 tr.ctypes.data_as(L.PD), None)
    else:
        rc = L.lag_solve_acoustic(ctx, C.byref(g), pc, pr, C.byref(lag), C.byref(sv), C.byref(w), len(s.sources),
                                  L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                  tr.ctypes.data_as(L.PD), None)
    L.check(rc, ctx)
    return tr


def _wait(ctx, ticket, shape, timeout=300.0):
    out = np.zeros(shape)
    res = L.lag_result()
    res.traces_host = out.ctypes.data_as(L.PD)
    t0 = time.time()
    while True:
        rc = L.lag_serve_poll(ctx, ticket, C.byref(res))
        if rc == L.LAG_OK:
            return res, out
        assert rc == L.LAG_EAGAIN
        assert time.time() - t0 < timeout
        time.sleep(0.002)


def _workload():
    a1 = inputs.two_layer(n_harm=10, nx=64, nz=48)
    a2 = inputs.random_layered(nx=96, nz=64, hx=10.0, n_harm=14, sources=[(10, 3), (50, 30)], f0=12.0)
    a2.receivers = a2.receivers[:8]
    e1 = inputs.elastic_layered(nx=40, nz=32, hx=2.5, n_harm=5, nsrc=1)
    e1.receivers = e1.receivers[:5]
    a3 = inputs.random_layered(nx=128, nz=40, hx=10.0, n_harm=8, seed=77, f0=12.0)
    a3.receivers = a3.receivers[:6]
    return [(a1, False), (a2, False), (e1, True), (a3, False)]


def test_results_same_alone_and_in_the_mix():
    ctx = L.create(0)
    try:
        work = _workload()
        alone = [_alone(ctx, s, el) for s, el in work]
        L.check(L.lag_serve_start(ctx, 4), ctx)
        keep, tickets = [], []
        for s, el in work:
            req, _ = _request(s, el, keep=keep)
            t = C.c_uint64()
            L.check(L.lag_serve_submit(ctx, C.byref(req), C.byref(t)), ctx)
            tickets.append(t.value)
        results = []
        for (s, el), t, ref in zip(work, tickets, alone):
            res, tr = _wait(ctx, t, ref.shape)
            assert res.status == L.LAG_OK
            assert np.array_equal(tr, ref)                      # bit-identical alone and in the mix
            assert res.t_submit <= res.t_admit <= res.t_done and res.total_iters > 0
            results.append(res)
        # requests overlapped on the device: a later one was admitted before an earlier one ended
        assert min(r.t_admit for r in results[1:]) < max(r.t_done for r in results[:1])
        L.check(L.lag_serve_stop(ctx), ctx)
    finally:
        L.lag_destroy(ctx)


def test_poisoned_request_fails_alone_others_finish():
    ctx = L.create(0)
    try:
        work = _workload()[:2]
        alone = [_alone(ctx, s, el) for s, el in work]
        bad = inputs.two_layer(n_harm=6, nx=32, nz=32)
        bad.rho = bad.rho.copy()
        bad.rho[5, 7] = np.nan                                   # a corrupted input on the host
        keep, tickets = [], []
        for s, el in [work[0], (bad, False), work[1]]:
            req, _ = _request(s, el, keep=keep)
            t = C.c_uint64()
            L.check(L.lag_serve_submit(ctx, C.byref(req), C.byref(t)), ctx)
            tickets.append(t.value)
        r0, tr0 = _wait(ctx, tickets[0], alone[0].shape)
        rb, _ = _wait(ctx, tickets[1], (1, 1, len(bad.receivers), bad.t_out.size))
        r2, tr2 = _wait(ctx, tickets[2], alone[1].shape)
        assert rb.status == L.LAG_ENUMERIC
        assert r0.status == L.LAG_OK and np.array_equal(tr0, alone[0])
        assert r2.status == L.LAG_OK and np.array_equal(tr2, alone[1])
    finally:
        L.lag_destroy(ctx)


def test_budget_admission_and_cancel():
    small = inputs.two_layer(n_harm=4, nx=32, nz=32)
    big = inputs.random_layered(nx=2048, nz=1024, hx=5.0, n_harm=4)   # ~8 float64 fields of 16.8 MB alone
    ctx = L.create(0, budget=96 << 20)
    try:
        keep = []
        rq_big, _ = _request(big, keep=keep)
        rq_small, _ = _request(small, keep=keep)
        tb, ts = C.c_uint64(), C.c_uint64()
        L.check(L.lag_serve_submit(ctx, C.byref(rq_big), C.byref(tb)), ctx)
        L.check(L.lag_serve_submit(ctx, C.byref(rq_small), C.byref(ts)), ctx)
        rb, _ = _wait(ctx, tb.value, (1, 1, len(big.receivers), big.t_out.size))
        assert rb.status == L.LAG_ENOMEM                        # can never fit the budget: rejected
        rs, _ = _wait(ctx, ts.value, (1, 1, len(small.receivers), small.t_out.size))
        assert rs.status == L.LAG_OK and rs.device_bytes <= 96 << 20
        # cancel a long request right after submitting it
        long = inputs.two_layer(n_harm=2000, nx=64, nz=64)
        rq_long, _ = _request(long, keep=keep)
        tl = C.c_uint64()
        L.check(L.lag_serve_submit(ctx, C.byref(rq_long), C.byref(tl)), ctx)
        L.check(L.lag_serve_cancel(ctx, tl.value), ctx)
        rl, _ = _wait(ctx, tl.value, (1, 1, len(long.receivers), long.t_out.size))
        assert rl.status == L.LAG_ECANCELED
        assert L.lag_serve_poll(ctx, tl.value, C.byref(L.lag_result())) == L.LAG_EINVAL  # already collected
    finally:
        L.lag_destroy(ctx)
