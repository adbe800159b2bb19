"""Layered preconditioner (per-row midranges kappa~(z), rho~(z): an extension of Eq. 21 that keeps
Sec. 2.4's separation of variables): the partitioned tridiagonal solve with one factor set per
partition, the whole plan on both paths, layout changes and the autotuner, and shots, each
against the oracle (oracle.precond.apply_inverse_layered, oracle.solve.acoustic_shot)."""
import ctypes as C

import numpy as np
import pytest

from oracle import dst as odst, precond as opre, solve
from oracle.tridiag import thomas
from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, plan, plan_info, ptr, rel, rel_l2

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2207)


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


def rows(nz, contrast=8.0):
    """Per-row coefficients of a strongly layered acoustic medium (kappa in Pa, rho h^2/4)."""
    ax = 2.0e9 * RNG.uniform(1.0, contrast, nz)
    az = ax * RNG.uniform(0.8, 1.25, nz)
    d = RNG.uniform(1.0e6, 5.0e7, nz)
    return ax, az, d


def layered_plan(ctx, nx, nz, dx, dz, ax, az, d, prec=L.LAG_FP64, partitions=0, free_surface=False):
    p = C.c_void_p()
    g = L.grid(nx, nz, dx, dz, free_surface)
    a_, pa = L.f64(ax)
    z_, pz = L.f64(az)
    d_, pd = L.f64(d)
    L.check(L.lag_precond_create_layered(ctx, C.byref(g), pa, pz, pd, prec, partitions, C.byref(p)), ctx)
    assert L.lag_precond_is_layered(p) == 1
    return p


def zsolve_ref(rhs, dx, dz, ax, az, d, free_surface):
    """T_j^{-1} along z for every mode j (the layered rows of the oracle), rhs [b, nz, nx]."""
    nz, nx = rhs.shape[-2:]
    f = opre._z_faces(np.asarray(az, dtype=np.float64), free_surface)
    lam = odst.laplace_eigenvalues(nx, dx)
    sub = (-f[:nz] / dz ** 2)[:, None, None]
    sup = (-f[1:] / dz ** 2)[:, None, None]
    diag = ((f[:nz] + f[1:]) / dz ** 2)[:, None] + ax[:, None] * lam[None, :] + d[:, None]
    col = np.moveaxis(rhs, 1, 0)
    return np.moveaxis(thomas(sub, diag[:, None, :], sup, col), 0, 1)


@pytest.mark.parametrize("P", [1, 2, 4, 8, 32])
@pytest.mark.parametrize("nz,nx", [(4, 3), (100, 64), (1024, 40), (777, 130)])
def test_tridiag_layered_every_partition_count(ctx, P, nz, nx):
    dx, dz = 5.0, 3.0
    ax, az, d = rows(nz)
    p = layered_plan(ctx, nx, nz, dx, dz, ax, az, d, partitions=P)
    rhs = RNG.standard_normal((3, nz, nx))
    dd, yd = dev(rhs), empty(rhs.shape)
    L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(yd), 3), ctx)
    assert rel(host(yd), zsolve_ref(rhs, dx, dz, ax, az, d, False)) < 1e-12
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("free_surface", [False, True])
@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
@pytest.mark.parametrize("nz,nx", [(33, 20), (128, 128), (64, 1024), (300, 257)])
def test_precond_apply_layered(ctx, free_surface, prec, tol, nz, nx):
    dx, dz = 5.0, 5.0
    ax, az, d = rows(nz)
    p = layered_plan(ctx, nx, nz, dx, dz, ax, az, d, prec=prec, free_surface=free_surface)
    r = RNG.standard_normal((2, nz, nx))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    ref = opre.apply_inverse_layered(r, dx, dz, ax, az, d, free_surface)
    assert rel(host(zd), ref) < tol
    # and it is not the constant-coefficient preconditioner
    const = opre.apply_inverse(r, dx, dz, opre.midrange(ax), opre.midrange(az), opre.midrange(d), free_surface)
    assert rel(const, ref) > 10 * tol
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-13), (L.LAG_MIXED, 2e-4)])
def test_layered_with_constant_rows_is_the_constant_plan(ctx, prec, tol):
    nz, nx, dx, dz, ax, az, d = 96, 200, 5.0, 4.0, 3.0e9, 2.0e9, 1.0e7
    one = np.ones(nz)
    pl = layered_plan(ctx, nx, nz, dx, dz, ax * one, az * one, d * one, prec=prec)
    pc = plan(ctx, nx, nz, dx, dz, ax, az, d, prec=prec)
    r = RNG.standard_normal((2, nz, nx))
    rd, zl, zc = dev(r), empty(r.shape), empty(r.shape)
    L.check(L.lag_precond_apply(pl, ptr(rd), ptr(zl), 2), ctx)
    L.check(L.lag_precond_apply(pc, ptr(rd), ptr(zc), 2), ctx)
    assert rel(host(zl), host(zc)) < tol
    assert rel(host(zl), opre.apply_inverse(r, dx, dz, ax, az, d)) < tol
    L.lag_precond_destroy(pl)
    L.lag_precond_destroy(pc)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
def test_layered_layouts_and_autotune(ctx, prec, tol):
    nz, nx, dx, dz = 512, 384, 5.0, 5.0
    ax, az, d = rows(nz)
    p = layered_plan(ctx, nx, nz, dx, dz, ax, az, d, prec=prec)
    r = RNG.standard_normal((4, nz, nx))
    ref = opre.apply_inverse_layered(r, dx, dz, ax, az, d)
    rd, zd = dev(r), empty(r.shape)
    tiles = (4, 8) if prec == L.LAG_FP64 else (8, 16, 32)
    # P = 8: partitions of 64 rows (shared-memory tile kernel for float64); 16, 32: register kernel
    for P, mts in ((8, (0,)), (16, tiles), (32, tiles)):
        for mt in mts:
            L.check(L.lag_precond_set_layout(p, P, mt), ctx)
            assert plan_info(p)[0] == P and (mt == 0 or plan_info(p)[2] == mt)
            L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 4), ctx)
            assert rel(host(zd), ref) < tol, (P, mt)
    Pt, mtt, prod, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    L.check(L.lag_precond_autotune(p, 4, C.byref(Pt), C.byref(mtt), C.byref(prod), C.byref(ms)), ctx)
    assert L.lag_precond_is_layered(p) == 1
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 4), ctx)
    # the tuner may drop bf16 products of the mixed DST (fewer products: a coarser preconditioner)
    assert rel(host(zd), ref) < (tol if prec == L.LAG_FP64 or prod.value == 3 else 2e-2)
    L.lag_precond_destroy(p)


def test_layered_plan_rejects_bad_rows(ctx):
    nz, nx = 16, 16
    ax, az, d = rows(nz)
    g = L.grid(nx, nz, 5.0, 5.0)
    p = C.c_void_p()
    for bad in (ax * 0.0, -ax, np.full(nz, np.nan)):
        b_, pb = L.f64(bad)
        z_, pz = L.f64(az)
        d_, pd = L.f64(d)
        assert L.lag_precond_create_layered(ctx, C.byref(g), pb, pz, pd, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL
    a_, pa = L.f64(ax)
    z_, pz = L.f64(az)
    d_, pd = L.f64(-d)
    assert L.lag_precond_create_layered(ctx, C.byref(g), pa, pz, pd, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL


def _shot(ctx, s, prec, tol, layered, free_surface=False):
    g = L.grid(s.nx, s.nz, s.hx, s.hz, free_surface)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=tol, prec=prec, layered=layered)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    traces = np.zeros((1, 1, len(s.receivers), s.t_out.size))
    its = np.zeros((1, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    L.check(L.lag_solve_acoustic(ctx, C.byref(g), pc, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                                 L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                 traces.ctypes.data_as(L.PD), C.byref(st)), ctx)
    return traces[0, 0], its[0]


@pytest.mark.parametrize("free_surface", [False, True])
@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_layered_shot_matches_oracle(ctx, free_surface, prec, tol, gate):
    s = inputs.random_layered(nx=96, nz=64, hx=10.0, n_harm=10)
    tr, its = _shot(ctx, s, prec, tol, 1, free_surface)
    ref = solve.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                              s.t_out, s.f0, s.t0, tol=tol, free_surface=free_surface, layered=True)
    assert rel_l2(tr, ref["traces"]) < gate
    if prec == L.LAG_FP64:  # the same Krylov iteration as the oracle's, to a step
        assert np.abs(its - ref["iters"]).max() <= 1
    _, its_c = _shot(ctx, s, prec, tol, 0, free_surface)
    assert its.sum() * 2 < its_c.sum()


def test_layered_shot_one_iteration_on_a_z_only_medium(ctx):
    # kappa and rho depending on z only: the layered preconditioner is A itself
    s = inputs.random_layered(nx=80, nz=48, hx=10.0, n_harm=6)
    s.c = np.repeat(s.c[:, :1], s.nx, axis=1)
    s.rho = np.repeat(s.rho[:, :1], s.nx, axis=1)
    _, its = _shot(ctx, s, L.LAG_FP64, 1e-10, 1)
    assert np.all(its == 1), its


def _elastic_shot(ctx, s, prec, tol, layered):
    g = L.grid(s.nx, s.nz, s.hx, s.hz)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=tol, prec=prec, restart_k=s.restart, layered=layered)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    traces = np.zeros((1, 2, len(s.receivers), s.t_out.size))
    its = np.zeros((1, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    L.check(L.lag_solve_elastic(ctx, C.byref(g), pc, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                                L.points(s.sources[:1]), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                                traces.ctypes.data_as(L.PD), C.byref(st)), ctx)
    return traces[0], its[0]


@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_layered_elastic_shot_matches_oracle(ctx, prec, tol, gate):
    # Eq. 22's K with per-row midranges (B1: (l+2m)~(z), mu~(z); B2 swapped) on the layered elastic
    # model with its dipping interface: the traces of the oracle's layered FGMRES, fewer iterations
    # than with the whole-medium K
    s = inputs.elastic_layered(nx=64, nz=40, hx=2.5, n_harm=6, nsrc=1)
    s.receivers = s.receivers[:8]
    tr, its = _elastic_shot(ctx, s, prec, tol, 1)
    ref = solve.elastic_shot(s.c, s.vs, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                             s.t_out, s.f0, s.t0, tol=tol, restart=s.restart, layered=True)
    assert rel_l2(tr, ref["traces"]) < gate
    if prec == L.LAG_FP64:
        assert np.abs(its - ref["iters"]).max() <= 1
        _, its_c = _elastic_shot(ctx, s, prec, tol, 0)
        assert its.sum() < its_c.sum(), (its, its_c)


def test_layered_cylindrical_elastic_rejected(ctx):
    s = inputs.cylindrical(nr=16, nz=12, h=10.0, n_harm=2, elastic=True)
    g = L.grid(s.nx, s.nz, s.hx, s.hz, cylindrical=True)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=1e-8, layered=1)
    w = L.wavelet(s.f0, s.t0)
    c_, pc = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    traces = np.zeros((1, 2, len(s.receivers), s.t_out.size))
    rc = L.lag_solve_elastic(ctx, C.byref(g), pc, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                             L.points(s.sources[:1]), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                             traces.ctypes.data_as(L.PD), None)
    assert rc == L.LAG_EINVAL
