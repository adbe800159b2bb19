"""Free surface at z = 0 (Sec. 2.1, Eq. 3: du/dz = 0): the operator, the partitioned tridiagonal
solve (its first partition's factors carry the changed first row), the preconditioner on both
paths, PCG and a whole shot, each against the oracle with the same zero-flux reading."""
import ctypes as C

import numpy as np
import pytest

from oracle import fd, laguerre, precond as opre, solve
from oracle.tridiag import thomas
from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, medium, plan, plan_info, ptr, rel, rel_l2, torch

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2101)


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


@pytest.mark.parametrize("nz,nx", [(1, 1), (2, 3), (23, 37), (70, 257)])
def test_operator_free_surface(ctx, nz, nx):
    c = RNG.uniform(1500, 4500, (nz, nx))
    rho = RNG.uniform(1000, 2600, (nz, nx))
    h, dx, dz = 200.0, 5.0, 7.5
    m = medium(ctx, nx, nz, dx, dz, c, rho, h, free_surface=True)
    p = RNG.standard_normal((2, nz, nx))
    pd, qd = dev(p), empty(p.shape)
    L.check(L.lag_apply_operator(m, ptr(pd), ptr(qd), 2), ctx)
    ref = fd.apply_A(p, fd.kappa_from_velocity(c, rho), rho, h, dx, dz, free_surface=True)
    assert rel(host(qd), ref) < 1e-14
    L.lag_medium_destroy(m)


@pytest.mark.parametrize("P", [1, 2, 4, 8, 32])
@pytest.mark.parametrize("nz,nx", [(4, 3), (100, 64), (1024, 40)])
def test_tridiag_free_surface_every_partition_count(ctx, P, nz, nx):
    dx, dz, ax, az, d = 5.0, 3.0, 2.0e9, 1.5e9, 4.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, partitions=P, free_surface=True)
    rhs = RNG.standard_normal((2, nz, nx))
    diag = np.broadcast_to(opre.mode_diagonals(nx, dx, dz, ax, az, d), (nz, nx)).copy()
    diag[0] -= az / dz ** 2
    off = -az / dz ** 2
    ref = np.moveaxis(thomas(off, diag[:, None, :], off, np.moveaxis(rhs, 1, 0)), 0, 1)
    dd, yd = dev(rhs), empty(rhs.shape)
    L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(yd), 2), ctx)
    assert rel(host(yd), ref) < 1e-13
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
@pytest.mark.parametrize("nz,nx", [(33, 20), (128, 128), (64, 1024)])
def test_precond_apply_free_surface(ctx, prec, tol, nz, nx):
    dx, dz, ax, az, d = 5.0, 5.0, 2.0e10, 2.0e10, 1.0e7
    p = plan(ctx, nx, nz, dx, dz, ax, az, d, prec=prec, free_surface=True)
    r = RNG.standard_normal((2, nz, nx))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    ref = opre.apply_inverse(r, dx, dz, ax, az, d, free_surface=True)
    assert rel(host(zd), ref) < tol
    # and it differs from the Dirichlet preconditioner where the surface matters
    assert rel(opre.apply_inverse(r, dx, dz, ax, az, d), ref) > 10 * tol
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_shot_free_surface(ctx, prec, tol, gate):
    # a layered model with a free surface, source and receivers just below it
    s = inputs.random_layered(nx=96, nz=64, hx=10.0, n_harm=12, sources=[(48, 2)], f0=12.0)
    s.receivers = [(i, 0) for i in range(4, 92, 8)]
    g = L.grid(s.nx, s.nz, s.hx, s.hz, free_surface=True)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=tol, prec=prec)
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
    ref = solve.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                              s.t_out, s.f0, s.t0, tol=tol, free_surface=True)
    assert rel_l2(traces[0, 0], ref["traces"]) < gate
    dirichlet = solve.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                                    s.t_out, s.f0, s.t0, tol=tol)
    assert rel_l2(dirichlet["traces"], ref["traces"]) > 1e-2    # the surface changes the traces


def test_elastic_free_surface_rejected(ctx):
    s = inputs.elastic_layered(nx=16, nz=12, hx=2.5, n_harm=2, nsrc=1)
    m = C.c_void_p()
    g = L.grid(s.nx, s.nz, s.hx, s.hz, free_surface=True)
    c_, pc = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    assert L.lag_medium_create_elastic(ctx, C.byref(g), pc, pv, pr, s.h, C.byref(m)) == L.LAG_EINVAL
