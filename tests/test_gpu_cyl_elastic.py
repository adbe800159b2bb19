"""The paper's 2.5D axisymmetric elastic problem (Sec. 2.2, Eq. 22) through the C ABI: the
energy-derived operator C on the (r, z) grid, the preconditioner blocks B1 (with its hoop term) and
B2, and elastic shots, each against the oracle (oracle.cyl_elastic).  Fields are [2][nr][nz]
(component 0 = Q = u_r, 1 = U = u_z; depth fastest)."""
import ctypes as C

import numpy as np
import pytest

from oracle import cyl_elastic as ce
from oracle.solve import elastic_lame
from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, ptr, rel, rel_l2

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2504)


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


def _medium_arrays(nr, nz):
    vp = RNG.uniform(2000, 5000, (nr, nz))
    vs = vp / RNG.uniform(1.5, 2.2, (nr, nz))
    rho = RNG.uniform(1800, 2600, (nr, nz))
    return vp, vs, rho


def _cyl_medium(ctx, vp, vs, rho, hr, hz, h):
    m = C.c_void_p()
    nr, nz = vp.shape
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    p_, pp = L.f64(vp)
    v_, pv = L.f64(vs)
    r_, pr = L.f64(rho)
    L.check(L.lag_medium_create_elastic(ctx, C.byref(g), pp, pv, pr, h, C.byref(m)), ctx)
    return m


@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 3), (5, 1), (23, 37), (70, 257), (129, 64)])
def test_operator_cylindrical_elastic(ctx, nr, nz):
    hr, hz, h = 5.0, 7.5, 300.0
    vp, vs, rho = _medium_arrays(nr, nz)
    m = _cyl_medium(ctx, vp, vs, rho, hr, hz, h)
    u = RNG.standard_normal((2, 2, nr, nz))              # [rhs][comp][r][z]
    ud, qd = dev(u), empty(u.shape)
    L.check(L.lag_apply_operator(m, ptr(ud), ptr(qd), 2), ctx)
    lam, mu = elastic_lame(vp, vs, rho)
    co = ce.coefficients(lam, mu, hr, hz)
    got = host(qd)
    for b in range(2):
        cq, cu = ce.apply_C(u[b, 0], u[b, 1], co, rho, h, hr, hz)
        assert rel(got[b, 0], cq) < 1e-13 and rel(got[b, 1], cu) < 1e-13
    # the midranges the preconditioner blocks are built from
    mid = np.zeros(3)
    L.check(L.lag_medium_midranges(m, mid.ctypes.data_as(L.PD)), ctx)
    (p1, p2) = ce.precond_params(lam, mu, rho, h)
    assert rel(mid[:2], [p1[0], p1[1]]) < 1e-15
    assert rel(mid[2] * h ** 2 / 4.0, p1[2]) < 1e-15
    L.lag_medium_destroy(m)


def test_operator_is_symmetric_through_the_abi(ctx):
    # the energy-derived C is symmetric: (v, C u) = (u, C v) for any two fields (E1)
    nr, nz, hr, hz, h = 37, 29, 4.0, 6.0, 300.0
    vp, vs, rho = _medium_arrays(nr, nz)
    m = _cyl_medium(ctx, vp, vs, rho, hr, hz, h)
    u = RNG.standard_normal((2, 2, nr, nz))
    ud, qd = dev(u), empty(u.shape)
    L.check(L.lag_apply_operator(m, ptr(ud), ptr(qd), 2), ctx)
    q = host(qd)
    a, b = np.vdot(u[1], q[0]), np.vdot(u[0], q[1])
    assert abs(a - b) < 1e-12 * np.linalg.norm(q[0]) * np.linalg.norm(u[1])
    assert np.vdot(u[0], q[0]) > 0 and np.vdot(u[1], q[1]) > 0
    L.lag_medium_destroy(m)


def _block_ref(r, hr, hz, *params):
    """The oracle's B^{-1} (one [nr][nz] field per call) for each right-hand side."""
    return np.stack([ce.apply_inverse_block(x, hr, hz, *params) for x in r])


def _cyl_block(ctx, nr, nz, hr, hz, ax, az, d, hoop, prec=L.LAG_FP64, partitions=0):
    p = C.c_void_p()
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    L.check(L.lag_precond_create_cyl(ctx, C.byref(g), ax, az, d, hoop, prec, partitions, C.byref(p)), ctx)
    return p


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
@pytest.mark.parametrize("nr,nz", [(1, 1), (7, 2), (33, 17), (64, 128), (300, 257)])
def test_preconditioner_blocks(ctx, prec, tol, nr, nz):
    hr, hz, h = 5.0, 4.0, 300.0
    lam = RNG.uniform(2e9, 9e9, (nr, nz))
    mu = RNG.uniform(1e9, 5e9, (nr, nz))
    rho = RNG.uniform(1800, 2600, (nr, nz))
    for params in ce.precond_params(lam, mu, rho, h):     # B1 (hoop term) and B2
        p = _cyl_block(ctx, nr, nz, hr, hz, *params, prec=prec)
        r = RNG.standard_normal((2, nr, nz))
        rd, zd = dev(r), empty(r.shape)
        L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
        assert rel(host(zd), _block_ref(r, hr, hz, *params)) < tol, params
        L.lag_precond_destroy(p)


@pytest.mark.parametrize("P", [1, 4, 32])
def test_hoop_block_every_partition_count(ctx, P):
    # B1's diagonal carries (l+2m)~ / r_i, largest on the axis row: the partitioned solve along r
    nr, nz, hr, hz = 777, 40, 2.5, 2.5
    pt, mt, dt = 9e9, 2e9, 2200.0 * 300.0 ** 2 / 4.0
    p = _cyl_block(ctx, nr, nz, hr, hz, pt, mt, dt, pt, partitions=P)
    r = RNG.standard_normal((3, nr, nz))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 3), ctx)
    assert rel(host(zd), _block_ref(r, hr, hz, pt, mt, dt, pt)) < 1e-12
    L.lag_precond_destroy(p)


def test_homogeneous_block_inverts_the_operator_block(ctx):
    # homogeneous medium: B2 is the U-U block of C exactly, so B2^{-1} (C [0; U])_U = U
    nr, nz, hr, hz, h = 40, 33, 5.0, 4.0, 300.0
    vp, vs, rho = np.full((nr, nz), 3500.0), np.full((nr, nz), 2000.0), np.full((nr, nz), 2300.0)
    m = _cyl_medium(ctx, vp, vs, rho, hr, hz, h)
    lam, mu = elastic_lame(vp, vs, rho)
    _, p2 = ce.precond_params(lam, mu, rho, h)
    p = _cyl_block(ctx, nr, nz, hr, hz, *p2)
    u = np.zeros((1, 2, nr, nz))
    u[0, 1] = RNG.standard_normal((nr, nz))
    ud, qd, zd = dev(u), empty(u.shape), empty((1, nr, nz))
    L.check(L.lag_apply_operator(m, ptr(ud), ptr(qd), 1), ctx)
    L.check(L.lag_precond_apply(p, ptr(qd[0, 1]), ptr(zd), 1), ctx)
    assert rel(host(zd)[0], u[0, 1]) < 1e-11
    L.lag_precond_destroy(p)
    L.lag_medium_destroy(m)


def _model(nr, nz, hx, n_harm, f0=12.0):
    s = inputs.cylindrical(nr=nr, nz=nz, h=hx, n_harm=n_harm, layered=True, f0=f0)
    s.vs = s.c / 1.73
    s.vs[:, : nz // 3] = s.c[:, : nz // 3] / 2.0     # a slower top: Poisson ratio varies with depth
    s.h, s.alpha = 300.0, 8
    s.t0 = 1.2 / f0
    s.t_out = np.linspace(0.005, 0.5, 120)
    return s


def _shot(ctx, s, prec, tol, restart=20):
    g = L.grid(s.nx, s.nz, s.hx, s.hz, cylindrical=True)
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=tol, prec=prec, restart_k=restart)
    w = L.wavelet(s.f0, s.t0)
    p_, pp = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    traces = np.zeros((1, 2, len(s.receivers), s.t_out.size))
    its = np.zeros((1, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    rc = L.lag_solve_elastic(ctx, C.byref(g), pp, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                             L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                             traces.ctypes.data_as(L.PD), C.byref(st))
    return rc, traces[0], its[0]


@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_cylindrical_elastic_shot_matches_oracle(ctx, prec, tol, gate):
    # a vertical force on the axis three rows deep, receivers along the surface row and one
    # column; random layers along z
    s = _model(96, 72, 10.0, 8)
    s.sources = [(0, 3)]
    s.receivers = [(i, 0) for i in range(0, 96, 8)] + [(5, k) for k in range(2, 72, 9)]
    rc, tr, its = _shot(ctx, s, prec, tol)
    L.check(rc, ctx)
    ref = ce.elastic_shot(s.c, s.vs, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                          s.t_out, s.f0, s.t0, tol=tol, restart=20)
    assert rel_l2(tr, ref["traces"]) < gate
    for comp in range(2):                     # both components carry signal
        assert np.abs(tr[comp]).max() > 1e-3 * np.abs(tr).max()
    if prec == L.LAG_FP64:
        assert np.abs(its - ref["iters"]).max() <= 1
    assert np.all(its > 1)


def test_cylindrical_elastic_ragged_grid(ctx):
    # odd sizes on both axes (a ragged last tile of the stencil and of the DCT), a source off row 0
    s = _model(37, 29, 12.5, 5)
    s.sources = [(0, 11)]
    s.receivers = [(0, 0), (36, 28), (18, 11), (3, 20)]
    rc, tr, _ = _shot(ctx, s, L.LAG_FP64, 1e-13)
    L.check(rc, ctx)
    ref = ce.elastic_shot(s.c, s.vs, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers,
                          s.t_out, s.f0, s.t0, tol=1e-13, restart=20)
    assert rel_l2(tr, ref["traces"]) < 1e-10


def test_cylindrical_elastic_rejections(ctx):
    s = _model(16, 12, 10.0, 2)
    g = L.grid(16, 12, 5.0, 5.0)                        # Cartesian: no hoop term, no B1 with 1/r
    p = C.c_void_p()
    assert L.lag_precond_create_cyl(ctx, C.byref(g), 1e9, 1e9, 1e6, 1e9, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL
    g = L.grid(16, 12, 5.0, 5.0, cylindrical=True)
    assert L.lag_precond_create_cyl(ctx, C.byref(g), 1e9, 1e9, 1e6, 0.0, L.LAG_FP64, 33,
                                    C.byref(p)) == L.LAG_EINVAL
    sv = L.solver(tol=1e-8, layered=1)                  # the layered preconditioner is acoustic, Cartesian
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    w = L.wavelet(s.f0, s.t0)
    p_, pp = L.f64(s.c)
    v_, pv = L.f64(s.vs)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    tr = np.zeros((2, 1, s.t_out.size))
    rc = L.lag_solve_elastic(ctx, C.byref(g), pp, pv, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                             L.points([(0, 0)]), 1, L.points([(1, 1)]), s.t_out.size, pt,
                             tr.ctypes.data_as(L.PD), None)
    assert rc == L.LAG_EINVAL
