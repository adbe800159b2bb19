"""The paper's 2.5D axisymmetric acoustic problem (Sec. 2.1, the r-weighted scheme of Sec. 2.3,
the cylindrical preconditioner of Eq. 21): the DCT-II along z and its inverse, the general
tridiagonal systems along r, the whole preconditioner on both paths, the operator, and shots,
each against the oracle (oracle.cyl).  Fields are [nr][nz], depth fastest."""
import ctypes as C

import numpy as np
import pytest

from oracle import cyl
from oracle.fd import kappa_from_velocity
from paper_1005_0542_gb300 import inputs
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, plan_info, ptr, rel, rel_l2

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2503)
SHAPES = [(1, 1), (7, 2), (33, 17), (64, 128), (300, 257)]


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


def cyl_plan(ctx, nr, nz, hr, hz, kt, dt, prec=L.LAG_FP64, partitions=0):
    p = C.c_void_p()
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    L.check(L.lag_precond_create_sep(ctx, C.byref(g), kt, kt, dt, prec, partitions, C.byref(p)), ctx)
    return p


def cyl_medium(ctx, c, rho, hr, hz, h):
    m = C.c_void_p()
    nr, nz = c.shape
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    c_, pc = L.f64(c)
    r_, pr = L.f64(rho)
    L.check(L.lag_medium_create_acoustic(ctx, C.byref(g), pc, pr, h, C.byref(m)), ctx)
    return m


@pytest.mark.parametrize("nr,nz", SHAPES)
def test_dct_forward_and_inverse(ctx, nr, nz):
    p = cyl_plan(ctx, nr, nz, 5.0, 4.0, 3e9, 1e7)
    V = cyl.dct_matrix(nz)
    x = RNG.standard_normal((2, nr, nz))
    xd, yd, zd = dev(x), empty(x.shape), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), 2), ctx)
    assert rel(host(yd), x @ V) < 1e-13
    L.check(L.lag_precond_dst_inverse(p, ptr(yd), ptr(zd), 2), ctx)
    assert rel(host(zd), x) < 1e-13
    L.check(L.lag_precond_dst_inverse(p, ptr(xd), ptr(zd), 2), ctx)
    assert rel(host(zd), x @ V.T) < 1e-13
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("P", [1, 2, 4, 8, 32])
@pytest.mark.parametrize("nr,nz", [(4, 3), (100, 64), (1024, 40), (777, 130)])
def test_tridiag_along_r_every_partition_count(ctx, P, nr, nz):
    hr, hz, kt, dt = 5.0, 3.0, 4e9, 2e7
    p = cyl_plan(ctx, nr, nz, hr, hz, kt, dt, partitions=P)
    y = RNG.standard_normal((3, nr, nz))                   # a spectrum: [r][z-mode]
    V = cyl.dct_matrix(nz)
    ref = cyl.apply_inverse(y @ V.T, hr, hz, kt, dt) @ V    # T_q^{-1} along r for every mode q
    dd, yd = dev(y), empty(y.shape)
    L.check(L.lag_precond_tridiag(p, ptr(dd), ptr(yd), 3), ctx)
    assert rel(host(yd), ref) < 1e-12
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
@pytest.mark.parametrize("nr,nz", SHAPES)
def test_precond_apply_cylindrical(ctx, prec, tol, nr, nz):
    hr, hz, h = 5.0, 4.0, 400.0
    kappa = RNG.uniform(2e9, 9e9, (nr, nz))
    rho = RNG.uniform(1000, 2600, (nr, nz))
    kt, dt = cyl.precond_params(kappa, rho, h)
    p = C.c_void_p()
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    L.check(L.lag_precond_create(ctx, C.byref(g), kt, dt * 4.0 / h ** 2, h, prec, C.byref(p)), ctx)
    # tensor cores from 16 depth nodes on (float64: exact slices; mixed: split bf16)
    assert L.lag_precond_uses_tensor_cores(p) == (1 if nz >= 16 else 0)
    r = RNG.standard_normal((2, nr, nz))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    assert rel(host(zd), cyl.apply_inverse(r, hr, hz, kt, dt)) < tol
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 3), (23, 37), (70, 257)])
def test_operator_cylindrical(ctx, nr, nz):
    hr, hz, h = 5.0, 7.5, 400.0
    c = RNG.uniform(1500, 4500, (nr, nz))
    rho = RNG.uniform(1000, 2600, (nr, nz))
    m = cyl_medium(ctx, c, rho, hr, hz, h)
    p = RNG.standard_normal((2, nr, nz))
    pd, qd = dev(p), empty(p.shape)
    L.check(L.lag_apply_operator(m, ptr(pd), ptr(qd), 2), ctx)
    a1, a2, w = cyl.coefficients(kappa_from_velocity(c, rho), rho, hr, hz, h)
    assert rel(host(qd), cyl.apply_A(p, a1, a2, w, hr, hz)) < 1e-14
    L.lag_medium_destroy(m)


def test_static_apply_equals_plan_apply(ctx):
    # the no-allocation entry point runs the SIMT DCT; the plan the exact-slice tensor-core one
    nr, nz, hr, hz, kt, dt = 96, 80, 5.0, 5.0, 3e9, 1e7
    p = cyl_plan(ctx, nr, nz, hr, hz, kt, dt)
    r = RNG.standard_normal((2, nr, nz))
    rd, z1, z2 = dev(r), empty(r.shape), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(z1), 2), ctx)
    L.check(L.lag_precond_apply_static(p, ptr(rd), ptr(z2), 2), ctx)
    ref = cyl.apply_inverse(r, hr, hz, kt, dt)
    assert rel(host(z1), ref) < 1e-12 and rel(host(z2), ref) < 1e-12
    assert rel(host(z1), host(z2)) < 1e-13
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("nr,nz", [(40, 2048), (3, 4097)])
def test_dct_exact_slices_large(ctx, nr, nz):
    # long rows: several K stages and N tiles of the exact-slice GEMM, odd length with a middle mode
    p = cyl_plan(ctx, nr, nz, 5.0, 4.0, 3e9, 1e7)
    assert L.lag_precond_uses_tensor_cores(p) == (1 if nz <= 8448 else 0)
    V = cyl.dct_matrix(nz)
    x = RNG.standard_normal((1, nr, nz)) * np.logspace(-100, 100, nr)[None, :, None]
    xd, yd, zd = dev(x), empty(x.shape), empty(x.shape)
    L.check(L.lag_precond_dst(p, ptr(xd), ptr(yd), 1), ctx)
    y = host(yd)
    ref = x @ V
    for i in range(nr):  # row by row: every row keeps its own scale
        assert rel(y[0, i], ref[0, i]) < 1e-13
    L.check(L.lag_precond_dst_inverse(p, ptr(yd), ptr(zd), 1), ctx)
    z = host(zd)
    for i in range(nr):
        assert rel(z[0, i], x[0, i]) < 1e-13
    L.lag_precond_destroy(p)


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
def test_cylindrical_layouts_and_autotune(ctx, prec, tol):
    nr, nz, hr, hz, kt, dt = 512, 384, 5.0, 5.0, 3e9, 2e7
    p = cyl_plan(ctx, nr, nz, hr, hz, kt, dt, prec=prec)
    r = RNG.standard_normal((4, nr, nz))
    ref = cyl.apply_inverse(r, hr, hz, kt, dt)
    rd, zd = dev(r), empty(r.shape)
    tiles = (4, 8) if prec == L.LAG_FP64 else (8, 16, 32)
    for P, mts in ((8, (0,)), (16, tiles), (32, tiles)):
        for mt in mts:
            L.check(L.lag_precond_set_layout(p, P, mt), ctx)
            assert plan_info(p)[0] == P
            L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 4), ctx)
            assert rel(host(zd), ref) < tol, (P, mt)
    Pt, mtt, prod, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    L.check(L.lag_precond_autotune(p, 4, C.byref(Pt), C.byref(mtt), C.byref(prod), C.byref(ms)), ctx)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 4), ctx)
    # the tuner may drop bf16 products of the mixed transform (a coarser preconditioner)
    assert rel(host(zd), ref) < (tol if prec == L.LAG_FP64 or prod.value == 3 else 2e-2)
    L.lag_precond_destroy(p)


def _shot(ctx, s, prec, tol, layered=0, free_surface=True):
    g = L.grid(s.nx, s.nz, s.hx, s.hz, free_surface=free_surface)
    g.cylindrical = 1
    lag = L.laguerre(s.h, s.alpha, s.n_harm)
    sv = L.solver(tol=tol, prec=prec, layered=layered)
    w = L.wavelet(s.f0, s.t0, 4.0, L.LAG_WAVELET_PAPER)
    c_, pc = L.f64(s.c)
    r_, pr = L.f64(s.rho)
    t_, pt = L.f64(s.t_out)
    traces = np.zeros((1, 1, len(s.receivers), s.t_out.size))
    its = np.zeros((1, s.n_harm), dtype=np.int32)
    st = L.lag_stats(its.ctypes.data_as(L.PI), None, 0, 0.0)
    rc = L.lag_solve_acoustic(ctx, C.byref(g), pc, pr, C.byref(lag), C.byref(sv), C.byref(w), 1,
                              L.points(s.sources), len(s.receivers), L.points(s.receivers), s.t_out.size, pt,
                              traces.ctypes.data_as(L.PD), C.byref(st))
    return rc, traces[0, 0], its[0]


def _oracle_shot(s, tol):
    return cyl.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers, s.t_out,
                             s.f0, s.t0, tol=tol, wavelet="paper")


@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_cylindrical_shot_matches_oracle(ctx, prec, tol, gate):
    s = inputs.cylindrical(nr=96, nz=64, h=10.0, n_harm=10, layered=True)
    s.sources = [(0, 3)]
    s.receivers = [(i, 3) for i in range(0, 96, 8)]
    rc, tr, its = _shot(ctx, s, prec, tol)
    L.check(rc, ctx)
    ref = _oracle_shot(s, tol)
    assert rel_l2(tr, ref["traces"]) < gate
    if prec == L.LAG_FP64:
        assert np.abs(its - ref["iters"]).max() <= 1
    assert np.all(its > 2)


def test_cylindrical_homogeneous_one_iteration(ctx):
    # homogeneous medium: the cylindrical preconditioner is the operator itself
    s = inputs.cylindrical(nr=128, nz=96, h=10.0, n_harm=8)
    rc, tr, its = _shot(ctx, s, L.LAG_FP64, 1e-10)
    L.check(rc, ctx)
    assert np.all(its == 1), its
    ref = _oracle_shot(s, 1e-12)
    assert rel_l2(tr, ref["traces"]) < 1e-9


def test_cylindrical_rejections(ctx):
    s = inputs.cylindrical(nr=16, nz=12, h=10.0, n_harm=2)
    rc, _, _ = _shot(ctx, s, L.LAG_FP64, 1e-8, free_surface=False)      # the half space has a surface
    assert rc == L.LAG_EINVAL
    g = L.grid(16, 12, 5.0, 5.0, cylindrical=True)
    p = C.c_void_p()
    a_, pa = L.f64(np.ones(16))
    z_, pz = L.f64(np.zeros(16))
    # radial rows must be positive (d >= 0)
    assert L.lag_precond_create_layered(ctx, C.byref(g), pz, pa, pa, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL
    assert L.lag_precond_create_layered(ctx, C.byref(g), pa, pz, pa, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL


@pytest.mark.parametrize("prec,tol", [(L.LAG_FP64, 1e-12), (L.LAG_MIXED, 2e-4)])
@pytest.mark.parametrize("nr,nz", [(1, 1), (7, 2), (33, 17), (300, 257)])
def test_radial_precond_apply(ctx, prec, tol, nr, nz):
    # per-radius coefficients (the radial variant of the layered plan): against the oracle
    hr, hz, h = 5.0, 4.0, 400.0
    kappa = RNG.uniform(2e9, 9e9, (nr, nz))
    rho = RNG.uniform(1000, 2600, (nr, nz))
    kr, dr = cyl.precond_params_radial(kappa, rho, h)
    kz = kr * RNG.uniform(0.5, 2.0, nr)   # a z coefficient apart from the r-face one
    g = L.grid(nr, nz, hr, hz, cylindrical=True)
    p = C.c_void_p()
    k_, pk = L.f64(kr)
    kz_, pkz = L.f64(kz)
    d_, pd = L.f64(dr)
    L.check(L.lag_precond_create_layered(ctx, C.byref(g), pk, pkz, pd, prec, 0, C.byref(p)), ctx)
    assert L.lag_precond_is_layered(p) == 1
    r = RNG.standard_normal((2, nr, nz))
    rd, zd = dev(r), empty(r.shape)
    L.check(L.lag_precond_apply(p, ptr(rd), ptr(zd), 2), ctx)
    assert rel(host(zd), cyl.apply_inverse_radial(r, hr, hz, kr, dr, kz=kz)) < tol
    L.lag_precond_destroy(p)


def test_whole_medium_cylindrical_plans_are_not_layered(ctx):
    # only lag_precond_create_layered plans report themselves as layered
    g = L.grid(24, 16, 5.0, 4.0, cylindrical=True)
    p = C.c_void_p()
    L.check(L.lag_precond_create(ctx, C.byref(g), 4e9, 1500.0, 400.0, L.LAG_FP64, C.byref(p)), ctx)
    assert L.lag_precond_is_layered(p) == 0
    L.lag_precond_destroy(p)
    L.check(L.lag_precond_create_cyl(ctx, C.byref(g), 9e9, 3e9, 1500.0 * 400.0 ** 2 / 4, 9e9, L.LAG_FP64, 0,
                                     C.byref(p)), ctx)
    assert L.lag_precond_is_layered(p) == 0
    L.lag_precond_destroy(p)
    gc = L.grid(24, 16, 5.0, 4.0)
    L.check(L.lag_precond_create(ctx, C.byref(gc), 4e9, 1500.0, 400.0, L.LAG_FP64, C.byref(p)), ctx)
    assert L.lag_precond_is_layered(p) == 0
    L.lag_precond_destroy(p)
    # a non-finite per-radius coefficient is rejected like the Cartesian layered rows
    a_, pa = L.f64(np.full(24, 4e9))
    i_ = np.full(24, 4e9)
    i_[5] = np.inf
    ib_, pi = L.f64(i_)
    assert L.lag_precond_create_layered(ctx, C.byref(g), pi, pa, pa, L.LAG_FP64, 0, C.byref(p)) == L.LAG_EINVAL


def _radial_model(nr, nz, h, n_harm, noise):
    # velocity layered along r (the radial preconditioner's case) with optional lateral noise
    s = inputs.cylindrical(nr=nr, nz=nz, h=h, n_harm=n_harm, layered=True)
    rng = np.random.default_rng(77)
    layers = (np.arange(nr) * 8) // nr
    cr = rng.uniform(1500, 4500, 8)[layers]
    s.c = np.repeat(cr[:, None], nz, axis=1) * (1 + noise * rng.standard_normal((nr, nz)))
    s.rho = 310.0 * s.c ** 0.25
    return s


@pytest.mark.parametrize("prec,tol,gate", [(L.LAG_FP64, 1e-13, 1e-10), (L.LAG_MIXED, 1e-11, 1e-8)])
def test_radial_shot_matches_oracle(ctx, prec, tol, gate):
    s = _radial_model(96, 64, 10.0, 8, 0.02)
    s.sources = [(0, 3)]
    s.receivers = [(i, 3) for i in range(0, 96, 8)]
    rc, tr, its = _shot(ctx, s, prec, tol, layered=1)
    L.check(rc, ctx)
    ref = cyl.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers, s.t_out,
                            s.f0, s.t0, tol=tol, wavelet="paper", radial=True)
    assert rel_l2(tr, ref["traces"]) < gate
    if prec == L.LAG_FP64:
        assert np.abs(its - ref["iters"]).max() <= 1
        _, _, its_c = _shot(ctx, s, prec, tol)
        assert its.sum() < its_c.sum(), (its, its_c)


def test_radial_shot_r_only_medium_one_iteration(ctx):
    s = _radial_model(80, 48, 10.0, 6, 0.0)
    rc, tr, its = _shot(ctx, s, L.LAG_FP64, 1e-10, layered=1)
    L.check(rc, ctx)
    assert np.all(its == 1), its
