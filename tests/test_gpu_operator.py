"""Parity of the stencil operators (acoustic A, elastic C) with the oracle, through the C ABI."""
import ctypes as C

import numpy as np
import pytest

from oracle import fd
from oracle import solve as osolve
from paper_1005_0542_gb300 import lagwave as L

from gpu_util import make_ctx, dev, empty, host, medium, ptr, rel

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(91)


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lag_destroy(c)


@pytest.mark.parametrize("nz,nx", [(1, 1), (2, 3), (23, 37), (128, 128), (70, 257)])
def test_acoustic_operator(ctx, nz, nx):
    c = RNG.uniform(1500, 4500, (nz, nx))
    rho = RNG.uniform(1000, 2600, (nz, nx))
    h, dx, dz = 200.0, 5.0, 7.5
    m = medium(ctx, nx, nz, dx, dz, c, rho, h)
    p = RNG.standard_normal((3, nz, nx))
    pd, qd = dev(p), empty(p.shape)
    L.check(L.lag_apply_operator(m, ptr(pd), ptr(qd), 3), ctx)
    ref = fd.apply_A(p, fd.kappa_from_velocity(c, rho), rho, h, dx, dz)
    assert rel(host(qd), ref) < 1e-14
    mid = (C.c_double * 3)()
    L.check(L.lag_medium_midranges(m, mid))
    kap = fd.kappa_from_velocity(c, rho)
    assert mid[0] == pytest.approx(0.5 * (kap.min() + kap.max()), rel=1e-15)
    assert mid[1] == pytest.approx(0.5 * (rho.min() + rho.max()), rel=1e-15)
    L.lag_medium_destroy(m)


@pytest.mark.parametrize("nz,nx", [(1, 1), (3, 2), (19, 26), (64, 96)])
def test_elastic_operator(ctx, nz, nx):
    vp = RNG.uniform(2000, 5000, (nz, nx))
    vs = vp / 1.73
    rho = RNG.uniform(1800, 2600, (nz, nx))
    h, dx, dz = 300.0, 2.5, 3.0
    m = medium(ctx, nx, nz, dx, dz, vp, rho, h, vs=vs)
    u = RNG.standard_normal((2, 2, nz, nx))   # [rhs][comp][z][x]
    ud, qd = dev(u), empty(u.shape)
    L.check(L.lag_apply_operator(m, ptr(ud), ptr(qd), 2), ctx)
    lam, mu = osolve.elastic_lame(vp, vs, rho)
    got = host(qd)
    for b in range(2):
        cu, cw = fd.apply_C(u[b, 0], u[b, 1], lam, mu, rho, h, dx, dz)
        assert rel(got[b, 0], cu) < 1e-14 and rel(got[b, 1], cw) < 1e-14
    L.lag_medium_destroy(m)
