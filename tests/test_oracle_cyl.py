"""Pins of the cylindrical (2.5D axisymmetric) oracle against what the paper and the mathematics
fix: the DCT-II diagonalises the zero-flux second difference, the r-weighted operator is SPD and
approximates the 3D Laplacian of an axisymmetric field at second order (axis included), the
preconditioner inverts the operator of a homogeneous medium, and a whole shot converges at second
order to the exact 3D point-source solution with its free-surface image (Sec. 3.2)."""
import numpy as np
import pytest

from oracle import analytic, cyl, krylov, laguerre

RNG = np.random.default_rng(1005)


def neumann_second_difference(n, h):
    """Zero-flux second difference written from its faces: interior (1, -2, 1)/h^2, the end
    rows lose their outer face."""
    D = np.zeros((n, n))
    for k in range(n):
        if k > 0:
            D[k, k - 1] += 1.0 / h ** 2
            D[k, k] -= 1.0 / h ** 2
        if k < n - 1:
            D[k, k + 1] += 1.0 / h ** 2
            D[k, k] -= 1.0 / h ** 2
    return D


@pytest.mark.parametrize("n", [1, 2, 7, 16, 33])
def test_dct_diagonalises_zero_flux_second_difference(n):
    V = cyl.dct_matrix(n)
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    D = neumann_second_difference(n, 3.0)
    assert np.abs(V.T @ D @ V + np.diag(cyl.neumann_eigenvalues(n, 3.0))).max() < 1e-13 / 9.0 * 4


def test_operator_symmetric_positive_definite():
    nr, nz, hr, hz, h = 6, 5, 4.0, 3.0, 200.0
    kappa = RNG.uniform(1e9, 9e9, (nr, nz))
    rho = RNG.uniform(1000, 2600, (nr, nz))
    a1, a2, w = cyl.coefficients(kappa, rho, hr, hz, h)
    M = cyl.assemble_A(a1, a2, w, hr, hz)
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0
    # the axis face carries no flux, the ghost face beyond the last radius does
    assert np.all(a1[0] == 0) and np.all(a1[nr] > 0)
    assert np.all(a2[:, 0] == 0) and np.all(a2[:, nz] == 0)


def _laplacian_error(hr):
    # homogeneous kappa = 1, no mass: (A u) / r must approach -Lap_3D u of the axisymmetric
    # Gaussian u = exp(-(r^2 + (z - zc)^2) / s^2), whose Laplacian is (4 R^2/s^4 - 6/s^2) u
    L, s = 8.0, 1.0
    nr = int(round(L / hr))
    nz = 2 * nr
    r, z = cyl.mesh(nr, nz, hr, hr)
    R2 = r[:, None] ** 2 + (z[None, :] - L) ** 2
    u = np.exp(-R2 / s ** 2)
    a1, a2, w = cyl.coefficients(np.ones((nr, nz)), np.zeros((nr, nz)), hr, hr, 0.0)
    Au = cyl.apply_A(u, a1, a2, w, hr, hr) / r[:, None]
    exact = -(4.0 * R2 / s ** 4 - 6.0 / s ** 2) * u
    return np.abs(Au - exact).max() / np.abs(exact).max(), np.abs(Au[0] - exact[0]).max() / np.abs(exact).max()


def test_operator_is_the_cylindrical_laplacian_at_second_order():
    e1, a1 = _laplacian_error(0.2)
    e2, a2 = _laplacian_error(0.1)
    assert e2 < 2e-2
    assert 3.5 < e1 / e2 < 4.5
    assert 3.5 < a1 / a2 < 4.5               # on the axis row too


@pytest.mark.parametrize("nr,nz", [(1, 1), (5, 4), (23, 17)])
def test_preconditioner_inverts_the_homogeneous_operator(nr, nz):
    hr, hz, h = 5.0, 4.0, 300.0
    kappa = RNG.uniform(1e9, 9e9, (nr, nz))
    rho = RNG.uniform(1000, 2600, (nr, nz))
    kt, dt = cyl.precond_params(kappa, rho, h)
    rhot = dt * 4.0 / h ** 2
    a1, a2, w = cyl.coefficients(np.full((nr, nz), kt), np.full((nr, nz), rhot), hr, hz, h)
    y = RNG.standard_normal((2, nr, nz))
    By = cyl.apply_A(y, a1, a2, w, hr, hz)
    assert np.abs(cyl.apply_inverse(By, hr, hz, kt, dt) - y).max() < 1e-11
    M = cyl.assemble_A(a1, a2, w, hr, hz)
    b = RNG.standard_normal((nr, nz))
    ref = np.linalg.solve(M, b.ravel()).reshape(nr, nz)
    assert np.abs(cyl.apply_inverse(b, hr, hz, kt, dt) - ref).max() < 1e-12 * np.abs(ref).max()


def test_preconditioned_cg_converges_on_a_layered_medium():
    nr, nz, hr, h = 40, 48, 10.0, 200.0
    layers = (np.arange(nz) * 6) // nz
    c = RNG.uniform(1500, 4500, 6)[layers][None, :] * (1 + 0.02 * RNG.standard_normal((nr, nz)))
    rho = 310 * c ** 0.25
    kappa = rho * c ** 2
    a1, a2, w = cyl.coefficients(kappa, rho, hr, hr, h)
    kt, dt = cyl.precond_params(kappa, rho, h)
    b = RNG.standard_normal(nr * nz)
    x, it, _ = krylov.pcg(lambda v: cyl.apply_A(v.reshape(nr, nz), a1, a2, w, hr, hr).ravel(),
                          lambda v: cyl.apply_inverse(v.reshape(nr, nz), hr, hr, kt, dt).ravel(), b, 1e-10)
    M = cyl.assemble_A(a1, a2, w, hr, hr)
    assert np.linalg.norm(M @ x - b) / np.linalg.norm(b) < 1e-9
    assert 3 < it < 200


def _point_source_error(hx):
    # homogeneous half space with a free surface, the source on the axis 400 m deep, a receiver
    # 300 m away at the source depth; exact: direct wave + its mirror image above the surface.
    # The window ends before the bottom face or the outer radius send anything back.
    f0, h, alpha, c0, rho0 = 10.0, 400.0, 9, 2000.0, 1000.0
    t0 = 2.5 / f0
    t = np.linspace(0.01, 0.75, 100)
    n = int(round(1200.0 / hx))
    ks = int(round(400.0 / hx - 0.5))
    zs = (ks + 0.5) * hx
    off = int(round(300.0 / hx - 0.5))
    rr = (off + 0.5) * hx
    out = cyl.acoustic_shot(np.full((n, n), c0), np.full((n, n), rho0), hx, hx, h, alpha, 160,
                            (0, ks), [(off, ks)], t, f0, t0, tol=1e-12)
    f = laguerre.ricker(f0, t0)
    kap = rho0 * c0 ** 2
    ua = analytic.point_source_3d(rr, t, kap, rho0, f) + analytic.point_source_3d(np.hypot(rr, 2 * zs), t, kap, rho0, f)
    eps = np.sqrt(np.sum((out["traces"][0] - ua) ** 2) / np.sum(ua ** 2))   # Sec. 3.2 accuracy
    return eps, out["iters"]


def test_shot_matches_3d_point_source_with_image_at_second_order():
    # measured: 0.412 (20 m), 0.107 (10 m), 0.026 (5 m)
    e10, it10 = _point_source_error(10.0)
    e5, it5 = _point_source_error(5.0)
    assert np.all(it10 == 1) and np.all(it5 == 1)       # homogeneous: A == B
    assert e5 < 0.04
    assert 3.3 < e10 / e5 < 5.0                           # O(h^2)


def test_radial_preconditioner_is_A_for_an_r_only_medium():
    # kappa, rho depending on r only: the radial B equals A (PCG takes one iteration); constant
    # radii give the whole-medium B
    nr, nz, hr, hz, h = 11, 9, 5.0, 4.0, 400.0
    kappa = np.repeat(RNG.uniform(2e9, 9e9, nr)[:, None], nz, axis=1)
    rho = np.repeat(RNG.uniform(1000, 2600, nr)[:, None], nz, axis=1)
    a1, a2, w = cyl.coefficients(kappa, rho, hr, hz, h)
    kr, dr = cyl.precond_params_radial(kappa, rho, h)
    y = RNG.standard_normal((nr, nz))
    assert np.abs(cyl.apply_inverse_radial(cyl.apply_A(y, a1, a2, w, hr, hz), hr, hz, kr, dr) - y).max() < 1e-11
    kt, dt = 4e9, 3e7
    r = RNG.standard_normal((2, nr, nz))
    a = cyl.apply_inverse_radial(r, hr, hz, np.full(nr, kt), np.full(nr, dt))
    b = cyl.apply_inverse(r, hr, hz, kt, dt)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


def test_radial_preconditioner_keeps_the_r_and_z_coefficients_apart():
    # separate per-radius coefficients for the r faces (a1 = rbar ax~, mean of the two radii at a
    # face, the outer face its radius's value) and for the z direction (a2 = r az~, zero-flux
    # surface and bottom): with nothing depending on z the DCT-II along z separates exactly, so
    # B^{-1} inverts the operator assembled from those faces; swapping ax~ and az~ does not
    nr, nz, hr, hz = 13, 10, 5.0, 4.0
    ax = RNG.uniform(2e9, 9e9, nr)
    az = RNG.uniform(2e9, 9e9, nr)
    dd = RNG.uniform(1e6, 5e7, nr)
    r, _ = cyl.mesh(nr, nz, hr, hz)
    rbar = np.arange(nr + 1) * hr
    af = np.concatenate([[0.0], 0.5 * (ax[:-1] + ax[1:]), [ax[-1]]])
    a1 = np.repeat((rbar * af)[:, None], nz, axis=1)
    a2 = np.zeros((nr, nz + 1))
    a2[:, 1:nz] = (r * az)[:, None]
    w = np.repeat((r * dd)[:, None], nz, axis=1)
    y = RNG.standard_normal((2, nr, nz))
    Ay = cyl.apply_A(y, a1, a2, w, hr, hz)
    assert np.abs(cyl.apply_inverse_radial(Ay, hr, hz, ax, dd, kz=az) - y).max() < 1e-11
    assert np.abs(cyl.apply_inverse_radial(Ay, hr, hz, az, dd, kz=ax) - y).max() > 1e-3
