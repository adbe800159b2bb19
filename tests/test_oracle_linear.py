"""Pins of the oracle's linear-algebra pieces against mathematics and library routines.

Each test fixes a property the paper or the mathematics guarantees, chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at least one."""
import numpy as np
import pytest
import scipy.fft

from oracle import dst, fd, krylov, precond
from oracle.tridiag import thomas

RNG = np.random.default_rng(20240601)


# ---------------------------------------------------------------------------------- DST-I
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 31, 64, 127])
def test_dst_involution_and_scipy(n):
    S = dst.dst_matrix(n)
    assert np.allclose(S, S.T, atol=0, rtol=0) or np.abs(S - S.T).max() < 1e-15
    assert np.abs(S @ S - np.eye(n)).max() < 1e-13           # orthonormal DST-I: S^2 = I
    x = RNG.standard_normal((3, n))
    ref = scipy.fft.dst(x, type=1, norm="ortho", axis=-1)     # library DST-I
    assert np.abs(dst.dst_x(x, S) - ref).max() < 1e-13


@pytest.mark.parametrize("n,hx", [(7, 1.0), (32, 0.25), (100, 5.0)])
def test_dst_diagonalises_dirichlet_second_difference(n, hx):
    T = (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / hx ** 2
    S = dst.dst_matrix(n)
    lam = dst.laplace_eigenvalues(n, hx)
    assert np.abs(T @ S - S * lam).max() / lam.max() < 1e-13


def test_dst_large_angle_reduction():
    # entries for large n must still be a sine of the exact angle (reduced modulo 2(n+1))
    n = 2048
    S = dst.dst_matrix(n)
    j, k = 2047, 2047
    ang = np.pi * ((j + 1) * (k + 1) % (2 * (n + 1))) / (n + 1)
    assert S[j, k] == pytest.approx(np.sqrt(2.0 / (n + 1)) * np.sin(ang), abs=1e-16)
    assert np.abs(S[:, :8].T @ S[:, :8] - np.eye(8)).max() < 1e-13


# --------------------------------------------------------------------------------- Thomas
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_thomas_matches_dense_solve(n):
    sub = RNG.uniform(-1, 1, n)
    sup = RNG.uniform(-1, 1, n)
    diag = np.abs(sub) + np.abs(sup) + RNG.uniform(0.5, 2.0, n)
    d = RNG.standard_normal((n, 4))
    M = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    y = thomas(sub[:, None], diag[:, None], sup[:, None], d)
    assert np.abs(y - np.linalg.solve(M, d)).max() < 1e-12


# ----------------------------------------------------------------------- acoustic operator
def _medium(nz, nx):
    c = RNG.uniform(1500, 4500, (nz, nx))
    rho = RNG.uniform(1000, 2600, (nz, nx))
    return fd.kappa_from_velocity(c, rho), rho


def test_apply_A_matches_entrywise_assembly_and_is_spd():
    nz, nx, hx, hz, h = 5, 7, 10.0, 7.0, 200.0
    kappa, rho = _medium(nz, nx)
    M = fd.assemble_A(kappa, rho, h, hx, hz)
    cols = np.stack([fd.apply_A(e.reshape(nz, nx), kappa, rho, h, hx, hz).ravel()
                     for e in np.eye(nz * nx)], axis=1)
    assert np.abs(cols - M).max() / np.abs(M).max() < 1e-14
    assert np.abs(M - M.T).max() / np.abs(M).max() < 1e-15          # A = A* (Sec. 2.3)
    assert np.linalg.eigvalsh(M).min() > 0                           # A > 0


def test_apply_A_homogeneous_eigenfunction():
    # homogeneous medium: A sin(p) sin(q) = (kappa (lam_p + mu_q) + rho h^2/4) sin(p) sin(q)
    nz, nx, hx, hz, h = 9, 12, 3.0, 4.0, 50.0
    kappa, rho = 7.0, 2.0
    Sx, Sz = dst.dst_matrix(nx), dst.dst_matrix(nz)
    p, q = 4, 6
    v = np.outer(Sz[:, q], Sx[:, p])
    Av = fd.apply_A(v, np.full((nz, nx), kappa), np.full((nz, nx), rho), h, hx, hz)
    ev = kappa * (dst.laplace_eigenvalues(nx, hx)[p] + dst.laplace_eigenvalues(nz, hz)[q]) + rho * h * h / 4
    assert np.abs(Av - ev * v).max() < 1e-12 * ev


def _manufactured_error(n):
    # -div(kappa grad u) + w u with kappa = 1 + 0.5 sin x cos z, u = sin x sin 2z on [0, pi]^2
    L = np.pi
    hh = L / (n + 1)
    xs = hh * np.arange(1, n + 1)
    X, Z = np.meshgrid(xs, xs)          # [z, x]
    kap = 1 + 0.5 * np.sin(X) * np.cos(Z)
    kx, kz = 0.5 * np.cos(X) * np.cos(Z), -0.5 * np.sin(X) * np.sin(Z)
    u = np.sin(X) * np.sin(2 * Z)
    ux, uxx = np.cos(X) * np.sin(2 * Z), -np.sin(X) * np.sin(2 * Z)
    uz, uzz = 2 * np.sin(X) * np.cos(2 * Z), -4 * np.sin(X) * np.sin(2 * Z)
    rho, h = 3.0, 2.0
    exact = -(kx * ux + kap * uxx + kz * uz + kap * uzz) + rho * h * h / 4 * u
    got = fd.apply_A(u, kap, np.full_like(u, rho), h, hh, hh)
    return np.abs(got - exact)[2:-2, 2:-2].max()      # interior nodes (boundary faces: reading A-2)


def test_apply_A_second_order_truncation():
    e1, e2 = _manufactured_error(40), _manufactured_error(81)
    assert 3.5 < e1 / e2 < 4.5


# ------------------------------------------------------------------------- preconditioner
@pytest.mark.parametrize("nz,nx", [(1, 1), (3, 5), (16, 16), (33, 20)])
def test_precond_inverts_separable_operator(nz, nx):
    hx, hz = 5.0, 3.0
    for (ax, az, d) in [(2.0, 2.0, 0.3), (5.0, 1.5, 0.01)]:
        y = RNG.standard_normal((2, nz, nx))
        By = precond.apply_separable(y, hx, hz, ax, az, d)
        assert np.abs(precond.apply_inverse(By, hx, hz, ax, az, d) - y).max() < 1e-12
        # the separable operator with ax == az == kappa~ and d == rho~ h^2/4 is A with a
        # homogeneous medium (Eq. 21 vs Eqs. 16-18)
    kap, rho, h = 4.0, 2.0, 1.3
    y = RNG.standard_normal((nz, nx))
    Ay = fd.apply_A(y, np.full((nz, nx), kap), np.full((nz, nx), rho), h, hx, hz)
    By = precond.apply_separable(y, hx, hz, kap, kap, rho * h * h / 4)
    assert np.abs(Ay - By).max() < 1e-12 * np.abs(Ay).max()


def test_precond_eigenvector_closed_form():
    nz, nx, hx, hz = 11, 14, 2.0, 3.0
    ax, az, d = 3.0, 1.0, 0.2
    p, q = 3, 7
    v = np.outer(dst.dst_matrix(nz)[:, q], dst.dst_matrix(nx)[:, p])
    ev = ax * dst.laplace_eigenvalues(nx, hx)[p] + az * dst.laplace_eigenvalues(nz, hz)[q] + d
    assert np.abs(precond.apply_inverse(v, hx, hz, ax, az, d) - v / ev).max() < 1e-13 / ev


def test_midrange_and_params():
    kappa = np.array([[1.0, 9.0], [4.0, 2.0]])
    rho = np.array([[1.0, 3.0], [2.0, 2.0]])
    ax, az, d = precond.acoustic_params(kappa, rho, 10.0)
    assert (ax, az) == (5.0, 5.0) and d == pytest.approx(2.0 * 100 / 4)
    lam = np.array([[1.0, 2.0]])
    mu = np.array([[1.0, 3.0]])
    (p1, m1, d1), (m2, p2, d2) = precond.elastic_params(lam, mu, np.array([[2.0, 4.0]]), 2.0)
    assert p1 == p2 == pytest.approx(0.5 * (3.0 + 8.0)) and m1 == m2 == 2.0 and d1 == d2 == 3.0


# ------------------------------------------------------------------------------- Krylov
def test_pcg_equals_dense_solve_and_homogeneous_one_iteration():
    nz, nx, hx, hz, h = 12, 10, 5.0, 5.0, 200.0
    kappa, rho = _medium(nz, nx)
    M = fd.assemble_A(kappa, rho, h, hx, hz)
    b = RNG.standard_normal(nz * nx)
    pr = precond.acoustic_params(kappa, rho, h)
    x, it, hist = krylov.pcg(lambda v: M @ v,
                             lambda v: precond.apply_inverse(v.reshape(nz, nx), hx, hz, *pr).ravel(),
                             b, 1e-13)
    xd = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11
    assert 1 < it < 100
    # homogeneous medium: A == B, so PCG converges in one iteration
    kh, rh = np.full((nz, nx), 9e9), np.full((nz, nx), 2000.0)
    pr = precond.acoustic_params(kh, rh, h)
    x, it, _ = krylov.pcg(lambda v: fd.apply_A(v.reshape(nz, nx), kh, rh, h, hx, hz).ravel(),
                          lambda v: precond.apply_inverse(v.reshape(nz, nx), hx, hz, *pr).ravel(),
                          b, 1e-12)
    assert it == 1


def test_pcg_iterations_nearly_mesh_independent():
    # Sec. 2.4: the iteration count practically does not depend on the number of mesh nodes
    its = []
    for n in (32, 64, 128):
        xs = (np.arange(n) + 1) / (n + 1)
        X, Z = np.meshgrid(xs, xs)
        c = 2000 + 1500 * np.sin(3 * X) ** 2 * np.cos(2 * Z) ** 2
        rho = 310 * c ** 0.25
        kappa = fd.kappa_from_velocity(c, rho)
        hx = 2560.0 / (n + 1)
        pr = precond.acoustic_params(kappa, rho, 200.0)
        b = np.zeros((n, n))
        b[n // 4, n // 2] = 1.0 / hx ** 2
        _, it, _ = krylov.pcg(lambda v: fd.apply_A(v.reshape(n, n), kappa, rho, 200.0, hx, hx).ravel(),
                              lambda v: precond.apply_inverse(v.reshape(n, n), hx, hx, *pr).ravel(),
                              b.ravel(), 1e-10)
        its.append(it)
    assert max(its) - min(its) <= 6, its


def test_gmres_dense_limits():
    n = 30
    A = np.eye(n) * 4 + RNG.uniform(-1, 1, (n, n)) * 0.4          # nonsymmetric, positive definite part
    b = RNG.standard_normal(n)
    xd = np.linalg.solve(A, b)
    ident = lambda v: v
    x, it, hist = krylov.gmres(lambda v: A @ v, ident, b, k=n, tol=1e-13)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11 and it <= n
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))  # monotone
    x1, it1, _ = krylov.gmres(lambda v: A @ v, ident, b, k=1, tol=1e-10)       # GMRES(1) converges
    assert np.linalg.norm(x1 - xd) / np.linalg.norm(xd) < 1e-8
    # right preconditioning by the exact inverse converges in one step
    Ainv = np.linalg.inv(A)
    x2, it2, _ = krylov.gmres(lambda v: A @ v, lambda v: Ainv @ v, b, k=5, tol=1e-12)
    assert it2 == 1 and np.linalg.norm(x2 - xd) / np.linalg.norm(xd) < 1e-11


# ------------------------------------------------------------------- free surface (Eq. 3)
def _neumann_dirichlet_mode(nz, q, hz):
    """Closed form of the z-operator with no flux through the top face and u = 0 below row
    nz - 1: v_k = cos(theta (k + 1/2)), theta = pi (q + 1/2) / (nz + 1/2), eigenvalue
    (4 / hz^2) sin^2(theta / 2) (the mirror ghost v_{-1} = v_0 holds since cos is even about
    k = -1/2, and v_nz = cos(pi (q + 1/2)) = 0)."""
    th = np.pi * (q + 0.5) / (nz + 0.5)
    return np.cos(th * (np.arange(nz) + 0.5)), 4.0 / hz ** 2 * np.sin(th / 2) ** 2


def test_free_surface_operator_closed_form_eigenfunction():
    nz, nx, hx, hz, h = 9, 12, 3.0, 4.0, 50.0
    kappa, rho = 7.0, 2.0
    p, q = 4, 6
    vz, mu = _neumann_dirichlet_mode(nz, q, hz)
    v = np.outer(vz, dst.dst_matrix(nx)[:, p])
    Av = fd.apply_A(v, np.full((nz, nx), kappa), np.full((nz, nx), rho), h, hx, hz, free_surface=True)
    ev = kappa * (dst.laplace_eigenvalues(nx, hx)[p] + mu) + rho * h * h / 4
    assert np.abs(Av - ev * v).max() < 1e-12 * ev
    # the Dirichlet operator does not have this eigenvector: its row 0 differs by the top-face
    # flux kappa v_0 / hz^2 (and by nothing else)
    Ad = fd.apply_A(v, np.full((nz, nx), kappa), np.full((nz, nx), rho), h, hx, hz)
    assert np.allclose((Ad - Av)[0], kappa / hz ** 2 * v[0], rtol=1e-12, atol=0)
    assert np.abs((Ad - Av)[1:]).max() < 1e-12 * ev


def test_free_surface_assembly_spd_and_only_top_row_changes():
    nz, nx, hx, hz, h = 5, 7, 10.0, 7.0, 200.0
    kappa, rho = _medium(nz, nx)
    M = fd.assemble_A(kappa, rho, h, hx, hz, free_surface=True)
    cols = np.stack([fd.apply_A(e.reshape(nz, nx), kappa, rho, h, hx, hz, free_surface=True).ravel()
                     for e in np.eye(nz * nx)], axis=1)
    assert np.abs(cols - M).max() / np.abs(M).max() < 1e-14
    assert np.abs(M - M.T).max() / np.abs(M).max() < 1e-15
    assert np.linalg.eigvalsh(M).min() > 0
    D = fd.assemble_A(kappa, rho, h, hx, hz) - M
    # the difference is the top-face flux of row 0 only: kappa_{0,i} / hz^2 on those diagonals
    assert np.allclose(np.diag(D)[:nx], kappa[0] / hz ** 2, rtol=1e-14)
    D[np.arange(nx), np.arange(nx)] = 0.0
    assert np.abs(D).max() == 0.0


def test_free_surface_preconditioner_closed_form_and_inverse():
    nz, nx, hx, hz = 11, 14, 2.0, 3.0
    ax, az, d = 3.0, 1.0, 0.2
    p, q = 3, 7
    vz, mu = _neumann_dirichlet_mode(nz, q, hz)
    v = np.outer(vz, dst.dst_matrix(nx)[:, p])
    ev = ax * dst.laplace_eigenvalues(nx, hx)[p] + az * mu + d
    assert np.abs(precond.apply_inverse(v, hx, hz, ax, az, d, free_surface=True) - v / ev).max() < 1e-13 / ev
    y = RNG.standard_normal((2, nz, nx))
    By = precond.apply_separable(y, hx, hz, ax, az, d, free_surface=True)
    assert np.abs(precond.apply_inverse(By, hx, hz, ax, az, d, free_surface=True) - y).max() < 1e-12


def test_free_surface_pcg_homogeneous_one_iteration():
    nz, nx, hx, hz, h = 12, 10, 5.0, 5.0, 200.0
    kh, rh = np.full((nz, nx), 9e9), np.full((nz, nx), 2000.0)
    pr = precond.acoustic_params(kh, rh, h)
    b = RNG.standard_normal(nz * nx)
    x, it, _ = krylov.pcg(lambda v: fd.apply_A(v.reshape(nz, nx), kh, rh, h, hx, hz, free_surface=True).ravel(),
                          lambda v: precond.apply_inverse(v.reshape(nz, nx), hx, hz, *pr, free_surface=True).ravel(),
                          b, 1e-12)
    assert it == 1
    M = fd.assemble_A(kh, rh, h, hx, hz, free_surface=True)
    assert np.linalg.norm(M @ x - b) / np.linalg.norm(b) < 1e-11


# ------------------------------------------------ layered preconditioner (design extension)
@pytest.mark.parametrize("free_surface", [False, True])
def test_layered_precond_inverts_its_operator_and_reduces_to_constant(free_surface):
    nz, nx, hx, hz = 17, 23, 4.0, 3.0
    ax = RNG.uniform(1.0, 3.0, nz)
    az = RNG.uniform(1.0, 3.0, nz)
    d = RNG.uniform(0.1, 0.5, nz)
    y = RNG.standard_normal((2, nz, nx))
    By = precond.apply_separable_layered(y, hx, hz, ax, az, d, free_surface)
    assert np.abs(precond.apply_inverse_layered(By, hx, hz, ax, az, d, free_surface) - y).max() < 1e-12
    # constant rows: the layered preconditioner is the constant one
    c = np.ones(nz)
    r = RNG.standard_normal((nz, nx))
    a = precond.apply_inverse_layered(r, hx, hz, 2.0 * c, 1.5 * c, 0.3 * c, free_surface)
    b = precond.apply_inverse(r, hx, hz, 2.0, 1.5, 0.3, free_surface)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("free_surface", [False, True])
def test_layered_precond_equals_A_for_a_z_only_medium(free_surface):
    # kappa and rho depending on z only: the layered operator IS A, and PCG takes one iteration
    nz, nx, hx, hz, h = 14, 11, 5.0, 4.0, 200.0
    kz = RNG.uniform(1e9, 9e9, nz)
    rz = RNG.uniform(1000.0, 2500.0, nz)
    kappa = np.repeat(kz[:, None], nx, axis=1)
    rho = np.repeat(rz[:, None], nx, axis=1)
    ax, az, d = precond.acoustic_params_layered(kappa, rho, h)
    y = RNG.standard_normal((nz, nx))
    Ay = fd.apply_A(y, kappa, rho, h, hx, hz, free_surface)
    By = precond.apply_separable_layered(y, hx, hz, ax, az, d, free_surface)
    assert np.abs(Ay - By).max() < 1e-12 * np.abs(Ay).max()
    b = RNG.standard_normal(nz * nx)
    x, it, _ = krylov.pcg(lambda v: fd.apply_A(v.reshape(nz, nx), kappa, rho, h, hx, hz, free_surface).ravel(),
                          lambda v: precond.apply_inverse_layered(v.reshape(nz, nx), hx, hz, ax, az, d,
                                                                  free_surface).ravel(), b, 1e-12)
    assert it == 1


def test_layered_precond_needs_fewer_iterations_on_layers():
    # the property the extension is for: on a layered model with noise it beats the constant one
    nz, nx, hx, h = 48, 40, 10.0, 200.0
    layers = (np.arange(nz) * 6) // nz
    c = RNG.uniform(1500, 4500, 6)[layers][:, None] * (1 + 0.02 * RNG.standard_normal((nz, nx)))
    rho = 310 * c ** 0.25
    kappa = fd.kappa_from_velocity(c, rho)
    A = lambda v: fd.apply_A(v.reshape(nz, nx), kappa, rho, h, hx, hx).ravel()
    b = RNG.standard_normal(nz * nx)
    pc = precond.acoustic_params(kappa, rho, h)
    pl = precond.acoustic_params_layered(kappa, rho, h)
    _, it_c, _ = krylov.pcg(A, lambda v: precond.apply_inverse(v.reshape(nz, nx), hx, hx, *pc).ravel(), b, 1e-10)
    xl, it_l, _ = krylov.pcg(A, lambda v: precond.apply_inverse_layered(v.reshape(nz, nx), hx, hx, *pl).ravel(), b, 1e-10)
    assert it_l < it_c / 2
    M = fd.assemble_A(kappa, rho, h, hx, hx)
    assert np.linalg.norm(M @ xl - b) / np.linalg.norm(b) < 1e-9


def test_layered_elastic_blocks_equal_the_diagonal_blocks_of_C_for_a_z_only_medium():
    # lambda, mu, rho depending on z only: the layered B1 is the u-u block of C and B2 the w-w
    # block (the face rule of the elastic operator is the layered preconditioner's), so K differs
    # from C by the mixed u-w terms alone
    nz, nx, hx, hz, h = 13, 10, 2.5, 3.0, 300.0
    lam = np.repeat(RNG.uniform(2e9, 9e9, nz)[:, None], nx, axis=1)
    mu = np.repeat(RNG.uniform(1e9, 5e9, nz)[:, None], nx, axis=1)
    rho = np.repeat(RNG.uniform(1800.0, 2600.0, nz)[:, None], nx, axis=1)
    p1, p2 = precond.elastic_params_layered(lam, mu, rho, h)
    y = RNG.standard_normal((nz, nx))
    zero = np.zeros_like(y)
    cu, _ = fd.apply_C(y, zero, lam, mu, rho, h, hx, hz)
    _, cw = fd.apply_C(zero, y, lam, mu, rho, h, hx, hz)
    # the mixed terms of a field in one component only land in the other component
    assert np.abs(cu - precond.apply_separable_layered(y, hx, hz, *p1)).max() < 1e-12 * np.abs(cu).max()
    assert np.abs(cw - precond.apply_separable_layered(y, hx, hz, *p2)).max() < 1e-12 * np.abs(cw).max()
    # constant rows: the layered blocks are Eq. 22's constant ones
    c1, c2 = precond.elastic_params(lam[:1].repeat(nz, 0), mu[:1].repeat(nz, 0), rho[:1].repeat(nz, 0), h)
    l1, l2 = precond.elastic_params_layered(lam[:1].repeat(nz, 0), mu[:1].repeat(nz, 0), rho[:1].repeat(nz, 0), h)
    r = RNG.standard_normal((nz, nx))
    for c, l in ((c1, l1), (c2, l2)):
        a = precond.apply_inverse_layered(r, hx, hz, *l)
        b = precond.apply_inverse(r, hx, hz, *c)
        assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


def test_layered_elastic_precond_needs_fewer_iterations_on_layers():
    # FGMRES(20) on a layered elastic model with lateral noise: per-row midranges beat Eq. 22's
    # whole-medium ones, and the solution satisfies the dense system
    nz, nx, hx, h = 36, 30, 5.0, 300.0
    layers = (np.arange(nz) * 5) // nz
    vp = RNG.uniform(2000, 5000, 5)[layers][:, None] * (1 + 0.02 * RNG.standard_normal((nz, nx)))
    vs = vp / 1.8
    rho = RNG.uniform(1800, 2600, 5)[layers][:, None] * np.ones((1, nx))
    from oracle.solve import elastic_lame
    lam, mu = elastic_lame(vp, vs, rho)
    n = nz * nx

    def C(v):
        a, b = fd.apply_C(v[:n].reshape(nz, nx), v[n:].reshape(nz, nx), lam, mu, rho, h, hx, hx)
        return np.concatenate([a.ravel(), b.ravel()])

    def K(params, inv):
        return lambda v: np.concatenate([inv(v[:n].reshape(nz, nx), hx, hx, *params[0]).ravel(),
                                         inv(v[n:].reshape(nz, nx), hx, hx, *params[1]).ravel()])
    b = RNG.standard_normal(2 * n)
    _, it_c, _ = krylov.gmres(C, K(precond.elastic_params(lam, mu, rho, h), precond.apply_inverse), b, 20, 1e-10, 2000)
    x, it_l, _ = krylov.gmres(C, K(precond.elastic_params_layered(lam, mu, rho, h), precond.apply_inverse_layered),
                              b, 20, 1e-10, 2000)
    assert it_l < 0.75 * it_c
    assert np.linalg.norm(C(x) - b) / np.linalg.norm(b) < 1e-9
