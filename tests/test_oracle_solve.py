"""Pins of the oracle's whole-shot solves and of the elastic operator."""
import numpy as np
import pytest

from oracle import analytic, fd, krylov, laguerre, precond, solve


def _point_source_error(hx, n_nodes):
    # homogeneous 2 km x 2 km box, source in the middle, receiver 300 m away; the window ends
    # before the first boundary reflection reaches the receiver
    f0, h, alpha, c0, rho0 = 10.0, 400.0, 9, 2000.0, 1000.0
    t0 = 2.5 / f0
    t = np.linspace(0.01, 0.9, 120)
    N = n_nodes
    off = int(round(300.0 / hx))
    out = solve.acoustic_shot(np.full((N, N), c0), np.full((N, N), rho0), hx, hx, h, alpha, 160,
                              (N // 2, N // 2), [(N // 2 + off, N // 2)], t, f0, t0, tol=1e-12)
    ua = analytic.point_source_2d(off * hx, t, rho0 * c0 ** 2, rho0, laguerre.ricker(f0, t0))
    eps = np.sqrt(np.sum((out["traces"][0] - ua) ** 2) / np.sum(ua ** 2))   # Sec. 3.2 accuracy
    return eps, out["iters"]


def test_acoustic_shot_matches_2d_point_source_at_second_order():
    e20, it20 = _point_source_error(20.0, 99)
    e10, it10 = _point_source_error(10.0, 199)
    assert np.all(it20 == 1) and np.all(it10 == 1)        # homogeneous: A == B
    assert e10 < 0.08
    assert 3.0 < e20 / e10 < 5.5                             # O(h^2) (Sec. 3.2)


def _free_surface_error(hx, n_nodes):
    # homogeneous 2 km x 2 km box with a free surface on top (the zero-flux face half a cell
    # above node row 0); source and receiver 500 m below it, 300 m apart.  Method of images:
    # u = G(direct) + G(mirror image above the surface); the window ends before the Dirichlet
    # sides or bottom send anything back.
    f0, h, alpha, c0, rho0 = 10.0, 400.0, 9, 2000.0, 1000.0
    t0 = 2.5 / f0
    t = np.linspace(0.01, 0.95, 120)
    N = n_nodes
    off = int(round(300.0 / hx))
    ks = int(round(500.0 / hx - 0.5))            # depth below the surface: (ks + 1/2) hx
    depth = (ks + 0.5) * hx
    out = solve.acoustic_shot(np.full((N, N), c0), np.full((N, N), rho0), hx, hx, h, alpha, 160,
                              (N // 2, ks), [(N // 2 + off, ks)], t, f0, t0, tol=1e-12, free_surface=True)
    f = laguerre.ricker(f0, t0)
    kap = rho0 * c0 ** 2
    ua = (analytic.point_source_2d(off * hx, t, kap, rho0, f)
          + analytic.point_source_2d(np.hypot(off * hx, 2 * depth), t, kap, rho0, f))
    eps = np.sqrt(np.sum((out["traces"][0] - ua) ** 2) / np.sum(ua ** 2))
    return eps, out["iters"]


def test_free_surface_shot_matches_image_solution_at_second_order():
    # second order only with the surface on the zero-flux face: placing it on the ghost node
    # (half a cell higher) converges at first order (measured ratio 1.8 for these grids)
    e10, it10 = _free_surface_error(10.0, 199)
    e5, it5 = _free_surface_error(5.0, 399)
    assert np.all(it10 == 1) and np.all(it5 == 1)         # homogeneous: A == B with the surface too
    assert e5 < 0.04
    assert 3.3 < e10 / e5 < 5.0                              # O(h^2)


def test_acoustic_shot_two_layer_small():
    from paper_1005_0542_gb300 import inputs
    s = inputs.two_layer(n_harm=8, nx=32, nz=32)
    out = solve.acoustic_shot(s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0],
                              s.receivers, s.t_out, s.f0, s.t0, tol=1e-12, keep_fields=True)
    # every harmonic solves A R_m = b_m: recheck the residual with the dense matrix
    kappa = fd.kappa_from_velocity(s.c, s.rho)
    M = fd.assemble_A(kappa, s.rho, s.h, s.hx, s.hz)
    R = out["fields"]
    for m in range(s.n_harm):
        b = np.zeros((32, 32))
        if m:
            b -= s.rho * s.h ** 2 * float(laguerre.c_m(m, s.alpha)) * laguerre.history_direct(list(R), m, s.alpha)
        b[s.sources[0][1], s.sources[0][0]] += out["fm"][m] / (s.hx * s.hz)
        assert np.linalg.norm(M @ R[m].ravel() - b.ravel()) <= 2e-12 * np.linalg.norm(b)
    assert np.all(out["iters"] > 1)


def test_layered_shot_same_traces_fewer_iterations():
    # the preconditioner changes the iteration, not the solution: traces equal to the tolerance,
    # and the per-row midranges take far fewer PCG iterations on a layered medium
    from paper_1005_0542_gb300 import inputs
    s = inputs.random_layered(nx=40, nz=32, hx=10.0, n_harm=6)
    args = (s.c, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0], s.receivers, s.t_out, s.f0, s.t0)
    a = solve.acoustic_shot(*args, tol=1e-12)
    b = solve.acoustic_shot(*args, tol=1e-12, layered=True)
    assert np.linalg.norm(a["traces"] - b["traces"]) <= 1e-9 * np.linalg.norm(a["traces"])
    assert b["iters"].sum() * 2 < a["iters"].sum()


# ------------------------------------------------------------------------- elastic operator
def _elastic_medium(nz, nx, seed=3):
    rng = np.random.default_rng(seed)
    vp = rng.uniform(2000, 5000, (nz, nx))
    rho = rng.uniform(1800, 2600, (nz, nx))
    return solve.elastic_lame(vp, vp / 1.73, rho) + (rho,)


def test_elastic_operator_symmetric_positive_definite():
    lam, mu, rho = _elastic_medium(5, 6)
    M = fd.assemble_C(lam, mu, rho, 300.0, 2.5, 3.0)
    assert np.abs(M - M.T).max() / np.abs(M).max() < 1e-14
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def _elastic_manufactured_error(n):
    sp = pytest.importorskip("sympy")
    x, z = sp.symbols("x z")
    lam = 2 + sp.Rational(1, 2) * sp.sin(x) * sp.cos(z)
    mu = 1 + sp.Rational(3, 10) * sp.cos(x) * sp.sin(z)
    u = sp.sin(x) * sp.sin(2 * z)
    w = sp.sin(2 * x) * sp.sin(z)
    rho, h = 3.0, 2.0
    p = lam + 2 * mu
    cu = -(sp.diff(p * sp.diff(u, x), x) + sp.diff(mu * sp.diff(u, z), z)
           + sp.diff(lam * sp.diff(w, z), x) + sp.diff(mu * sp.diff(w, x), z)) + rho * h * h / 4 * u
    cw = -(sp.diff(mu * sp.diff(w, x), x) + sp.diff(p * sp.diff(w, z), z)
           + sp.diff(mu * sp.diff(u, z), x) + sp.diff(lam * sp.diff(u, x), z)) + rho * h * h / 4 * w
    f = sp.lambdify((x, z), [lam, mu, u, w, cu, cw], "numpy")
    hh = np.pi / (n + 1)
    xs = hh * np.arange(1, n + 1)
    X, Z = np.meshgrid(xs, xs)
    L_, M_, U, W, CU, CW = [np.broadcast_to(np.asarray(a, dtype=float), X.shape) for a in f(X, Z)]
    gu, gw = fd.apply_C(U, W, L_, M_, np.full_like(X, rho), h, hh, hh)
    return max(np.abs(gu - CU)[2:-2, 2:-2].max(), np.abs(gw - CW)[2:-2, 2:-2].max())


def test_elastic_operator_second_order_truncation():
    # plane-strain reading of Eq. (12): every term (incl. both mixed terms) converges at O(h^2)
    e1, e2 = _elastic_manufactured_error(40), _elastic_manufactured_error(81)
    assert 3.5 < e1 / e2 < 4.5


def test_elastic_gmres_equals_dense_solve():
    nz, nx, h, hx, hz = 8, 9, 300.0, 2.5, 2.5
    lam, mu, rho = _elastic_medium(nz, nx, seed=11)
    M = fd.assemble_C(lam, mu, rho, h, hx, hz)
    b = np.random.default_rng(5).standard_normal(2 * nz * nx)
    p1, p2 = precond.elastic_params(lam, mu, rho, h)
    n = nz * nx

    def Kinv(v):
        return np.concatenate([precond.apply_inverse(v[:n].reshape(nz, nx), hx, hz, *p1).ravel(),
                               precond.apply_inverse(v[n:].reshape(nz, nx), hx, hz, *p2).ravel()])
    x, it, hist = krylov.gmres(lambda v: M @ v, Kinv, b, 20, 1e-13)
    xd = np.linalg.solve(M, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11
    assert it < 200


def test_elastic_shot_small_residuals():
    from paper_1005_0542_gb300 import inputs
    s = inputs.elastic_layered(nx=24, nz=16, hx=2.5, n_harm=6, nsrc=1)
    out = solve.elastic_shot(s.c, s.vs, s.rho, s.hx, s.hz, s.h, s.alpha, s.n_harm, s.sources[0],
                             s.receivers[:4], s.t_out, s.f0, s.t0, tol=1e-12, keep_fields=True)
    lam, mu = solve.elastic_lame(s.c, s.vs, s.rho)
    M = fd.assemble_C(lam, mu, s.rho, s.h, s.hx, s.hz)
    R = out["fields"]
    for m in range(s.n_harm):
        b = np.zeros((2, 16, 24))
        if m:
            b -= s.rho * s.h ** 2 * float(laguerre.c_m(m, s.alpha)) * laguerre.history_direct(list(R), m, s.alpha)
        b[1, s.sources[0][1], s.sources[0][0]] += out["fm"][m] / (s.hx * s.hz)
        assert np.linalg.norm(M @ R[m].ravel() - b.ravel()) <= 5e-12 * np.linalg.norm(b)
    assert out["traces"].shape == (2, 4, s.t_out.size)


# ---------------------------------------------------------------- Cartesian elastic shot (Sec. 2.2)
_LF = dict(lam=1000.0 * (2000.0 ** 2 - 2.0 * (2000.0 / 1.73) ** 2), mu=1000.0 * (2000.0 / 1.73) ** 2, rho=1000.0)


def _navier_residual(d, dt, swap_wake_sign=False):
    # rho u_tt - [(l+2m) grad div u - m curl curl u] by central differences (step d in space, dt
    # in time) at one point off the source, relative to the right-hand side
    lam, mu, rho = 2e9, 1.3e9, 1800.0
    f = laguerre.ricker(8.0, 2.5 / 8.0)
    x0, z0, t0 = 180.0, -140.0, np.array([0.55])
    wake = analytic._wake_integral

    def U(x, z, t):
        if swap_wake_sign:
            analytic._wake_integral = lambda *a: -wake(*a)
        try:
            return np.array(analytic.line_force_2d(x, z, t, lam, mu, rho, f, panels=256, order=12))[:, 0]
        finally:
            analytic._wake_integral = wake
    c = U(x0, z0, t0)
    utt = (U(x0, z0, t0 + dt) - 2 * c + U(x0, z0, t0 - dt)) / dt ** 2
    uxx = (U(x0 + d, z0, t0) - 2 * c + U(x0 - d, z0, t0)) / d ** 2
    uzz = (U(x0, z0 + d, t0) - 2 * c + U(x0, z0 - d, t0)) / d ** 2
    uxz = (U(x0 + d, z0 + d, t0) - U(x0 + d, z0 - d, t0) - U(x0 - d, z0 + d, t0) + U(x0 - d, z0 - d, t0)) / (4 * d * d)
    rx = (lam + 2 * mu) * uxx[0] + mu * uzz[0] + (lam + mu) * uxz[1]
    rz = (lam + 2 * mu) * uzz[1] + mu * uxx[1] + (lam + mu) * uxz[0]
    return max(abs(rho * utt[0] - rx) / abs(rx), abs(rho * utt[1] - rz) / abs(rz))


def test_line_force_solution_satisfies_navier_equation():
    # the derived plane-strain solution (oracle/analytic.py) solves the homogeneous Navier equation
    # away from the force: the finite-difference residual falls at O(d^2) (measured 0.0036, 0.00089);
    # the near-field term with the opposite sign leaves a residual of 10 %
    e2, e1 = _navier_residual(2.0, 2e-4), _navier_residual(1.0, 1e-4)
    assert e1 < 2e-3 and 3.5 < e2 / e1 < 4.5
    assert _navier_residual(2.0, 2e-4, swap_wake_sign=True) > 0.05


def _line_force_error(hx, history=None):
    # homogeneous box 1.4 km wide, a vertical force in the middle, four receivers 200-212 m away in
    # different directions (u_x vanishes on the two axes only); the window ends before the first
    # reflection off the Dirichlet sides returns.  Sec. 3.2's accuracy measure over both components.
    vp, rho0, f0, h, alpha = 2000.0, 1000.0, 8.0, 400.0, 8
    vs = vp / 1.73
    t = np.linspace(0.01, 0.72, 100)
    N = int(round(1400.0 / hx))
    N += (N + 1) % 2
    c = N // 2
    offs = [(200.0, 0.0), (0.0, 200.0), (150.0, 150.0), (-150.0, 100.0)]
    rcv = [(c + int(round(a / hx)), c + int(round(b / hx))) for a, b in offs]
    saved = laguerre.history_direct
    if history is not None:
        laguerre.history_direct = history
    try:
        out = solve.elastic_shot(np.full((N, N), vp), np.full((N, N), vs), np.full((N, N), rho0), hx, hx, h, alpha,
                                 120, (c, c), rcv, t, f0, 2.5 / f0, tol=1e-9)
    finally:
        laguerre.history_direct = saved
    f = laguerre.ricker(f0, 2.5 / f0)
    num = den = 0.0
    for j, (a, b) in enumerate(offs):
        ux, uz = analytic.line_force_2d(a, b, t, _LF["lam"], _LF["mu"], _LF["rho"], f)
        num += np.sum((out["traces"][0, j] - ux) ** 2) + np.sum((out["traces"][1, j] - uz) ** 2)
        den += np.sum(ux ** 2) + np.sum(uz ** 2)
    return np.sqrt(num / den)


def test_elastic_shot_matches_line_force_at_second_order():
    # pins the Cartesian elastic shot: the vertical force in the w-equation with weight
    # f_m / (hx hz), the history term of Eq. 12 and the inverse summation, against the plane-strain
    # line-force solution (measured eps 0.0876 at 10 m, 0.0223 at 5 m: ratio 3.9)
    e10, e5 = _line_force_error(10.0), _line_force_error(5.0)
    assert e5 < 0.03
    assert 3.3 < e10 / e5 < 4.8


def test_elastic_line_force_pin_rejects_a_wrong_history_weight():
    # the same shot with the history sum missing its (m - k) weight is far off the solution
    def no_weight(R_prev, m, alpha):
        acc = None
        for k in range(m):
            term = float(laguerre.chat_k(k, alpha)) * R_prev[k]
            acc = term if acc is None else acc + term
        return acc
    assert _line_force_error(10.0, history=no_weight) > 0.5
