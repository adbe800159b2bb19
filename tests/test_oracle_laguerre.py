"""Pins of the oracle's Laguerre pieces (Sec. 2.1, Eqs. (7)-(9)) against closed forms,
library routines and an independent ODE integration."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.special import roots_genlaguerre

from oracle import laguerre as L


@pytest.mark.parametrize("alpha", [2, 8, 9])
def test_ell_recurrence_matches_definition(alpha):
    x = np.array([0.05, 0.5, 3.0, 7.3, 40.0, 150.0, 400.0])
    tab = L.ell_table(80, x, alpha)
    direct = np.array([L.ell_direct(m, x, alpha) for m in range(80)])
    assert np.abs(tab - direct).max() < 1e-13


@pytest.mark.parametrize("alpha", [2, 9])
def test_ell_orthonormal_by_gauss_laguerre(alpha):
    # int_0^inf ell_m ell_n dx = delta_mn; Gauss-Laguerre with weight x^alpha e^{-x} is exact
    # for the polynomial part L_m L_n when m + n < 2N.
    N = 60
    xg, wg = roots_genlaguerre(N, alpha)
    tab = L.ell_table(40, xg, alpha)
    G = (tab * (wg / (xg ** alpha * np.exp(-xg)))) @ tab.T
    assert np.abs(G - np.eye(40)).max() < 1e-11


def test_ell_large_argument_scaled():
    # ht far beyond e^{-ht/2} underflow: compare with mpmath at high precision
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    alpha, x = 8, 2400.0
    tab = L.ell_table(1200, np.array([x]), alpha)[:, 0]
    for m in (500, 700, 1100, 1199):
        ref = (mpmath.sqrt(mpmath.factorial(m) / mpmath.factorial(m + alpha))
               * mpmath.power(x, alpha / 2) * mpmath.exp(-x / 2) * mpmath.laguerre(m, alpha, x))
        ref = float(ref)
        assert abs(tab[m] - ref) <= 1e-10 * max(abs(ref), 1e-3), (m, tab[m], ref)


def test_forward_transform_closed_form():
    # u(t) = (ht)^alpha e^{-ht/2}  =>  R_0 = sqrt(alpha!/h),  R_m = 0 (m > 0)
    h, alpha = 400.0, 9
    R = L.forward_coeffs(lambda t: (h * t) ** alpha * np.exp(-h * t / 2), 12, h, alpha, 0.5)
    assert R[0] == pytest.approx(math.sqrt(math.factorial(alpha) / h), rel=1e-13)
    assert np.abs(R[1:]).max() < 1e-12 * R[0]
    t = np.linspace(0.001, 0.2, 17)
    u = L.inverse_sum(R, t, h, alpha)
    ref = (h * t) ** alpha * np.exp(-h * t / 2)
    assert np.abs(u - ref).max() < 1e-12 * ref.max()


def test_forward_transform_parseval():
    # orthonormal l_m in L^2(dt): sum R_m^2 = int u^2 (ht)^{-alpha} dt
    h, alpha = 300.0, 8
    u = lambda t: (h * t) ** alpha * np.exp(-h * t / 3) * np.sin(40 * t)
    R = L.forward_coeffs(u, 200, h, alpha, 1.0)
    t, w = L.gauss_legendre_panels(0.0, 1.0, 400)
    ref = np.sum(w * u(t) ** 2 * (h * t) ** (-alpha))
    assert np.sum(R ** 2) == pytest.approx(ref, rel=1e-11)


def test_forward_quadrature_converged_by_doubling():
    f0 = 25.0
    fun = L.ricker(f0, 2.5 / f0)
    t_end = 2.5 / f0 + 4.0 / f0
    R1 = L.forward_coeffs(fun, 512, 200.0, 9, t_end)
    R2 = L.forward_coeffs(fun, 512, 200.0, 9, t_end, panels=2 * (4 * 512 + 64 + int(8 * 200 * t_end / 16)))
    assert np.abs(R1 - R2).max() < 1e-13 * np.abs(R1).max()


def test_round_trip_ricker():
    f0, h, alpha = 25.0, 200.0, 9
    fun = L.ricker(f0, 2.5 / f0)
    R = L.forward_coeffs(fun, 512, h, alpha, 2.5 / f0 + 4.0 / f0)
    t = np.linspace(0.002, 0.5, 200)
    assert np.abs(L.inverse_sum(R, t, h, alpha) - fun(t)).max() < 1e-9


def test_spectral_recurrence_scalar_oscillator():
    # One mode of the semi-discrete problem: rho u'' + q u = f(t).  Transforming it gives the
    # scalar form of Eq. (9):  (q + rho h^2/4) R_m = f_m - rho h^2 c_m sum_{k<m} (m-k) c^_k R_k.
    # R_m of the true u (integrated independently by an ODE solver) must satisfy it.
    rho, q, h, alpha, f0 = 1.5, 2.0e5, 200.0, 9, 25.0
    t0 = 2.5 / f0
    fun = L.ricker(f0, t0)
    n = 48
    T = (4 * n + 200) / h
    sol = solve_ivp(lambda t, y: [y[1], (fun(t) - q * y[0]) / rho], (0.0, T), [0.0, 0.0],
                    method="DOP853", rtol=1e-13, atol=1e-20, dense_output=True)
    R = L.forward_coeffs(lambda t: sol.sol(t)[0], n, h, alpha, T, panels=3000)
    fm = L.forward_coeffs(fun, n, h, alpha, t0 + 4.0 / f0)
    scale = np.abs(R).max()
    for m in range(n):
        hist = L.history_direct(list(R[:m]), m, alpha) if m else 0.0
        lhs = (q + rho * h * h / 4) * R[m]
        rhs = fm[m] - rho * h * h * float(L.c_m(m, alpha)) * hist
        assert abs(lhs - rhs) <= 1e-8 * (q + rho * h * h / 4) * scale, m


def test_history_accumulators_equal_direct_sum():
    # T_{m+1} = T_m + c^_m R_m, S_{m+1} = S_m + T_{m+1} reproduces sum_{k<m}(m-k) c^_k R_k
    rng = np.random.default_rng(7)
    alpha = 9
    R = [rng.standard_normal(5) for _ in range(40)]
    T = np.zeros(5)
    S = np.zeros(5)
    for m in range(40):
        if m:
            assert np.allclose(S, L.history_direct(R, m, alpha), rtol=1e-13, atol=0)
        T = T + float(L.chat_k(m, alpha)) * R[m]
        S = S + T
