"""Laguerre transform pieces (oracle).  Test infrastructure only.

Sec. 2.1 (the display defining l_m^alpha and Eqs. (7)-(9)):

  orthonormal Laguerre functions
      l_m(ht) = sqrt(h m!/(m+alpha)!) (ht)^{alpha/2} e^{-ht/2} L_m^alpha(ht)
  forward transform      R_m = int_0^inf u(t) (ht)^{-alpha/2} l_m(ht) dt           (Eq. 7)
  inverse summation      u(t) = (ht)^{alpha/2} sum_m R_m l_m(ht)                     (Eq. 8)
  source coefficients    f_m = int_0^inf f(t) (ht)^{-alpha/2} l_m(ht) dt            (below Eq. 9)
  spectral recurrence    (Eq. 9, moved to the SPD form A R_m = b_m)
      b_m = delta_s f_m - rho h^2 c_m sum_{k<m} (m-k) c^_k R_k,
      c_m = sqrt(m!/(m+alpha)!),  c^_k = sqrt((k+alpha)!/k!).

The paper labels both Eq. 7 and Eq. 8 "series_lag"; the reading above (forward transform with
weight (ht)^{-alpha/2}, inverse with factor (ht)^{alpha/2}) is the only one under which the
two are inverse to each other for orthonormal l_m.

Evaluation of l_m for large ht (silent in the paper): e^{-ht/2} underflows for ht > ~1400, so
the normalised functions ell_m(x) = sqrt(m!/(m+alpha)!) x^{alpha/2} e^{-x/2} L_m^alpha(x) are
produced by the three-term recurrence of the classical polynomials (Abramowitz & Stegun 22.7.12),
renormalised:

    ell_{m+1} = [(2m+alpha+1-x) ell_m - sqrt(m(m+alpha)) ell_{m-1}] / sqrt((m+1)(m+alpha+1)),

started from log ell_0 = (alpha/2) ln x - x/2 - (1/2) ln Gamma(alpha+1), with the values carried
as mantissa * exp(log-scale) and rescaled whenever a mantissa leaves [2^-500, 2^500].
"""
import math

import numpy as np
from scipy.special import gammaln

_BIG = 2.0 ** 500


def c_m(m, alpha):
    """c_m = sqrt(m!/(m+alpha)!) via log-gamma."""
    m = np.asarray(m, dtype=np.float64)
    return np.exp(0.5 * (gammaln(m + 1.0) - gammaln(m + alpha + 1.0)))


def chat_k(k, alpha):
    """c^_k = sqrt((k+alpha)!/k!) = 1/c_k."""
    k = np.asarray(k, dtype=np.float64)
    return np.exp(0.5 * (gammaln(k + alpha + 1.0) - gammaln(k + 1.0)))


def ell_table(n, x, alpha, extra_log=None):
    """ell_m(x) for m = 0..n-1 and every x (array); returns [n, len(x)].

    ``extra_log`` (array like x) is added to the starting log-scale; it lets callers multiply
    by a positive power of x inside the scaled arithmetic (e.g. (ht)^{alpha/2} for Eq. 8)
    without leaving the representable range."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros((n, x.size))
    with np.errstate(divide="ignore"):
        logx = np.where(x > 0, np.log(np.where(x > 0, x, 1.0)), -np.inf)
    logs = 0.5 * alpha * logx - 0.5 * x - 0.5 * gammaln(alpha + 1.0)
    if extra_log is not None:
        logs = logs + np.asarray(extra_log, dtype=np.float64)
    zero = ~np.isfinite(logs)              # x = 0 with alpha > 0: every ell_m(0) = 0
    logs = np.where(zero, 0.0, logs)
    prev = np.zeros_like(x)                # ell_{-1} = 0
    cur = np.ones_like(x)                  # mantissa of ell_0
    for m in range(n):
        with np.errstate(divide="ignore"):
            mag = np.exp(np.log(np.abs(cur)) + logs)       # |ell_m| = |mantissa| e^{log-scale}
        out[m] = np.where(zero, 0.0, np.sign(cur) * mag)
        nxt = ((2 * m + alpha + 1.0 - x) * cur - math.sqrt(m * (m + alpha)) * prev) \
            / math.sqrt((m + 1.0) * (m + alpha + 1.0))
        prev, cur = cur, nxt
        big = np.abs(cur) > _BIG
        if np.any(big):
            prev = np.where(big, prev / _BIG, prev)
            cur = np.where(big, cur / _BIG, cur)
            logs = np.where(big, logs + 500.0 * math.log(2.0), logs)
    return out


def ell_direct(m, x, alpha):
    """ell_m(x) straight from its definition with scipy's L_m^alpha (moderate x only)."""
    from scipy.special import eval_genlaguerre
    x = np.asarray(x, dtype=np.float64)
    return c_m(m, alpha) * x ** (alpha / 2.0) * np.exp(-x / 2.0) * eval_genlaguerre(m, alpha, x)


def gauss_legendre_panels(t0, t1, panels, order=16):
    """Composite Gauss-Legendre nodes and weights on [t0, t1]."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(t0, t1, panels + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])[:, None]
    half = 0.5 * (edges[1:] - edges[:-1])[:, None]
    return (mid + half * xg).ravel(), (half * wg).ravel()


def forward_coeffs(fun, n, h, alpha, t_end, panels=None, order=16):
    """R_m = int_0^t_end u(t) (ht)^{-alpha/2} l_m(ht) dt for m < n (Eq. 7 / f_m below Eq. 9).

    The integrand equals sqrt(h) c_m e^{-ht/2} L_m(ht) u(t) = sqrt(h) (ht)^{-alpha/2} ell_m(ht) u(t);
    it is evaluated as sqrt(h) * ell_m(ht) with the log-scale lowered by (alpha/2) ln(ht).
    ``fun`` must be negligible beyond t_end.  Panels default to enough 16-point rules to put
    >= 16 nodes in every local oscillation of ell_{n-1} and of fun."""
    if panels is None:
        panels = max(64, 4 * n + int(8 * h * t_end / 16) + 64)
    t, wq = gauss_legendre_panels(0.0, t_end, panels, order)
    x = h * t
    tab = ell_table(n, x, alpha, extra_log=-0.5 * alpha * np.log(x))
    return math.sqrt(h) * tab @ (wq * fun(t))


def inverse_sum(R, t, h, alpha):
    """u(t) = (ht)^{alpha/2} sqrt(h) sum_m R_m ell_m(ht)  (Eq. 8).  R: [n, ...] -> [len(t), ...]."""
    R = np.asarray(R, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    x = h * t
    with np.errstate(divide="ignore"):
        extra = np.where(x > 0, 0.5 * alpha * np.log(np.where(x > 0, x, 1.0)), 0.0)
    tab = ell_table(R.shape[0], x, alpha, extra_log=extra)     # [n, nt] incl. (ht)^{alpha/2}
    return math.sqrt(h) * np.tensordot(tab.T, R, axes=(1, 0))


def history_direct(R_prev, m, alpha):
    """sum_{k<m} (m-k) c^_k R_k exactly as printed in Eq. (9).  R_prev: list of arrays R_0..R_{m-1}."""
    acc = None
    for k in range(m):
        term = (m - k) * float(chat_k(k, alpha)) * R_prev[k]
        acc = term if acc is None else acc + term
    return acc


def ricker(f0, t0):
    """Ricker wavelet f(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).

    Reading of the workload's source: the paper's own wavelet (Eq. 23) is offered by
    ``paper_wavelet``; t0 defaults upstream to 1.5/f0 so that f(0) ~ 1e-8 (initial data Eq. 4)."""
    def f(t):
        a = (math.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
        return (1.0 - 2.0 * a) * np.exp(-a)
    return f


def paper_wavelet(f0, t0, gamma):
    """Eq. (23): exp[-(2 pi f0 (t-t0))^2 / gamma^2] sin(2 pi f0 (t-t0))."""
    def f(t):
        s = 2.0 * math.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)
        return np.exp(-(s ** 2) / gamma ** 2) * np.sin(s)
    return f
