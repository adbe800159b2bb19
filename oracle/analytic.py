"""Closed-form solutions used to pin the oracle (test infrastructure only).

* ``point_source_2d``: homogeneous 2D medium, rho u_tt = kappa Lap u + delta(x - x0) f(t),
  zero initial data (Eq. 4).  With c = sqrt(kappa/rho) (Sec. 3.2) the free-space Green's
  function of the 2D wave equation gives
      u(r, t) = 1/(2 pi kappa) int_0^{t - r/c} f(tau) / sqrt((t - tau)^2 - r^2/c^2) d tau.
  This is the Cartesian analogue of the paper's exact solution f(t - r/c)/(2 pi r) of Sec. 3.2
  (which is 3D, on a free surface); it is derived here, not printed in the paper.  The
  substitution tau = t - r/c - s^2 removes the inverse-square-root singularity:
      u = 1/(2 pi kappa) int_0^{sqrt(t - r/c)} 2 f(t - r/c - s^2) / sqrt(2r/c + s^2) ds.

* ``point_source_3d``: homogeneous 3D medium, rho u_tt = kappa Lap u + delta_3(x - x0) f(t):
      u(R, t) = f(t - R/c) / (4 pi kappa R),   R = |x - x0|.
  In cylindrical coordinates delta_3 = delta(r) delta(z - z0) / (2 pi r) on the axis, the source of
  Eq. 1; a free surface at z = 0 adds the mirror source at -z0 (the paper's exact solution of
  Sec. 3.2, f(t - r/c) / (2 pi r) with kappa = 1, is the case z0 = 0 seen on the surface).

* ``point_force_3d``: homogeneous isotropic elastic medium, rho u_tt = div sigma + e_z delta_3(x - x0)
  f(t) (a vertical point force), zero initial data.  Stokes' solution (the classical elastodynamic
  Green's function, near, intermediate and far field), with R = |x - x0|, gamma = (x - x0) / R,
  alpha / beta the P / S speeds:
      u_i = (3 g_i g_z - d_iz) / (4 pi rho R^3) int_{R/alpha}^{R/beta} tau f(t - tau) d tau
          + g_i g_z / (4 pi rho alpha^2 R) f(t - R/alpha) - (g_i g_z - d_iz) / (4 pi rho beta^2 R) f(t - R/beta).
  Returned as the radial (i = r, d_rz = 0) and vertical (i = z) components about the force axis.

* ``line_force_2d``: homogeneous isotropic elastic medium in plane strain,
  rho u_tt = div sigma + e_z delta(x - x0) f(t) (a vertical line force, the Cartesian source of
  Eq. 12), zero initial data.  Derived here (the paper prints no Cartesian elastic solution): split
  the force as e_z delta = grad div(e_z G0) - curl curl(e_z G0) with Lap G0 = delta; each part
  propagates with its own speed, u = (1/rho) [grad div(e_z (h_P - h_S)) + e_z g_S], where g_c is
  the 2D wave Green's function (g_tt - c^2 Lap g = delta(x) delta(t): g = H(ct - r) / (2 pi c
  sqrt(c^2 t^2 - r^2))) and Lap h_c = g_c.  For radial h, the Hessian is
  h'' g_i g_j + (h'/r)(d_ij - g_i g_j) with (r h')' = r g, which gives, with
  gamma = (x - x0)/r, alpha / beta the P / S speeds,
      rho u_i = g_i g_z (g_P * f) + (d_iz - g_i g_z) (g_S * f) + (d_iz - 2 g_i g_z) (K * f),
      K(r, t) = [H(beta t - r) sqrt(t^2 - r^2/beta^2) - H(alpha t - r) sqrt(t^2 - r^2/alpha^2)] / (2 pi r^2)
  (* a convolution in time).  (1/rho) g_c * f is point_source_2d with kappa = rho c^2; the K terms
  take the same substitution tau = t - r/c - s^2, under which sqrt((t - tau)^2 - r^2/c^2) d tau
  becomes 2 s^2 sqrt(2r/c + s^2) ds.

* ``oscillator``: one mode of the semi-discrete problem, rho u'' + q u = f(t), u(0)=u'(0)=0:
      u(t) = 1/(rho w) int_0^t sin(w (t - tau)) f(tau) d tau,  w = sqrt(q/rho).
  Its Laguerre coefficients must satisfy the scalar form of the spectral recurrence (Eq. 9):
      (q + rho h^2/4) R_m = f_m - rho h^2 c_m sum_{k<m} (m-k) c^_k R_k.
"""
import math

import numpy as np


def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def point_source_2d(r, t, kappa, rho, fun, nodes=400, panels=64):
    """u(r, t) for scalar r > 0 and an array of t (composite Gauss-Legendre in s)."""
    c = math.sqrt(kappa / rho)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    for j, tj in enumerate(t):
        smax2 = tj - r / c
        if smax2 <= 0.0:
            continue
        smax = math.sqrt(smax2)
        edges = np.linspace(0.0, smax, panels + 1)
        acc = 0.0
        for a, b in zip(edges[:-1], edges[1:]):
            s, w = _gl(a, b, max(8, nodes // panels))
            acc += np.sum(w * 2.0 * fun(tj - r / c - s * s) / np.sqrt(2.0 * r / c + s * s))
        out[j] = acc / (2.0 * math.pi * kappa)
    return out


def point_source_3d(R, t, kappa, rho, fun):
    """u(R, t) for scalar R > 0 and an array of t."""
    c = math.sqrt(kappa / rho)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.where(t > R / c, fun(t - R / c), 0.0) / (4.0 * math.pi * kappa * R)


def point_force_3d(r, dz, t, lam, mu, rho, fun, order=24, panels=16):
    """(u_r, u_z) at horizontal distance r >= 0 and height dz = z - z0 (R > 0) for an array of t."""
    a = math.sqrt((lam + 2.0 * mu) / rho)
    b = math.sqrt(mu / rho)
    R = math.hypot(r, dz)
    gr, gz = r / R, dz / R
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    near = np.zeros_like(t)
    edges = np.linspace(R / a, R / b, panels + 1)
    for lo, hi in zip(edges[:-1], edges[1:]):
        tau, w = _gl(lo, hi, order)
        near += np.sum(w[None, :] * tau[None, :] * fun(t[:, None] - tau[None, :]), axis=1)
    fa = fun(t - R / a)
    fb = fun(t - R / b)
    c = 1.0 / (4.0 * math.pi * rho)
    ur = c * (3.0 * gr * gz) / R ** 3 * near + c * gr * gz / (a * a * R) * fa - c * gr * gz / (b * b * R) * fb
    uz = (c * (3.0 * gz * gz - 1.0) / R ** 3 * near + c * gz * gz / (a * a * R) * fa
          - c * (gz * gz - 1.0) / (b * b * R) * fb)
    return ur, uz


def _wake_integral(r, t, c, fun, panels=64, order=8):
    """int_0^{t - r/c} sqrt((t - tau)^2 - r^2/c^2) f(tau) d tau for scalar r > 0 and an array of t."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    for j, tj in enumerate(t):
        smax2 = tj - r / c
        if smax2 <= 0.0:
            continue
        edges = np.linspace(0.0, math.sqrt(smax2), panels + 1)
        acc = 0.0
        for a, b in zip(edges[:-1], edges[1:]):
            s, w = _gl(a, b, order)
            acc += np.sum(w * 2.0 * s * s * np.sqrt(2.0 * r / c + s * s) * fun(tj - r / c - s * s))
        out[j] = acc
    return out


def line_force_2d(dx, dz, t, lam, mu, rho, fun, panels=64, order=8):
    """(u_x, u_z) at the offset (dx, dz) from a vertical line force (r > 0), array t."""
    a = math.sqrt((lam + 2.0 * mu) / rho)
    b = math.sqrt(mu / rho)
    r = math.hypot(dx, dz)
    gx, gz = dx / r, dz / r
    nodes = panels * order
    gp = point_source_2d(r, t, lam + 2.0 * mu, rho, fun, nodes=nodes, panels=panels)   # (1/rho) g_P * f
    gs = point_source_2d(r, t, mu, rho, fun, nodes=nodes, panels=panels)               # (1/rho) g_S * f
    kf = (_wake_integral(r, t, b, fun, panels, order) - _wake_integral(r, t, a, fun, panels, order)) / (
        2.0 * math.pi * r * r * rho)                                                     # (1/rho) K * f
    ux = gx * gz * gp - gx * gz * gs - 2.0 * gx * gz * kf
    uz = gz * gz * gp + (1.0 - gz * gz) * gs + (1.0 - 2.0 * gz * gz) * kf
    return ux, uz


def oscillator(t, q, rho, fun, panels=256, order=16):
    """u(t) of rho u'' + q u = f(t) from zero data, by Duhamel's integral (array t)."""
    w = math.sqrt(q / rho)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    for j, tj in enumerate(t):
        if tj <= 0.0:
            continue
        edges = np.linspace(0.0, tj, panels + 1)
        acc = 0.0
        for a, b in zip(edges[:-1], edges[1:]):
            tau, wq = _gl(a, b, order)
            acc += np.sum(wq * np.sin(w * (tj - tau)) * fun(tau))
        out[j] = acc / (rho * w)
    return out
