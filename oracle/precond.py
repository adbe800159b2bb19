"""Laplace-operator preconditioner (oracle).  Test infrastructure only.

Sec. 2.4, Eq. (21): B = Lambda_r + Lambda_z - d with constant coefficients equal to the
midrange of the medium's (footnote to Eq. 21: f~ = (min f + max f)/2).  Reading of the sign
garble: Eq. (21) as printed is negative definite; the oracle uses -B, the SPD operator of the
same form as A (Eqs. 16-18) with kappa == kappa~ and rho == rho~, in Cartesian form:

    -B y = -kappa~ (D_xx + D_zz) y + (rho~ h^2/4) y     (Dirichlet on all sides).

Separation of variables (Sec. 2.4; Sec. 3.1 names FFT + Dichotomy as the two steps):
  1. y^ = DST_x(r)                                        (orthonormal DST-I, S^2 = I)
  2. for each x-mode j: T_j y~_j = y^_j along z, with
        T_j = tridiag(-az~/hz^2,  2 az~/hz^2 + ax~ lambda_j + d~,  -az~/hz^2)
  3. y = DST_x(y~).

The separable operator is written with separate x / z coefficients (ax~, az~, d~) because
Eq. (22) needs them: the elastic K = diag(B1, B2) uses
  B1: ax~ = (lambda+2mu)~, az~ = mu~;   B2: ax~ = mu~, az~ = (lambda+2mu)~;   d~ = rho~ h^2/4
(the cylindrical 1/r term of B1 has no Cartesian counterpart and is dropped).
"""
import numpy as np

from . import dst as _dst
from .tridiag import thomas


def midrange(f):
    """f~ = (min f + max f) / 2 over all nodes (footnote to Eq. 21)."""
    f = np.asarray(f, dtype=np.float64)
    return 0.5 * (f.min() + f.max())


def acoustic_params(kappa, rho, h_lag):
    """(ax~, az~, d~) of the acoustic preconditioner B (Eq. 21)."""
    kt = midrange(kappa)
    return kt, kt, midrange(rho) * h_lag ** 2 / 4.0


def elastic_params(lam, mu, rho, h_lag):
    """((ax~, az~, d~) of B1, (ax~, az~, d~) of B2) for K = diag(B1, B2) (Eq. 22)."""
    pt = midrange(np.asarray(lam) + 2.0 * np.asarray(mu))
    mt = midrange(mu)
    dt = midrange(rho) * h_lag ** 2 / 4.0
    return (pt, mt, dt), (mt, pt, dt)


def mode_diagonals(nx, hx, hz, ax_t, az_t, d_t):
    """Main diagonal of T_j for every mode j: 2 az~/hz^2 + ax~ lambda_j + d~  ([nx])."""
    return 2.0 * az_t / hz ** 2 + ax_t * _dst.laplace_eigenvalues(nx, hx) + d_t


def apply_inverse(r, hx, hz, ax_t, az_t, d_t, free_surface=False):
    """y = (-B)^{-1} r for r [..., nz, nx]: DST along x, Thomas along z per mode, DST back.
    With a free surface the first row of every T_j loses the flux through the top face:
    diagonal az~/hz^2 + ax~ lambda_j + d~ (the same zero-flux reading as the operator)."""
    r = np.asarray(r, dtype=np.float64)
    nz, nx = r.shape[-2:]
    S = _dst.dst_matrix(nx)
    rh = _dst.dst_x(r, S)                                   # [..., nz, nx]
    diag = mode_diagonals(nx, hx, hz, ax_t, az_t, d_t)      # [nx]
    if free_surface:
        diag = np.broadcast_to(diag, (nz, nx)).copy()
        diag[0] -= az_t / hz ** 2
        diag = diag.reshape((nz,) + (1,) * (r.ndim - 2) + (nx,))
    off = -az_t / hz ** 2
    # move z to axis 0 so each (batch, mode) column is one independent system
    col = np.moveaxis(rh, -2, 0)                            # [nz, ..., nx]
    yt = thomas(off, diag, off, col)
    yh = np.moveaxis(yt, 0, -2)
    return _dst.dst_x(yh, S)


def apply_separable(y, hx, hz, ax_t, az_t, d_t, free_surface=False):
    """The separable operator itself: -ax~ D_xx y - az~ D_zz y + d~ y (Dirichlet; with a free
    surface the ghost above row 0 mirrors row 0, i.e. no flux through the top face), written as
    a 5-point stencil (used to pin apply_inverse)."""
    y = np.asarray(y, dtype=np.float64)
    pad = [(0, 0)] * (y.ndim - 2) + [(1, 1), (1, 1)]
    yp = np.pad(y, pad)
    if free_surface:
        yp[..., 0, 1:-1] = yp[..., 1, 1:-1]
    c = yp[..., 1:-1, 1:-1]
    dxx = (yp[..., 1:-1, 2:] - 2 * c + yp[..., 1:-1, :-2]) / hx ** 2
    dzz = (yp[..., 2:, 1:-1] - 2 * c + yp[..., :-2, 1:-1]) / hz ** 2
    return -ax_t * dxx - az_t * dzz + d_t * c


# ----------------------------------------------------------------------------------------
# Layered variant (a design extension beyond the paper): coefficients that vary with z only,
# ax~(z), az~(z), d~(z), each the midrange over its node row.  The x-operator still commutes
# with the DST along x (it only scales each row), so the separation of variables holds; the
# z-systems become general tridiagonal matrices (no longer Toeplitz):
#     T_j(k, k-1) = -az_f(k)/hz^2,   T_j(k, k+1) = -az_f(k+1)/hz^2,
#     T_j(k, k)   = (az_f(k) + az_f(k+1))/hz^2 + ax~(k) lambda_j + d~(k),
# with z-face coefficients az_f by the rule of the operator (mean of the two rows, a boundary face
# takes its row's value, the top face carries zero under a free surface).  For a medium whose
# kappa and rho depend on z only this operator equals A exactly.
# ----------------------------------------------------------------------------------------

def row_midranges(f):
    """Per-row midrange f~(z) = (min_x f + max_x f) / 2, shape [nz]."""
    f = np.asarray(f, dtype=np.float64)
    return 0.5 * (f.min(axis=1) + f.max(axis=1))


def acoustic_params_layered(kappa, rho, h_lag):
    """(ax~(z), az~(z), d~(z)) of the layered acoustic preconditioner."""
    kz = row_midranges(kappa)
    return kz, kz.copy(), row_midranges(rho) * h_lag ** 2 / 4.0


def elastic_params_layered(lam, mu, rho, h_lag):
    """((ax~(z), az~(z), d~(z)) of B1, the same of B2) of the layered elastic preconditioner:
    Eq. (22)'s K = diag(B1, B2) with each tilde taken over a node row (B1: ax = (lambda+2mu)~(z),
    az = mu~(z); B2: ax = mu~(z), az = (lambda+2mu)~(z); d = rho~(z) h^2/4)."""
    pz = row_midranges(np.asarray(lam) + 2.0 * np.asarray(mu))
    mz = row_midranges(mu)
    dz = row_midranges(rho) * h_lag ** 2 / 4.0
    return (pz, mz, dz), (mz.copy(), pz.copy(), dz.copy())


def _z_faces(az_z, free_surface):
    nz = az_z.shape[0]
    f = np.empty(nz + 1)
    f[1:nz] = 0.5 * (az_z[:-1] + az_z[1:])
    f[0] = 0.0 if free_surface else az_z[0]
    f[nz] = az_z[nz - 1]
    return f


def apply_inverse_layered(r, hx, hz, ax_z, az_z, d_z, free_surface=False):
    """y = (-B)^{-1} r for the layered preconditioner; r [..., nz, nx]."""
    r = np.asarray(r, dtype=np.float64)
    nz, nx = r.shape[-2:]
    ax_z, az_z, d_z = (np.asarray(v, dtype=np.float64) for v in (ax_z, az_z, d_z))
    S = _dst.dst_matrix(nx)
    rh = _dst.dst_x(r, S)
    lam = _dst.laplace_eigenvalues(nx, hx)
    f = _z_faces(az_z, free_surface)
    extra = (1,) * (r.ndim - 2)
    sub = (-f[:nz] / hz ** 2).reshape((nz,) + extra + (1,))
    sup = (-f[1:] / hz ** 2).reshape((nz,) + extra + (1,))
    diag = ((f[:nz] + f[1:]) / hz ** 2)[:, None] + ax_z[:, None] * lam[None, :] + d_z[:, None]
    diag = diag.reshape((nz,) + extra + (nx,))
    col = np.moveaxis(rh, -2, 0)
    yt = thomas(sub, diag, sup, col)
    return _dst.dst_x(np.moveaxis(yt, 0, -2), S)


def apply_separable_layered(y, hx, hz, ax_z, az_z, d_z, free_surface=False):
    """The layered operator itself as a 5-point stencil (used to pin apply_inverse_layered):
    -ax~(z) D_xx y - D_z(az_f D_z y) + d~(z) y, Dirichlet (free surface: no flux on top)."""
    y = np.asarray(y, dtype=np.float64)
    nz = y.shape[-2]
    ax_z, az_z, d_z = (np.asarray(v, dtype=np.float64) for v in (ax_z, az_z, d_z))
    pad = [(0, 0)] * (y.ndim - 2) + [(1, 1), (1, 1)]
    yp = np.pad(y, pad)
    c = yp[..., 1:-1, 1:-1]
    dxx = (yp[..., 1:-1, 2:] - 2 * c + yp[..., 1:-1, :-2]) / hx ** 2
    f = _z_faces(az_z, free_surface)
    south, north = yp[..., 2:, 1:-1], yp[..., :-2, 1:-1]
    flux = (f[1:, None] * (south - c) - f[:nz, None] * (c - north)) / hz ** 2
    return -ax_z[:, None] * dxx - flux + d_z[:, None] * c
