"""2.5D axisymmetric acoustic problem in cylindrical coordinates (r, z) (oracle).

Test infrastructure only: imported by tests, the smoke check and the benchmark's CPU legs, never
by the library.

Sec. 2.1 (Eqs. 1-5): rho u_tt = div(kappa grad u) + f(t) delta(x - x0) / (2 pi r) in the half
plane r >= 0, z >= 0, zero initial data, du/dz = 0 at z = 0 (free surface) and z = l2,
u = 0 at r = l1, du/dr = 0 on the axis.  After the Laguerre transform (Eq. 9) every harmonic is
    div(kappa grad R_m) - rho h^2/4 R_m = -f_m delta / (2 pi r) + rho h^2 c_m sum_k (m-k) c^_k R_k.
Sec. 2.3 (Eqs. 17-19) discretises the equation multiplied by r on the cell-centred mesh
r_i = (i - 1/2) hr, z_k = (k - 1/2) hz (1-based), with the coefficients
    a1 = rbar kappa(rbar, z)   (faces between r nodes, rbar = r + hr/2),
    a2 = r kappa(r, zbar)      (faces between z nodes),
    w  = r rho h^2 / 4.
Arrays here are [nr][nz] (the paper's (i, k) order; z fastest) with 0-based indices:
r_i = (i + 1/2) hr, z_k = (k + 1/2) hz.

Readings (where the paper is silent or garbled):
  C1  kappa on a face: mean of the two nodes it joins (as R2 of the Cartesian scheme); the outer
      r face takes its node's value.
  C2  boundaries: the axis is the face rbar = 0, where a1 = 0 (Eq. 5 needs nothing more); the top
      face z = 0 carries no flux (free surface, Eq. 3); the auxiliary bottom boundary z = l2 is a
      zero-flux face as well, half a cell below the last node (the paper puts its last node on
      l2 and prints a one-sided difference there whose sign and factor do not fit a Neumann
      condition; the boundary is artificial and only placed far enough away); u = 0 on the ghost
      node r = (nr + 1/2) hr = l1.
  C3  every term of the scheme carries the factor r, the history term of phi included (Eq. 19
      prints w with r but phi's history sum without it: read as a slip, the scheme being the
      r-weighted equation).
  C4  the source at node (i0, k0): the r-weighted equation's right-hand side there is
      f_m / (2 pi hr hz), the cell's share of int r delta(x - x0) / (2 pi r) dr dz = 1 / (2 pi).
  C5  preconditioner B (Eq. 21 with the paper's cylindrical coefficients a1 = rbar kappa~,
      a2 = r kappa~, d = r rho~ h^2/4): the operator of a homogeneous medium (kappa~, rho~).  It
      separates: along z the zero-flux second difference is diagonalised by the orthonormal
      DCT-II, V[k][q] = c_q cos(pi q (k + 1/2) / nz), eigenvalues mu_q = (4/hz^2) sin^2(pi q /
      (2 nz)); for each z-mode q one general tridiagonal system along r remains:
          -kappa~ i/hr y_{i-1} + (kappa~ (2i+1)/hr + r_i kappa~ mu_q + r_i d~) y_i
              - kappa~ (i+1)/hr y_{i+1}.
"""
import numpy as np

from . import krylov, laguerre, precond as _pre
from .fd import kappa_from_velocity
from .solve import source_coeffs
from .tridiag import thomas


def mesh(nr, nz, hr, hz):
    """Node coordinates r [nr], z [nz] (C2: the axis and the surface are faces)."""
    return (np.arange(nr) + 0.5) * hr, (np.arange(nz) + 0.5) * hz


def face_mean(f, axis):
    """Mean of neighbouring node values along `axis` (C1): shape n-1 along that axis."""
    f = np.moveaxis(np.asarray(f, dtype=np.float64), axis, 0)
    return np.moveaxis(0.5 * (f[:-1] + f[1:]), 0, axis)


def coefficients(kappa, rho, hr, hz, h):
    """(a1 [nr+1][nz], a2 [nr][nz+1], w [nr][nz]) of the r-weighted scheme (Eq. 19; C1-C3).
    a1[i] is the face between r nodes i-1 and i (a1[0] on the axis, a1[nr] at the ghost node),
    a2[:, k] the face between z nodes k-1 and k (a2[:, 0] the surface, a2[:, nz] the bottom)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    nr, nz = kappa.shape
    r, _ = mesh(nr, nz, hr, hz)
    rbar = np.arange(nr + 1) * hr                     # face radii: 0, hr, ..., nr hr
    kf = np.empty((nr + 1, nz))
    kf[0] = 0.0                                       # irrelevant: rbar = 0
    kf[1:nr] = face_mean(kappa, 0)
    kf[nr] = kappa[nr - 1]
    a1 = rbar[:, None] * kf
    a2 = np.zeros((nr, nz + 1))
    a2[:, 1:nz] = r[:, None] * face_mean(kappa, 1)
    w = r[:, None] * rho * h ** 2 / 4.0
    return a1, a2, w


def apply_A(y, a1, a2, w, hr, hz):
    """(A y)_{ik} = -[a1_{i+1}(y_{i+1}-y_i) - a1_i(y_i-y_{i-1})]/hr^2
                    -[a2_{k+1}(y_{k+1}-y_k) - a2_k(y_k-y_{k-1})]/hz^2 + w y   (SPD, Eqs. 17-19),
    y [..., nr, nz]; y = 0 on the ghost node beyond the last r node."""
    y = np.asarray(y, dtype=np.float64)
    pad = [(0, 0)] * (y.ndim - 2) + [(1, 1), (1, 1)]
    yp = np.pad(y, pad)
    c = yp[..., 1:-1, 1:-1]
    fr = a1 * (yp[..., 1:, 1:-1] - yp[..., :-1, 1:-1])     # flux across r faces 0..nr  [nr+1][nz]
    fz = a2 * (yp[..., 1:-1, 1:] - yp[..., 1:-1, :-1])     # flux across z faces 0..nz  [nr][nz+1]
    return -(fr[..., 1:, :] - fr[..., :-1, :]) / hr ** 2 - (fz[..., :, 1:] - fz[..., :, :-1]) / hz ** 2 + w * c


def assemble_A(a1, a2, w, hr, hz):
    """Dense matrix of apply_A (column by column; small grids only)."""
    nr, nz = w.shape
    n = nr * nz
    M = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = apply_A(e.reshape(nr, nz), a1, a2, w, hr, hz).ravel()
    return M


def dct_matrix(n):
    """Orthonormal DCT-II basis V[k][q] = c_q cos(pi q (k + 1/2) / n) (columns: z-modes), by its
    definition.  The integer product q (2k + 1) is reduced modulo 4n before the cosine, so that
    the angle pi q (2k + 1) / (2n) is exact to one rounding (the cosine is 2 pi-periodic)."""
    k = np.arange(n, dtype=np.int64)[:, None]
    q = np.arange(n, dtype=np.int64)[None, :]
    m = (q * (2 * k + 1)) % (4 * n)
    V = np.sqrt(2.0 / n) * np.cos(np.pi * m.astype(np.float64) / (2.0 * n))
    V[:, 0] = np.sqrt(1.0 / n)
    return V


def neumann_eigenvalues(n, hz):
    """mu_q = (4 / hz^2) sin^2(pi q / (2 n)) of the zero-flux second difference (C5)."""
    return 4.0 / hz ** 2 * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2


def precond_params(kappa, rho, h):
    """(kappa~, d~ = rho~ h^2 / 4): whole-medium midranges (footnote to Eq. 21)."""
    return _pre.midrange(kappa), _pre.midrange(rho) * h ** 2 / 4.0


def apply_inverse(rhs, hr, hz, kt, dt):
    """y = B^{-1} rhs for rhs [..., nr, nz] (C5): DCT-II along z, one tridiagonal system along r
    per z-mode (Thomas), inverse DCT."""
    rhs = np.asarray(rhs, dtype=np.float64)
    nr, nz = rhs.shape[-2:]
    V = dct_matrix(nz)
    mu = neumann_eigenvalues(nz, hz)
    r, _ = mesh(nr, nz, hr, hz)
    i = np.arange(nr)
    extra = (1,) * (rhs.ndim - 2)
    sub = (-kt * i / hr).reshape((nr,) + extra + (1,))
    sup = (-kt * (i + 1) / hr).reshape((nr,) + extra + (1,))
    diag = (kt * (2 * i + 1) / hr)[:, None] + (r * kt)[:, None] * mu[None, :] + (r * dt)[:, None]
    diag = diag.reshape((nr,) + extra + (nz,))
    yh = rhs @ V                                            # z-modes
    col = np.moveaxis(yh, -2, 0)                            # r first: one system per (batch, mode)
    yt = thomas(sub, diag, sup, col)
    return np.moveaxis(yt, 0, -2) @ V.T


# Radial variant (a design extension beyond the paper, the counterpart of the Cartesian layered
# preconditioner): kappa~(r), rho~(r), each the midrange over the depths of one radius.  The
# coefficients stay independent of z, so the DCT-II along z still separates the variables; the
# r-systems take a1 = rbar kappa~_face(r) (face mean of the two radii, the outer face its node's
# value), a2 = r kappa~(r), d = r rho~(r) h^2/4.  For a medium that varies with r only, B is A.
def precond_params_radial(kappa, rho, h):
    """(kappa~(r), d~(r) = rho~(r) h^2 / 4), shapes [nr]: per-radius midranges over z."""
    kappa = np.asarray(kappa, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    kr = 0.5 * (kappa.min(axis=1) + kappa.max(axis=1))
    dr = 0.5 * (rho.min(axis=1) + rho.max(axis=1)) * h ** 2 / 4.0
    return kr, dr


def apply_inverse_radial(rhs, hr, hz, kr, dr, kz=None):
    """y = B^{-1} rhs for the radial preconditioner; rhs [..., nr, nz].  kr(r) gives the r faces
    (a1 = rbar kr_face), kz(r) the z part (a2 = r kz; kz = kr when omitted, as Eq. 21 has one
    kappa~), dr(r) the mass term (d = r dr)."""
    rhs = np.asarray(rhs, dtype=np.float64)
    nr, nz = rhs.shape[-2:]
    kr = np.asarray(kr, dtype=np.float64)
    dr = np.asarray(dr, dtype=np.float64)
    kz = kr if kz is None else np.asarray(kz, dtype=np.float64)
    V = dct_matrix(nz)
    mu = neumann_eigenvalues(nz, hz)
    r, _ = mesh(nr, nz, hr, hz)
    kf = np.empty(nr + 1)                                   # face values; the axis face has rbar = 0
    kf[0] = 0.0
    kf[1:nr] = 0.5 * (kr[:-1] + kr[1:])
    kf[nr] = kr[nr - 1]
    a1 = np.arange(nr + 1) * hr * kf / hr ** 2               # rbar kappa~_face / hr^2
    extra = (1,) * (rhs.ndim - 2)
    sub = (-a1[:nr]).reshape((nr,) + extra + (1,))
    sup = (-a1[1:]).reshape((nr,) + extra + (1,))
    diag = (a1[:nr] + a1[1:])[:, None] + (r * kz)[:, None] * mu[None, :] + (r * dr)[:, None]
    diag = diag.reshape((nr,) + extra + (nz,))
    yh = rhs @ V
    col = np.moveaxis(yh, -2, 0)
    yt = thomas(sub, diag, sup, col)
    return np.moveaxis(yt, 0, -2) @ V.T


def acoustic_shot(c, rho, hr, hz, h, alpha, n_harm, src, rcv, t_out, f0, t0,
                  tol=1e-10, max_iter=2000, keep_fields=False, fm=None, wavelet="ricker", radial=False):
    """One axisymmetric acoustic shot.  c, rho: [nr, nz]; src = (ir, iz); rcv = [(ir, iz), ...].

    Returns dict(R_rcv [n, nrcv], traces [nrcv, nt], iters [n], fm [n], fields (optional))."""
    c = np.asarray(c, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    nr, nz = c.shape
    kappa = kappa_from_velocity(c, rho)
    a1, a2, w = coefficients(kappa, rho, hr, hz, h)
    r, _ = mesh(nr, nz, hr, hz)
    rrho = r[:, None] * rho                                 # C3: the history term carries r
    if radial:
        kt, dt = precond_params_radial(kappa, rho, h)
        inv = apply_inverse_radial
    else:
        kt, dt = precond_params(kappa, rho, h)
        inv = apply_inverse
    if fm is None:
        fm = source_coeffs(n_harm, h, alpha, f0, t0, kind=wavelet)

    def A(v):
        return apply_A(v.reshape(nr, nz), a1, a2, w, hr, hz).ravel()

    def Minv(v):
        return inv(v.reshape(nr, nz), hr, hz, kt, dt).ravel()

    R, iters = [], []
    for m in range(n_harm):
        b = np.zeros((nr, nz))
        if m > 0:
            b -= rrho * h ** 2 * float(laguerre.c_m(m, alpha)) * laguerre.history_direct(R, m, alpha)
        b[src[0], src[1]] += fm[m] / (2.0 * np.pi * hr * hz)  # C4
        x, it, _ = krylov.pcg(A, Minv, b.ravel(), tol, max_iter)
        R.append(x.reshape(nr, nz))
        iters.append(it)
    R_rcv = np.array([[Rm[ir, iz] for (ir, iz) in rcv] for Rm in R]).reshape(n_harm, len(rcv))
    traces = laguerre.inverse_sum(R_rcv, t_out, h, alpha).T
    out = dict(R_rcv=R_rcv, traces=traces, iters=np.array(iters), fm=np.asarray(fm))
    if keep_fields:
        out["fields"] = np.array(R)
    return out
