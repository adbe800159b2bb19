"""Finite-difference operators (oracle).  Test infrastructure only.

Grid reading (the paper's cell-centred cylindrical mesh of Sec. 2.3 goes with its Neumann
boundaries; the Cartesian Dirichlet problem solved here uses a node-centred grid):
interior nodes x_i = (i+1) hx, i = 0..nx-1 and z_k = (k+1) hz, k = 0..nz-1, with u = 0 on the
ghost nodes i = -1, nx and k = -1, nz.  Arrays are indexed [k, i] (z rows, x fastest).

Acoustic operator (Sec. 2.3, Eqs. (16)-(18), Cartesian form, sign flipped to the SPD form
A = -(Lambda_x + Lambda_z) + w, cf. "A = A* > 0" below Eq. (15)):

    (A y)_{k,i} = -[ax_{k,i+1/2}(y_{k,i+1}-y_{k,i}) - ax_{k,i-1/2}(y_{k,i}-y_{k,i-1})]/hx^2
                  -[az_{k+1/2,i}(y_{k+1,i}-y_{k,i}) - az_{k-1/2,i}(y_{k,i}-y_{k-1,i})]/hz^2
                  + w_{k,i} y_{k,i},          w = rho h^2 / 4   (h: Laguerre parameter).

Reading of "kappa at the half point" (Eq. 18): the arithmetic mean of the two adjacent nodal
values; a boundary face takes the value of its interior node.

Free surface (Sec. 2.1, Eq. (3): du/dz = 0 at z = 0): ``free_surface=True`` makes the top face of
node row k = 0 carry no flux, i.e. its coefficient az_{-1/2} is zero (the zero-flux finite-volume
form of the Neumann condition on this grid); the other three sides stay Dirichlet.
"""
import numpy as np


def kappa_from_velocity(c, rho):
    """Bulk modulus kappa = rho c^2 (Sec. 3.2: the exact solution travels at sqrt(kappa/rho))."""
    return np.asarray(rho, dtype=np.float64) * np.asarray(c, dtype=np.float64) ** 2


def face_x(coef):
    """Coefficient on the nx+1 x-faces of each row: face f lies between nodes f-1 and f.

    Returns an array [nz, nx+1]; interior faces hold the mean of their two nodes, the two
    boundary faces the value of the adjacent interior node."""
    coef = np.asarray(coef, dtype=np.float64)
    nz, nx = coef.shape
    out = np.empty((nz, nx + 1))
    out[:, 1:nx] = 0.5 * (coef[:, :-1] + coef[:, 1:])
    out[:, 0] = coef[:, 0]
    out[:, nx] = coef[:, nx - 1]
    return out


def face_z(coef, free_surface=False):
    """Coefficient on the nz+1 z-faces of each column ([nz+1, nx]), same rule as face_x; with a
    free surface the top face (above row 0) carries zero."""
    out = face_x(np.asarray(coef, dtype=np.float64).T).T
    if free_surface:
        out[0, :] = 0.0
    return out


def _pad(y):
    """Embed y [..., nz, nx] in a zero Dirichlet frame [..., nz+2, nx+2]."""
    y = np.asarray(y, dtype=np.float64)
    pad = [(0, 0)] * (y.ndim - 2) + [(1, 1), (1, 1)]
    return np.pad(y, pad)


def apply_A(y, kappa, rho, h_lag, hx, hz, free_surface=False):
    """Acoustic operator A y (Eqs. 16-18, Cartesian SPD form).  y: [..., nz, nx]."""
    kappa = np.asarray(kappa, dtype=np.float64)
    ax = face_x(kappa)   # [nz, nx+1]
    az = face_z(kappa, free_surface)   # [nz+1, nx]
    w = np.asarray(rho, dtype=np.float64) * h_lag ** 2 / 4.0
    yp = _pad(y)
    c = yp[..., 1:-1, 1:-1]
    east, west = yp[..., 1:-1, 2:], yp[..., 1:-1, :-2]
    south, north = yp[..., 2:, 1:-1], yp[..., :-2, 1:-1]
    lap_x = (ax[:, 1:] * (east - c) - ax[:, :-1] * (c - west)) / hx ** 2
    lap_z = (az[1:, :] * (south - c) - az[:-1, :] * (c - north)) / hz ** 2
    return -(lap_x + lap_z) + w * c


def assemble_A(kappa, rho, h_lag, hx, hz, free_surface=False):
    """Dense matrix of A (tiny grids only), unknown index k*nx + i.  Built entry by entry
    from the stencil written out, independently of ``apply_A``."""
    kappa = np.asarray(kappa, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    nz, nx = kappa.shape
    n = nz * nx
    M = np.zeros((n, n))

    def kx(k, f):  # x-face f of row k (between nodes f-1 and f)
        if f == 0:
            return kappa[k, 0]
        if f == nx:
            return kappa[k, nx - 1]
        return 0.5 * (kappa[k, f - 1] + kappa[k, f])

    def kz(f, i):  # z-face f of column i
        if f == 0:
            return 0.0 if free_surface else kappa[0, i]
        if f == nz:
            return kappa[nz - 1, i]
        return 0.5 * (kappa[f - 1, i] + kappa[f, i])

    for k in range(nz):
        for i in range(nx):
            r = k * nx + i
            e, wst = kx(k, i + 1) / hx ** 2, kx(k, i) / hx ** 2
            s, nth = kz(k + 1, i) / hz ** 2, kz(k, i) / hz ** 2
            M[r, r] = e + wst + s + nth + rho[k, i] * h_lag ** 2 / 4.0
            if i + 1 < nx:
                M[r, r + 1] = -e
            if i - 1 >= 0:
                M[r, r - 1] = -wst
            if k + 1 < nz:
                M[r, r + nx] = -s
            if k - 1 >= 0:
                M[r, r - nx] = -nth
    return M


# ----------------------------------------------------------------------------------------
# Elastic operator (Sec. 2.2 Eq. (12), Sec. 2.3 Eq. (19)).
#
# Reading (the paper states only "finite-volume, second order"): Cartesian plane strain,
#   rho u_tt = d_x[(l+2m) u_x] + d_z[m u_z] + d_x[l w_z] + d_z[m w_x]
#   rho w_tt = d_x[m w_x] + d_z[(l+2m) w_z] + d_x[m u_z] + d_z[l u_x]
# (l = lambda, m = mu).  Second-derivative terms use face-averaged coefficients exactly as in
# the acoustic operator; mixed terms are centred differences with nodal coefficients, e.g.
#   d_x[l d_z w]_{k,i} = [l_{k,i+1}(w_{k+1,i+1}-w_{k-1,i+1}) - l_{k,i-1}(w_{k+1,i-1}-w_{k-1,i-1})]/(4 hx hz)
#   d_z[l d_x u]_{k,i} = [l_{k+1,i}(u_{k+1,i+1}-u_{k+1,i-1}) - l_{k-1,i}(u_{k-1,i+1}-u_{k-1,i-1})]/(4 hx hz)
# Coefficients outside the grid are never needed (they multiply Dirichlet zeros).  The SPD
# form is C = -(elastic terms) + rho h^2/4 on each component.
# ----------------------------------------------------------------------------------------

def _nodal_pad(c):
    """Pad a nodal coefficient by one with zeros (the padded values always meet a zero field)."""
    return np.pad(np.asarray(c, dtype=np.float64), ((1, 1), (1, 1)))


def apply_C(u, w, lam, mu, rho, h_lag, hx, hz):
    """Elastic operator C [u; w] (plane-strain reading of Eq. 12).  u, w: [..., nz, nx]."""
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    p = lam + 2.0 * mu
    mass = np.asarray(rho, dtype=np.float64) * h_lag ** 2 / 4.0
    px, pz = face_x(p), face_z(p)
    mx, mz = face_x(mu), face_z(mu)
    up, wp = _pad(u), _pad(w)
    lp, mp = _nodal_pad(lam), _nodal_pad(mu)

    def second(fp, cx, cz):
        c = fp[..., 1:-1, 1:-1]
        e, wst = fp[..., 1:-1, 2:], fp[..., 1:-1, :-2]
        s, n = fp[..., 2:, 1:-1], fp[..., :-2, 1:-1]
        return ((cx[:, 1:] * (e - c) - cx[:, :-1] * (c - wst)) / hx ** 2,
                (cz[1:, :] * (s - c) - cz[:-1, :] * (c - n)) / hz ** 2)

    def dx_c_dz(cp, fp):
        # d_x[c d_z f] with nodal c at columns i+-1
        ce = cp[1:-1, 2:]
        cw = cp[1:-1, :-2]
        dz_e = fp[..., 2:, 2:] - fp[..., :-2, 2:]
        dz_w = fp[..., 2:, :-2] - fp[..., :-2, :-2]
        return (ce * dz_e - cw * dz_w) / (4.0 * hx * hz)

    def dz_c_dx(cp, fp):
        # d_z[c d_x f] with nodal c at rows k+-1
        cs = cp[2:, 1:-1]
        cn = cp[:-2, 1:-1]
        dx_s = fp[..., 2:, 2:] - fp[..., 2:, :-2]
        dx_n = fp[..., :-2, 2:] - fp[..., :-2, :-2]
        return (cs * dx_s - cn * dx_n) / (4.0 * hx * hz)

    uxx, uzz = second(up, px, mz)
    wxx, wzz = second(wp, mx, pz)
    cu = -(uxx + uzz + dx_c_dz(lp, wp) + dz_c_dx(mp, wp)) + mass * up[..., 1:-1, 1:-1]
    cw = -(wxx + wzz + dx_c_dz(mp, up) + dz_c_dx(lp, up)) + mass * wp[..., 1:-1, 1:-1]
    return cu, cw


def assemble_C(lam, mu, rho, h_lag, hx, hz):
    """Dense matrix of C by columns (applying C to unit vectors); unknown order [u; w]."""
    lam = np.asarray(lam, dtype=np.float64)
    nz, nx = lam.shape
    n = nz * nx
    M = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        e = np.zeros(2 * n)
        e[j] = 1.0
        cu, cw = apply_C(e[:n].reshape(nz, nx), e[n:].reshape(nz, nx), lam, mu, rho, h_lag, hx, hz)
        M[:n, j] = cu.ravel()
        M[n:, j] = cw.ravel()
    return M
