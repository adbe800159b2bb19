"""2.5D axisymmetric elastic problem in cylindrical coordinates (r, z) (oracle).

Test infrastructure only: imported by tests, the smoke check and the benchmark's CPU legs, never
by the library.

Sec. 2.2 (Eq. 10-12): displacements W = (u_r, u_z) = (Q, U), Lame coefficients lambda, mu and
density rho depending on (r, z); after the Laguerre transform every harmonic solves
    div sigma(R_m) - rho h^2/4 R_m = -F f_m + rho h^2 c_m sum_k (m-k) c^_k R_k,
with sigma the axisymmetric stress: sigma_rr = (l+2m) Q_r + l (Q/r + U_z), sigma_tt =
(l+2m) Q/r + l (Q_r + U_z), sigma_zz = (l+2m) U_z + l (Q_r + Q/r), sigma_rz = m (Q_z + U_r), and
div sigma = (d_r sigma_rr + d_z sigma_rz + (sigma_rr - sigma_tt)/r,
             d_r sigma_rz + d_z sigma_zz + sigma_rz / r).
The paper states the scheme only as a "finite-volume method with second order of accuracy" and
prints a free-surface condition with Q and U swapped (Sec. 2.2).  Readings:
  E1  the scheme is the gradient of a discrete strain energy, so C is symmetric by construction:
        E = 1/2 sum r [ (l+2m)(e_rr^2 + e_tt^2 + e_zz^2) + 2 l (e_rr e_tt + e_rr e_zz + e_tt e_zz)
                        + m (Q_z + U_r)^2 ] dr dz,
      each term sampled where its factors live on the cell-centred mesh of the acoustic problem
      (r_i = (i + 1/2) hr, z_k = (k + 1/2) hz, arrays [nr][nz]):
        r-faces (i+1/2, k), weight rbar = (i+1) hr: (l+2m) e_rr^2, m U_r^2, 2 l e_rr <e_tt>_r;
        z-faces (i, k+1/2), weight r_i:              (l+2m) e_zz^2, m Q_z^2, 2 l e_zz <e_tt>_z;
        nodes (i, k), weight r_i:                    (l+2m) e_tt^2, e_tt = Q / r;
        corners (i+1/2, k+1/2), weight rbar:          2 l <e_rr> <e_zz>, 2 m <Q_z> <U_r>;
      with <.> the mean of the two (corners: two) neighbouring values and face / corner
      coefficients the mean of the nodes around them.  The mass term is r rho h^2/4 at nodes.
  E2  boundaries: Q = U = 0 on the ghost nodes beyond the last radius (r = l1); the axis carries
      no energy (rbar = 0 there); the faces z = 0 and z = nz hz carry none either: the traction-
      free surface sigma_zz = sigma_rz = 0 is the natural condition of the energy (the paper's
      Eq. for sigma_zz with Q and U put back in place), and the auxiliary bottom is free as well.
  E3  the source: a vertical point force on the axis, F = e_z delta(r) delta(z - d) / (2 pi r) per
      unit volume (rho F read as the force density, as in the Cartesian elastic source): the
      r-weighted U-equation gets f_m / (2 pi hr hz) at the node (0, k_d); history r rho h^2.
  E4  preconditioner (Eq. 22 with the paper's coefficients): K = diag(B1, B2), B1 with
      a1 = rbar (l+2m)~, a2 = r m~, d = r rho~ h^2/4 + (l+2m)~ / r; B2 with a1 = rbar m~,
      a2 = r (l+2m)~, d = r rho~ h^2/4: for a homogeneous medium B2 is the U-U block of C and B1
      the Q-Q block without the 2 l e_rr <e_tt> coupling (in the continuum that term integrates
      to boundary values: l d_r(Q^2)); the e_tt^2 term gives the (l+2m)~/r of B1.  Each separates
      like the acoustic B (DCT-II along z, zero-flux faces; one tridiagonal system along r per
      z-mode).
  The scheme's local truncation error is O(h^2) except in the radial equation on the first node
  row off the axis (O(h): the half cell between the axis and that row is not sampled by the
  e_tt terms); the solution converges at O(h^2) (the point-force test).
"""
import numpy as np

from . import krylov, laguerre, precond as _pre
from .cyl import dct_matrix, mesh, neumann_eigenvalues
from .solve import elastic_lame, source_coeffs
from .tridiag import thomas


# ---------------------------------------------------------------- staggered differences (and their adjoints)
def _dr(x, hr):
    """(x[i+1] - x[i]) / hr on the r-faces i = 0..nr-1 (x = 0 on the ghost node nr)."""
    xp = np.concatenate([x, np.zeros((1,) + x.shape[1:])], axis=0)
    return (xp[1:] - xp[:-1]) / hr


def _dr_T(y, hr):
    out = -y / hr
    out[1:] += y[:-1] / hr
    return out


def _dz(x, hz):
    """(x[:, k+1] - x[:, k]) / hz on the interior z-faces k = 0..nz-2."""
    return (x[:, 1:] - x[:, :-1]) / hz


def _dz_T(y, hz, nz):
    out = np.zeros((y.shape[0], nz))
    out[:, 1:] += y / hz
    out[:, :-1] -= y / hz
    return out


def _avr(x):
    """Mean of node values across each r-face (ghost node nr = 0): [nr][...] -> [nr][...]."""
    xp = np.concatenate([x, np.zeros((1,) + x.shape[1:])], axis=0)
    return 0.5 * (xp[1:] + xp[:-1])


def _avr_T(y):
    out = 0.5 * y.copy()
    out[1:] += 0.5 * y[:-1]
    return out


def _avz(x):
    """Mean across each interior z-face: [..][nz] -> [..][nz-1]."""
    return 0.5 * (x[:, 1:] + x[:, :-1])


def _avz_T(y, nz):
    out = np.zeros((y.shape[0], nz))
    out[:, 1:] += 0.5 * y
    out[:, :-1] += 0.5 * y
    return out


def coefficients(lam, mu, hr, hz):
    """Face / node / corner coefficients of E1 (means of the nodes around each point)."""
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    nr, nz = lam.shape
    p = lam + 2.0 * mu

    def rface(f):  # [nr][nz]: faces i+1/2; the ghost face takes its node's value
        fp = np.concatenate([f, f[-1:]], axis=0)
        return 0.5 * (fp[1:] + fp[:-1])

    def zface(f):  # [nr][nz-1]
        return 0.5 * (f[:, 1:] + f[:, :-1])

    def corner(f):  # [nr][nz-1]: the four nodes (two of them ghost-side copies at the last radius)
        return zface(rface(f))

    r, _ = mesh(nr, nz, hr, hz)
    rbar = (np.arange(nr) + 1.0) * hr
    return dict(p_r=rface(p), m_r=rface(mu), l_r=rface(lam), p_z=zface(p), m_z=zface(mu), l_z=zface(lam),
                p_n=p, l_c=corner(lam), m_c=corner(mu), r=r, rbar=rbar)


def apply_C(Q, U, co, rho, h, hr, hz):
    """(C [Q; U]) per unit area: the gradient of E (E1) divided by hr hz, plus r rho h^2/4 [Q; U].
    Q, U: [nr][nz].  Returns (cQ, cU)."""
    Q = np.asarray(Q, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    nr, nz = Q.shape
    r = co["r"][:, None]
    rb = co["rbar"][:, None]
    # strains at their points
    err = _dr(Q, hr)                 # r-faces
    urr = _dr(U, hr)                 # r-faces: U_r
    ett_n = Q / r                    # nodes
    ett_r = _avr(Q / r)              # r-faces
    ezz = _dz(U, hz)                 # z-faces
    qzz = _dz(Q, hz)                 # z-faces: Q_z
    ett_z = _avz(Q / r)              # z-faces
    err_c = _avz(err)                # corners
    ezz_c = _avr(ezz)                # corners (ghost node: U = 0 so its z-face difference is 0)
    qz_c = _avr(qzz)                 # corners
    ur_c = _avz(urr)                 # corners
    # dE/d(strain) at each point (weights: rbar on r-faces and corners, r on z-faces and nodes)
    gQ = np.zeros_like(Q)
    gU = np.zeros_like(U)
    # r-faces: (l+2m) e_rr^2 + m U_r^2 + 2 l e_rr <e_tt>_r
    s_rr = rb * (co["p_r"] * err + co["l_r"] * ett_r)
    s_tt = rb * (co["l_r"] * err)
    s_ur = rb * (co["m_r"] * urr)
    gQ += _dr_T(s_rr, hr) + _avr_T(s_tt) / r
    gU += _dr_T(s_ur, hr)
    # z-faces: (l+2m) e_zz^2 + m Q_z^2 + 2 l e_zz <e_tt>_z
    s_zz = r * (co["p_z"] * ezz + co["l_z"] * ett_z)
    s_tz = r * (co["l_z"] * ezz)
    s_qz = r * (co["m_z"] * qzz)
    gU += _dz_T(s_zz, hz, nz)
    gQ += _avz_T(s_tz, nz) / r + _dz_T(s_qz, hz, nz)
    # nodes: (l+2m) e_tt^2
    gQ += r * co["p_n"] * ett_n / r
    # corners: 2 l <e_rr> <e_zz> + 2 m <Q_z> <U_r>
    c_rz = rb * co["l_c"]
    c_qu = rb * co["m_c"]
    gQ += _dr_T(_avz_T(c_rz * ezz_c, nz), hr)
    gU += _dz_T(_avr_T(c_rz * err_c), hz, nz)
    gQ += _dz_T(_avr_T(c_qu * ur_c), hz, nz)
    gU += _dr_T(_avz_T(c_qu * qz_c, nz), hr)
    w = r * rho * h ** 2 / 4.0
    return gQ + w * Q, gU + w * U


def assemble_C(co, rho, h, hr, hz):
    """Dense matrix of apply_C on [Q; U] (small grids only)."""
    nr, nz = rho.shape
    n = nr * nz
    M = np.empty((2 * n, 2 * n))
    for j in range(2 * n):
        e = np.zeros(2 * n)
        e[j] = 1.0
        cq, cu = apply_C(e[:n].reshape(nr, nz), e[n:].reshape(nr, nz), co, rho, h, hr, hz)
        M[:, j] = np.concatenate([cq.ravel(), cu.ravel()])
    return M


def precond_params(lam, mu, rho, h):
    """(B1, B2) coefficients (ax, az, d, hoop) of E4: whole-medium midranges."""
    pt = _pre.midrange(np.asarray(lam) + 2.0 * np.asarray(mu))
    mt = _pre.midrange(mu)
    dt = _pre.midrange(rho) * h ** 2 / 4.0
    return (pt, mt, dt, pt), (mt, pt, dt, 0.0)


def apply_inverse_block(rhs, hr, hz, ax, az, d, hoop):
    """B^{-1} rhs for one block: rows of the r-system for z-mode q
        (-ax i/hr, ax (2i+1)/hr + r_i az mu_q + r_i d + hoop / r_i, -ax (i+1)/hr)."""
    rhs = np.asarray(rhs, dtype=np.float64)
    nr, nz = rhs.shape[-2:]
    V = dct_matrix(nz)
    mu_q = neumann_eigenvalues(nz, hz)
    r, _ = mesh(nr, nz, hr, hz)
    i = np.arange(nr)
    sub = (-ax * i / hr)[:, None]
    sup = (-ax * (i + 1) / hr)[:, None]
    diag = (ax * (2 * i + 1) / hr + r * d + hoop / r)[:, None] + (r * az)[:, None] * mu_q[None, :]
    yh = rhs @ V
    return thomas(sub, diag, sup, yh) @ V.T


def elastic_shot(vp, vs, rho, hr, hz, h, alpha, n_harm, src, rcv, t_out, f0, t0,
                 tol=1e-10, restart=20, max_iter=4000, keep_fields=False, fm=None, wavelet="ricker"):
    """One axisymmetric elastic shot, vertical point force at (0, src[1]) on the axis.
    vp, vs, rho: [nr][nz]; rcv = [(ir, iz), ...].  Returns dict(R_rcv [n, 2, nrcv], traces
    [2, nrcv, nt] (component 0 = Q = u_r, 1 = U = u_z), iters [n], fm, fields (optional))."""
    lam, mu = elastic_lame(vp, vs, rho)
    rho = np.asarray(rho, dtype=np.float64)
    nr, nz = lam.shape
    n = nr * nz
    co = coefficients(lam, mu, hr, hz)
    r, _ = mesh(nr, nz, hr, hz)
    p1, p2 = precond_params(lam, mu, rho, h)
    if fm is None:
        fm = source_coeffs(n_harm, h, alpha, f0, t0, kind=wavelet)

    def C(v):
        cq, cu = apply_C(v[:n].reshape(nr, nz), v[n:].reshape(nr, nz), co, rho, h, hr, hz)
        return np.concatenate([cq.ravel(), cu.ravel()])

    def Kinv(v):
        yq = apply_inverse_block(v[:n].reshape(nr, nz), hr, hz, *p1)
        yu = apply_inverse_block(v[n:].reshape(nr, nz), hr, hz, *p2)
        return np.concatenate([yq.ravel(), yu.ravel()])

    rrho = r[:, None] * rho                       # E3: the history term carries r
    R, iters = [], []
    for m in range(n_harm):
        b = np.zeros((2, nr, nz))
        if m > 0:
            b -= rrho * h ** 2 * float(laguerre.c_m(m, alpha)) * laguerre.history_direct(R, m, alpha)
        b[1, src[0], src[1]] += fm[m] / (2.0 * np.pi * hr * hz)
        x, it, _ = krylov.gmres(C, Kinv, b.ravel(), restart, tol, max_iter)
        R.append(x.reshape(2, nr, nz))
        iters.append(it)
    R_rcv = np.array([[[Rm[comp, ir, iz] for (ir, iz) in rcv] for comp in range(2)] for Rm in R])
    traces = np.stack([laguerre.inverse_sum(R_rcv[:, comp, :], t_out, h, alpha).T for comp in range(2)])
    out = dict(R_rcv=R_rcv, traces=traces, iters=np.array(iters), fm=np.asarray(fm))
    if keep_fields:
        out["fields"] = np.array(R)
    return out
