"""Whole-shot Laguerre solves (oracle).  Test infrastructure only.

Sec. 2.1 (acoustic) and Sec. 2.2 (elastic): for m = 0, 1, ..., n-1 solve one elliptic problem
with the same operator and the right-hand side of Eq. (9) (Eq. (12) per displacement
component), then sum the series (Eq. 8 / Eq. 11) at the receivers.  The history sum
sum_{k<m} (m-k) c^_k R_k is evaluated exactly as printed (all R_k kept), so the oracle's cost
grows as n^2 field operations; it is meant for the small and sampled cases.

Readings (Cartesian, Dirichlet workload; see the module docstrings of fd / precond):
* discrete point source: 1/(hx hz) at the source node (the cylindrical 1/(2 pi r) factor of
  Eq. 3 does not apply in 2D Cartesian form);
* elastic: vertical point force, so only the w-equation carries delta_s f_m / (hx hz);
* lambda = rho (Vp^2 - 2 Vs^2), mu = rho Vs^2.
"""
import numpy as np

from . import fd, krylov, laguerre, precond


def source_coeffs(n, h, alpha, f0, t0, kind="ricker", gamma=4.0):
    """f_m, m < n, of the wavelet (below Eq. 9).  kind 'ricker' or 'paper' (Eq. 23)."""
    if kind == "ricker":
        fun = laguerre.ricker(f0, t0)
        t_end = t0 + 4.0 / f0
    else:
        fun = laguerre.paper_wavelet(f0, t0, gamma)
        t_end = t0 + 2.0 * gamma / f0
    return laguerre.forward_coeffs(fun, n, h, alpha, t_end)


def acoustic_shot(c, rho, hx, hz, h, alpha, n_harm, src, rcv, t_out, f0, t0,
                  tol=1e-10, max_iter=2000, keep_fields=False, fm=None, wavelet="ricker", free_surface=False,
                  layered=False):
    """One acoustic shot.  c, rho: [nz, nx]; src = (ix, iz); rcv = [(ix, iz), ...].
    layered: precondition with the per-row midranges (precond.apply_inverse_layered) instead of
    the whole-medium midranges of Eq. (21).

    Returns dict(R_rcv [n, nrcv], traces [nrcv, nt], iters [n], fm [n], fields (optional))."""
    c = np.asarray(c, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    nz, nx = c.shape
    kappa = fd.kappa_from_velocity(c, rho)
    ax_t, az_t, d_t = precond.acoustic_params(kappa, rho, h)
    if fm is None:
        fm = source_coeffs(n_harm, h, alpha, f0, t0, kind=wavelet)

    def A(v):
        return fd.apply_A(v.reshape(nz, nx), kappa, rho, h, hx, hz, free_surface).ravel()

    if layered:
        lz = precond.acoustic_params_layered(kappa, rho, h)

        def Minv(v):
            return precond.apply_inverse_layered(v.reshape(nz, nx), hx, hz, *lz, free_surface).ravel()
    else:
        def Minv(v):
            return precond.apply_inverse(v.reshape(nz, nx), hx, hz, ax_t, az_t, d_t, free_surface).ravel()

    R = []
    iters = []
    for m in range(n_harm):
        b = np.zeros((nz, nx))
        if m > 0:
            b -= rho * h ** 2 * float(laguerre.c_m(m, alpha)) * laguerre.history_direct(R, m, alpha)
        b[src[1], src[0]] += fm[m] / (hx * hz)
        x, it, _ = krylov.pcg(A, Minv, b.ravel(), tol, max_iter)
        R.append(x.reshape(nz, nx))
        iters.append(it)
    R_rcv = np.array([[Rm[iz, ix] for (ix, iz) in rcv] for Rm in R]).reshape(n_harm, len(rcv))
    traces = laguerre.inverse_sum(R_rcv, t_out, h, alpha).T
    out = dict(R_rcv=R_rcv, traces=traces, iters=np.array(iters), fm=np.asarray(fm))
    if keep_fields:
        out["fields"] = np.array(R)
    return out


def elastic_lame(vp, vs, rho):
    """(lambda, mu) from velocities and density."""
    vp = np.asarray(vp, dtype=np.float64)
    vs = np.asarray(vs, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    return rho * (vp ** 2 - 2.0 * vs ** 2), rho * vs ** 2


def elastic_shot(vp, vs, rho, hx, hz, h, alpha, n_harm, src, rcv, t_out, f0, t0,
                 tol=1e-10, restart=20, max_iter=4000, keep_fields=False, fm=None,
                 wavelet="ricker", layered=False):
    """One elastic shot with a vertical point force.  Returns dict(R_rcv [n, 2, nrcv],
    traces [2, nrcv, nt], iters [n], fm, fields (optional: [n, 2, nz, nx])).
    layered: K = diag(B1, B2) with per-row midranges (precond.elastic_params_layered)."""
    lam, mu = elastic_lame(vp, vs, rho)
    rho = np.asarray(rho, dtype=np.float64)
    nz, nx = lam.shape
    n = nz * nx
    if layered:
        p1, p2 = precond.elastic_params_layered(lam, mu, rho, h)
        inv = precond.apply_inverse_layered
    else:
        p1, p2 = precond.elastic_params(lam, mu, rho, h)
        inv = precond.apply_inverse
    if fm is None:
        fm = source_coeffs(n_harm, h, alpha, f0, t0, kind=wavelet)

    def C(v):
        cu, cw = fd.apply_C(v[:n].reshape(nz, nx), v[n:].reshape(nz, nx), lam, mu, rho, h, hx, hz)
        return np.concatenate([cu.ravel(), cw.ravel()])

    def Kinv(v):
        yu = inv(v[:n].reshape(nz, nx), hx, hz, *p1)
        yw = inv(v[n:].reshape(nz, nx), hx, hz, *p2)
        return np.concatenate([yu.ravel(), yw.ravel()])

    R = []
    iters = []
    for m in range(n_harm):
        b = np.zeros((2, nz, nx))
        if m > 0:
            b -= rho * h ** 2 * float(laguerre.c_m(m, alpha)) * laguerre.history_direct(R, m, alpha)
        b[1, src[1], src[0]] += fm[m] / (hx * hz)
        x, it, _ = krylov.gmres(C, Kinv, b.ravel(), restart, tol, max_iter)
        R.append(x.reshape(2, nz, nx))
        iters.append(it)
    R_rcv = np.array([[[Rm[comp, iz, ix] for (ix, iz) in rcv] for comp in range(2)] for Rm in R])
    traces = np.stack([laguerre.inverse_sum(R_rcv[:, comp, :], t_out, h, alpha).T for comp in range(2)])
    out = dict(R_rcv=R_rcv, traces=traces, iters=np.array(iters), fm=np.asarray(fm))
    if keep_fields:
        out["fields"] = np.array(R)
    return out
