"""Krylov solvers (oracle).  Test infrastructure only.

Sec. 2.3: the acoustic system A y = phi (A = A* > 0) is solved by conjugate gradients and
the elastic system C y = f by restarted GMRES(k); both are preconditioned (Sec. 2.4).  The
paper is silent on the initial guess, the residual norm and the CG beta variant.  Readings:
zero initial guess; stop when ||r||_2 / ||b||_2 <= tol on the unpreconditioned residual;
Fletcher-Reeves beta for CG; right preconditioning, modified Gram-Schmidt and Givens
rotations for GMRES(k).  Vectors are flat float64 arrays; the operators are callables.
"""
import numpy as np


def pcg(apply_A, apply_Minv, b, tol, max_iter=2000):
    """Preconditioned conjugate gradients.  Returns (x, iterations, relative residuals).

    Iteration i: q = A p; alpha = (r,z)/(p,q); x += alpha p; r -= alpha q; stop on the
    recursive residual; z = M^{-1} r; beta = (r,z)_new/(r,z)_old; p = z + beta p."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    r = b.copy()
    z = apply_Minv(r)
    p = z.copy()
    rz = float(np.dot(r, z))
    hist = [1.0]
    it = 0
    while it < max_iter:
        it += 1
        q = apply_A(p)
        alpha = rz / float(np.dot(p, q))
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= tol:
            break
        z = apply_Minv(r)
        rz_new = float(np.dot(r, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist


def gmres(apply_C, apply_Kinv, b, k, tol, max_iter=4000):
    """Restarted, right-preconditioned GMRES(k) with modified Gram-Schmidt and Givens
    rotations.  Returns (x, inner iterations, relative residual estimates)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    r = b - apply_C(x)
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    total = 0
    while beta / bnorm > tol and total < max_iter:
        V = [r / beta]
        Z = []
        H = np.zeros((k + 1, k))
        cs = np.zeros(k)
        sn = np.zeros(k)
        g = np.zeros(k + 1)
        g[0] = beta
        j_done = 0
        for j in range(k):
            zj = apply_Kinv(V[j])
            Z.append(zj)
            w = apply_C(zj)
            for i in range(j + 1):              # modified Gram-Schmidt
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            hnext = float(np.linalg.norm(w))
            H[j + 1, j] = hnext
            for i in range(j):                  # previous rotations on column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or hnext == 0.0 or total >= max_iter:
                break
            V.append(w / hnext)
        # back substitution on the rotated (upper-triangular) Hessenberg block
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_done], y[i + 1:j_done])) / H[i, i]
        for i in range(j_done):
            x += y[i] * Z[i]
        r = b - apply_C(x)
        beta = np.linalg.norm(r)
        if beta == 0.0:
            break
    return x, total, hist
