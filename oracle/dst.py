"""Orthonormal DST-I along x (oracle).  Test infrastructure only.

Sec. 2.4 inverts the Laplace preconditioner by separation of variables: a fast transform
along the direction where the coefficients are constant (the paper uses FFTW), then one
tridiagonal system per mode.  With Dirichlet ends on the node-centred grid the transform is
the DST-I.  Reading: orthonormal scaling, so the matrix is its own inverse,

    S[j, k] = sqrt(2/(N+1)) * sin(pi (j+1)(k+1) / (N+1)),   j, k = 0..N-1,

and the second difference with Dirichlet ends is diagonalised with eigenvalues
lambda_j = (4/hx^2) sin^2(pi (j+1) / (2(N+1))).
"""
import numpy as np


def dst_matrix(n):
    """S by its definition.  The integer product (j+1)(k+1) is reduced modulo 2(N+1) before
    the sine so that the angle is exact to one rounding (the sine is 2pi-periodic)."""
    idx = np.arange(1, n + 1, dtype=np.int64)
    prod = np.outer(idx, idx) % (2 * (n + 1))
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * prod.astype(np.float64) / (n + 1))


def dst_x(y, S=None):
    """Apply the DST-I along the last (x) axis: out[..., k] = sum_j y[..., j] S[j, k]."""
    y = np.asarray(y, dtype=np.float64)
    if S is None:
        S = dst_matrix(y.shape[-1])
    return y @ S


def laplace_eigenvalues(n, hx):
    """Eigenvalues of the Dirichlet second difference -D_xx for the DST-I modes."""
    j = np.arange(1, n + 1, dtype=np.float64)
    return (4.0 / hx ** 2) * np.sin(np.pi * j / (2.0 * (n + 1))) ** 2
