"""Thomas algorithm (oracle).  Test infrastructure only.

The paper solves its tridiagonal systems with the Dichotomy Algorithm (Sec. 1, Sec. 3.1),
whose body is not printed; the paper states that its result and accuracy match the
sequential elimination.  The oracle therefore solves each system by plain Gaussian
elimination without pivoting (Thomas), sweeping along axis 0.  Trailing axes hold
independent systems (numpy broadcasting over them adds no reordering along the sweep).

System: sub[k] y[k-1] + diag[k] y[k] + sup[k] y[k+1] = d[k], k = 0..n-1
(sub[0] and sup[n-1] are ignored).
"""
import numpy as np


def thomas(sub, diag, sup, d):
    """Solve along axis 0.  sub, diag, sup broadcast against d ([n, ...])."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    sub = np.broadcast_to(np.asarray(sub, dtype=np.float64), d.shape)
    diag = np.broadcast_to(np.asarray(diag, dtype=np.float64), d.shape)
    sup = np.broadcast_to(np.asarray(sup, dtype=np.float64), d.shape)
    cp = np.empty_like(d)
    dp = np.empty_like(d)
    cp[0] = sup[0] / diag[0]
    dp[0] = d[0] / diag[0]
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den if k < n - 1 else 0.0
        dp[k] = (d[k] - sub[k] * dp[k - 1]) / den
    y = np.empty_like(d)
    y[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        y[k] = dp[k] - cp[k] * y[k + 1]
    return y
