"""Plain FP64 CPU oracle for the Laguerre-transform wave solver of Fatyanov & Terekhov
("High-performance modeling acoustic and elastic waves using the Parallel Dichotomy
Algorithm", arXiv:1005.0542).

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct restatement of what the
paper's method computes, written in numpy/scipy in float64.  It exists to check the CUDA
library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The library
(``paper_1005_0542_gb300``) never imports it and shares no code with it; the only code both
sides use is the seeded input generator ``paper_1005_0542_gb300.inputs``, which holds none
of the method's arithmetic (the oracle does not import even that: it takes arrays).

Modules and what they follow (paper sections / equations):

* ``fd``        -- Sec. 2.3, Eqs. (15)-(18): conservative 5-point operator A (Cartesian reading),
                   Eq. (19) elastic operator C (plane-strain reading: the paper only says
                   "finite volume, second order"); pinned by symmetry, positivity, an O(h^2)
                   manufactured solution, and through whole elastic shots that converge at O(h^2)
                   to the plane-strain line-force solution (``analytic.line_force_2d``).
* ``dst``       -- Sec. 2.4 variable separation along x: orthonormal DST-I by its definition.
* ``tridiag``   -- Thomas algorithm (the sequential reference for the Dichotomy solve, Sec. 1).
* ``precond``   -- Sec. 2.4, Eqs. (21)-(22): Laplace preconditioner B with midrange coefficients
                   and the vector preconditioner K = diag(B1, B2).
* ``krylov``    -- Sec. 2.3: conjugate gradients (acoustic) and restarted GMRES(k) (elastic).
* ``laguerre``  -- Sec. 2.1, Eqs. (7)-(9): Laguerre functions, forward transform of the source,
                   the spectral recurrence, inverse summation.
* ``solve``     -- Sec. 2.1-2.2: whole harmonic loop for one shot (acoustic, elastic).
* ``analytic``  -- closed-form solutions used as pins (2D point source, 3D point source and point
                   force, 2D line force in plane strain, scalar oscillator).

Readings of silent / garbled passages are stated in each function's docstring.
"""
