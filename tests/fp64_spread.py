"""A second, independent FP64 run of the algorithm of Section III built on
library routines (BLAS matrix products, LAPACK Cholesky, triangular solves):
how far two correct FP64 implementations drift apart as the normal matrix
grows ill-conditioned.  Used by the parity tests to state the agreement that
FP64 rounding permits; it shares no code with the oracle or the GPU path."""
import numpy as np
import scipy.linalg as sl


def lapack_trajectory(A, b, c, x, y, s, iters, alpha=0.95):
    x, y, s = x.copy(), y.copy(), s.copy()
    out = []
    for _ in range(iters):
        D = x / s
        M = (A * D) @ A.T
        L = np.linalg.cholesky(M)
        dy = sl.solve_triangular(L, sl.solve_triangular(L, A @ x, lower=True), lower=True, trans="T")
        w = A.T @ dy
        ds = -w
        dx = D * w - x
        psi = max(np.max(-dx / x), np.max(-ds / s))
        th = 1.0 if psi <= 1 else alpha / psi
        x, y, s = x + th * dx, y + th * dy, s + th * ds
        out.append((x.copy(), y.copy(), s.copy(), psi))
    return out


def iterate_spread(ref_iterates, traj, n, m):
    """Per iteration: max over x, y, s of the normwise relative distance
    between the oracle's iterate and the LAPACK run's."""
    spread = []
    for it, (x, y, s, _) in zip(ref_iterates, traj):
        e = max(np.linalg.norm(v - o) / np.linalg.norm(o)
                for v, o in ((x, it[:n]), (y, it[n:n + m]), (s, it[n + m:])))
        spread.append(e)
    return np.array(spread)
