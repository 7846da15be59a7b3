"""Tolerances of the parity tests against the CPU oracle (shared helpers).

Both the GPU path and the oracle compute A^-1 by eliminations with partial
pivoting in FP64, in different association orders. Their difference is then
a forward-error difference: for a matrix of 2-norm condition number
kappa_2 = ||A||_2 ||A^-1||_2, each side is within about c n kappa_2 u of the
exact inverse (u = 2^-53) by the worst-case analysis, and within about
c sqrt(n) kappa_2 u with high probability when rounding errors behave like
independent random variables (the probabilistic rounding-error analysis of
Higham and Mary). The tests use the latter with c = 16, normwise
(||X - X_o||_F / ||X_o||_F) and elementwise (max |X - X_o| / max |X_o|);
measured errors on these inputs sit at 0.005..0.9 of sqrt(n) kappa_2 u, the
largest for the elementwise error of diagonally dominant matrices.
kappa_2 is estimated from ||A||_2 and ||X_o||_2 by power iteration.
"""
import numpy as np

U64 = 2.0 ** -53
C_FWD = 16.0


def norm2_est(M, iters=40, seed=0):
    """||M||_2 by power iteration on M^T M from a seeded start (converges from below)."""
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal(M.shape[1])
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        v = M.T @ (M @ v)
        s = np.linalg.norm(v)
        if s == 0.0:
            return 0.0
        v /= s
    return float(np.sqrt(s))


def kappa2(A, Xo):
    return norm2_est(A) * norm2_est(Xo)


def fwd_bound(A, Xo, c=C_FWD):
    return c * np.sqrt(A.shape[0]) * kappa2(A, Xo) * U64


def eps_norm(X, Xo):
    return float(np.linalg.norm(X - Xo) / np.linalg.norm(Xo))


def eps_max(X, Xo):
    return float(np.abs(X - Xo).max() / np.abs(Xo).max())
