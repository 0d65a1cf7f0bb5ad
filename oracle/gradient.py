"""Dense FP64 reference for differentiating a solve x = A^{-1} b (test infrastructure only).

For a loss L(x) with g = dL/dx:  lambda = A^{-T} g,  dL/db = lambda,  dL/dA = -lambda x^T.
Only the tests use this module.
"""
import numpy as np


def solve_grad(A, b, x_t):
    """L = 0.5 ||A^{-1} b - x_t||^2 with A dense.  Returns (x, L, dL/db, dL/dA)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.linalg.solve(A, b)
    g = x - x_t
    lam = np.linalg.solve(A.T, g)
    return x, 0.5 * float(g @ g), lam, -np.outer(lam, x)
