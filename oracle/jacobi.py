"""Cyclic Jacobi eigensolver in FP64, a cross-check of LAPACK's eigh.

Each plane rotation J(p, q, theta) is chosen so that (J^T A J)_pq = 0:
with zeta = (a_qq - a_pp) / (2 a_pq) the tangent t = tan(theta) is the
smaller root of t^2 + 2 zeta t - 1 = 0.  Sweeps visit every (p, q), p < q,
in row order until the off-diagonal Frobenius norm falls below
tol * ||A||_F.  The accumulated product of rotations is the eigenvector
matrix.  Pure Python loops: meant for the small k x k matrices of the LETKF.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eigh(A, tol=1e-15, max_sweeps=60):
    """Eigenvalues (ascending) and eigenvectors of a symmetric matrix."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    norm = math.sqrt(float(np.sum(A * A))) or 1.0
    for _ in range(max_sweeps):
        off = math.sqrt(2.0 * float(np.sum(np.triu(A, 1) ** 2)))
        if off <= tol * norm:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                zeta = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(zeta * zeta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                J = np.array([[c, s], [-s, c]])
                idx = [p, q]
                A[:, idx] = A[:, idx] @ J
                A[idx, :] = J.T @ A[idx, :]
                A[p, q] = A[q, p] = 0.0
                V[:, idx] = V[:, idx] @ J
    lam = np.diag(A).copy()
    order = np.argsort(lam)
    return lam[order], V[:, order]
