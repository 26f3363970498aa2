"""Brute-force model-space Kalman filter in FP64 (Sec. II-B, Eqs. kfx, kfp, kfk).

    K   = Pf H^T (H Pf H^T + R)^-1
    x^a = x^f + K (yo - H x^f)
    P^a = (I - K H) Pf

with the ensemble estimate of the covariance (Eq. enkf_p)
Pf = dX dX^T / (k - 1).  With a linear H and no localization, the
ensemble-space analysis must reproduce these exactly; this is the
independent pin of ``oracle.letkf``.
"""
from __future__ import annotations

import numpy as np


def ensemble_covariance(X):
    """Pf = dX dX^T / (k - 1) for members in the columns of X [n, k] (Eq. enkf_p)."""
    X = np.asarray(X, dtype=np.float64)
    dX = X - X.mean(axis=1, keepdims=True)
    return dX @ dX.T / (X.shape[1] - 1)


def kalman_gain(Pf, H, R):
    """K = Pf H^T (H Pf H^T + R)^-1 (Eq. kfk), via a linear solve."""
    S = H @ Pf @ H.T + R
    return np.linalg.solve(S.T, (Pf @ H.T).T).T


def kalman_analysis(xf, Pf, H, R, yo):
    """(x^a, P^a, K) from Eqs. kfx, kfp, kfk."""
    K = kalman_gain(Pf, H, R)
    xa = xf + K @ (yo - H @ xf)
    Pa = (np.eye(Pf.shape[0]) - K @ H) @ Pf
    return xa, Pa, K
