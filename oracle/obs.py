"""Observation operator y = h(x) in FP64 (Sec. II-B).

The paper observes the macroscopic fields at observation points: "y is
given by rho and u at observation points" (Sec. II-B) and V = 3 variables
(rho, u_x, u_y) in its evaluation (Sec. V).  Observations here are the
selected subset of (rho, u_x, u_y), in that order, for each observation
point; the vector y has length L * V with index l * V + v.

The operator is nonlinear in f (u = sum c f / rho), so the ensemble form
applies h to each member: Y^f[m, :] = h(x_m) (Algorithm 1, first step).
"""
from __future__ import annotations

import numpy as np

from .lbm import moments

VAR_RHO, VAR_U, VAR_V = 1, 2, 4


def var_list(obs_vars: int):
    """Observed variables in output order for the bit mask (1 rho, 2 u, 4 v)."""
    return [v for v in (VAR_RHO, VAR_U, VAR_V) if obs_vars & v]


def observe(f, obs_xy, obs_vars: int = VAR_U | VAR_V):
    """h(x) for one or many members: f [..., 9, ny, nx] -> y [..., L * V]."""
    rho, ux, uy = moments(f)
    xs = np.asarray(obs_xy)[:, 0]
    ys = np.asarray(obs_xy)[:, 1]
    fields = {VAR_RHO: rho, VAR_U: ux, VAR_V: uy}
    cols = [fields[v][..., ys, xs] for v in var_list(obs_vars)]
    y = np.stack(cols, axis=-1)  # [..., L, V]
    return y.reshape(y.shape[:-2] + (-1,))


def ensemble_obs(Yf):
    """Obs-space ensemble mean and perturbations (Eqs. enkf_ybar, enkf_deltay).

    Yf [k, p] -> (ybar [p], dY [k, p]) with dY[m] = Yf[m] - ybar.
    """
    Yf = np.asarray(Yf, dtype=np.float64)
    ybar = Yf.mean(axis=0)
    return ybar, Yf - ybar
