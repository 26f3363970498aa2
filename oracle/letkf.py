"""R-localized LETKF analysis in FP64 (Sec. II-B, Algorithm 1).

Ensemble-space analysis at one grid point (Eqs. letkf_xa .. enkf_deltay):

    Q       = (k - 1)/rho_infl I + dY^T R_loc^-1 dY          (Eq. letkf_q)
    P~a     = Q^-1
    wbar    = P~a dY^T R_loc^-1 (yo - ybar)                 (Eq. letkf_wa)
    dW      = sqrt(k - 1) (P~a)^{1/2}                        (Eq. letkf_dwa)
    x^a_m   = xbar + dX (wbar + dw_m)                        (Eq. letkf_xa)

P~a and its square root come from one eigendecomposition of Q (the paper's
route); (P~a)^{1/2} is read as the symmetric square root V L^{-1/2} V^T.
rho_infl is a multiplicative inflation (1 = none, the paper's form).

R-localization (Sec. II-B): R_loc^-1 = G o R^-1 with G diagonal.  Here G is
a Gaussian exp(-d^2 / (2 r^2)) of the periodic minimum-image distance d
from the grid point to the observation point, truncated where
d^2 >= (2 sqrt(10/3) r)^2; distances are integers so the cutoff test is
exact.  "No localization" uses G = 1 for every observation.  The paper's own
choice, Gaspari-Cohn (Sec. II-B), is the option kind="gc": G = GC(d / c), the
fifth-order piecewise rational function of Gaspari & Cohn (1999, Eq. 4.10)
with half-width c = sqrt(10/3) r, whose support d < 2c is the same cutoff.

One local problem is solved per grid point and its transform is applied to
all 9 populations of that point (Sec. II-B: the 9 velocities share the same
observation data).
"""
from __future__ import annotations

import math

import numpy as np

from .obs import ensemble_obs, var_list


def min_image(d, n):
    """Periodic minimum-image displacement of integer d on a ring of n cells."""
    d = np.asarray(d, dtype=np.int64)
    return ((d + n // 2) % n) - n // 2


def local_obs(x, y, obs_xy, nx, ny, cutoff2):
    """Observation points within the cutoff of grid point (x, y).

    Returns (indices, d2) for all points with integer squared periodic
    distance d2 < cutoff2 (cutoff2 = inf selects every point).
    """
    obs_xy = np.asarray(obs_xy, dtype=np.int64)
    dx = min_image(obs_xy[:, 0] - x, nx)
    dy = min_image(obs_xy[:, 1] - y, ny)
    d2 = dx * dx + dy * dy
    sel = np.nonzero(d2 < cutoff2)[0] if math.isfinite(cutoff2) else np.arange(len(d2))
    return sel, d2[sel]


def gaspari_cohn(z):
    """Gaspari-Cohn correlation function of the scaled distance z = d / c (Gaspari & Cohn
    1999, Eq. 4.10): a fifth-order piecewise rational function, 1 at z = 0, 0 for z >= 2."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    a = z <= 1.0
    za = z[a]
    out[a] = (((-0.25 * za + 0.5) * za + 0.625) * za - 5.0 / 3.0) * za * za + 1.0
    b = (z > 1.0) & (z < 2.0)
    zb = z[b]
    out[b] = ((((zb / 12.0 - 0.5) * zb + 0.625) * zb + 5.0 / 3.0) * zb - 5.0) * zb + 4.0 \
        - 2.0 / (3.0 * zb)
    return out


def localization_weight(d2, radius, kind="gauss"):
    """Localization weight G of squared distances d2: Gaussian exp(-d^2 / (2 r^2)), or
    (kind="gc") Gaspari-Cohn GC(d / c) with c = sqrt(10/3) r; radius = inf gives 1."""
    d2 = np.asarray(d2, dtype=np.float64)
    if not math.isfinite(radius):
        return np.ones_like(d2)
    if kind == "gc":
        return gaspari_cohn(np.sqrt(d2) / (math.sqrt(10.0 / 3.0) * radius))
    if kind != "gauss":
        raise ValueError(f"unknown localization {kind!r}")
    return np.exp(-d2 / (2.0 * radius * radius))


def local_analysis(Xb, dY, d, rinv, infl=1.0, eigh=np.linalg.eigh):
    """Analysis of one local problem.

    Xb   [n, k]  background members of the local state (rows: variables)
    dY   [p, k]  local obs-space perturbations (rows: local observed scalars)
    d    [p]     innovations yo - ybar
    rinv [p]     localized inverse observation-error variances G/sigma^2
    Returns a dict with Xa [n, k] and the intermediate quantities.
    """
    Xb = np.asarray(Xb, dtype=np.float64)
    dY = np.asarray(dY, dtype=np.float64).reshape(-1, Xb.shape[1])
    d = np.asarray(d, dtype=np.float64).reshape(-1)
    rinv = np.asarray(rinv, dtype=np.float64).reshape(-1)
    k = Xb.shape[1]
    xbar = Xb.mean(axis=1)
    dX = Xb - xbar[:, None]
    A = dY.T @ (rinv[:, None] * dY)
    c = dY.T @ (rinv * d)
    Q = (k - 1) / infl * np.eye(k) + A
    lam, V = eigh(Q)
    Pa = (V / lam) @ V.T
    wbar = Pa @ c
    dW = math.sqrt(k - 1) * (V / np.sqrt(lam)) @ V.T
    W = wbar[:, None] + dW
    Xa = xbar[:, None] + dX @ W
    return {"Xa": Xa, "A": A, "c": c, "Q": Q, "lam": lam, "V": V, "Pa": Pa,
            "wbar": wbar, "dW": dW, "W": W, "xbar": xbar, "dX": dX}


def point_inputs(x, y, Yf, yo, obs_xy, obs_err_var, nx, ny, radius, cutoff2, obs_vars,
                 ybar=None, dY=None, loc="gauss"):
    """Local obs-space inputs (dY_loc [p, k], d_loc [p], rinv [p], nloc) at (x, y)."""
    if ybar is None:
        ybar, dY = ensemble_obs(Yf)
    V = len(var_list(obs_vars))
    sel, d2 = local_obs(x, y, obs_xy, nx, ny, cutoff2)
    g = localization_weight(d2, radius, loc)
    idx = (sel[:, None] * V + np.arange(V)[None, :]).reshape(-1)
    gs = np.repeat(g, V)
    rinv = gs / np.asarray(obs_err_var, dtype=np.float64)[idx]
    d_loc = np.asarray(yo, dtype=np.float64)[idx] - ybar[idx]
    return dY[:, idx].T, d_loc, rinv, len(sel)


def analyze(f, Yf, yo, obs_xy, obs_err_var, radius, cutoff2, obs_vars, infl=1.0,
            points=None, loc="gauss"):
    """LETKF analysis of an ensemble (Algorithm 1), one local problem per point.

    f   [k, 9, ny, nx] forecast ensemble (member-major, post-streaming)
    Yf  [k, L*V]       forecast observations h(x_m)
    yo  [L*V]          observations
    points: None for every grid point, else an iterable of (x, y).
    Returns (Xa, info): Xa has f's shape (only the requested points are
    updated when ``points`` is given); info maps (x, y) -> local results.
    """
    f = np.asarray(f, dtype=np.float64)
    k, nv, ny, nx = f.shape
    ybar, dY = ensemble_obs(Yf)
    Xa = f.copy()
    info = {}
    if points is None:
        points = [(x, y) for y in range(ny) for x in range(nx)]
    for (x, y) in points:
        dYl, dl, rl, nloc = point_inputs(x, y, Yf, yo, obs_xy, obs_err_var, nx, ny, radius,
                                         cutoff2, obs_vars, ybar=ybar, dY=dY, loc=loc)
        res = local_analysis(f[:, :, y, x].T, dYl, dl, rl, infl)
        res["nloc"] = nloc
        Xa[:, :, y, x] = res["Xa"].T
        info[(x, y)] = res
    return Xa, info
