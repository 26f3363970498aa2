"""Matched GPU / oracle cases for the parity tests.

Inputs come from ``synth`` (seeded) only; each side then computes with its own
code: the oracle in FP64 NumPy, the library in CUDA.  Nothing here holds the
method's arithmetic besides calls into ``oracle``.
"""
from __future__ import annotations

import math

import numpy as np

import synth
from oracle import lbm, obs as oobs, letkf as oletkf

VARS_UV = oobs.VAR_U | oobs.VAR_V


W32 = lbm.W.astype(np.float32)
DW32 = (lbm.W - W32.astype(np.float64)).astype(np.float32)


def dev64(g32):
    """Device deviation g = f - w (FP32, exact weights w) as FP64."""
    return np.asarray(g32, np.float64)


def to_deviation32(f32):
    """The FP32 deviation the device forms from an FP32 f: (f - fl(w)) - fl(w - fl(w))."""
    sh = (9,) + (1,) * (np.ndim(f32) - 2)
    return ((f32 - W32.reshape(sh)) - DW32.reshape(sh)).astype(np.float32)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def ensemble_state(k, nx, ny, seed, u0=0.01, sigma=0.005, truth_noise=1e-3, tgv=True):
    """FP32 member-major f [k, 9, ny, nx] = f^eq(1, truth + perturbation), via the oracle's
    equilibrium (the inputs are velocities from synth; the equilibrium is the oracle's)."""
    if tgv:
        ux, uy = synth.taylor_green_velocity(nx, ny, u0)
    else:
        ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx))
    ux = ux + synth.gaussian((ny, nx), truth_noise, seed)
    uy = uy + synth.gaussian((ny, nx), truth_noise, seed + 1)
    dux = synth.gaussian((k, ny, nx), sigma, seed + 2)
    duy = synth.gaussian((k, ny, nx), sigma, seed + 3)
    rho = 1.0 + synth.gaussian((k, ny, nx), 1e-4, seed + 4)
    f = lbm.equilibrium(rho, ux[None] + dux, uy[None] + duy)
    return f.astype(np.float32)


def perturb_nonequilibrium(f, sigma, seed):
    return (f + synth.gaussian(f.shape, sigma, seed)).astype(np.float32)


def observations(f_truth, obs_xy, obs_vars, sigma, seed):
    """yo = h(truth) + N(0, sigma^2), FP32 (h evaluated by the oracle)."""
    y = oobs.observe(f_truth.astype(np.float64), obs_xy, obs_vars)
    return (y + synth.gaussian(y.shape, sigma, seed)).astype(np.float32)


def oracle_analysis(f32, yo, obs_xy, obs_var, radius, obs_vars, points=None, infl=1.0,
                    loc="gauss"):
    """Oracle analysis of the FP32 state f32 (as FP64)."""
    f = f32.astype(np.float64)
    Yf = oobs.observe(f, obs_xy, obs_vars)
    c2 = synth.loc_cutoff2(radius) if math.isfinite(radius) else math.inf
    return oletkf.analyze(f, Yf, yo.astype(np.float64), obs_xy, obs_var.astype(np.float64),
                          radius, c2, obs_vars, infl=infl, points=points, loc=loc)


def point_parity(xa_gpu, xa_orc, xf):
    """(mean rel err, mean-increment rel err, perturbation rel err) of [k, 9] blocks."""
    xa_gpu = np.asarray(xa_gpu, np.float64)
    xa_orc = np.asarray(xa_orc, np.float64)
    xf = np.asarray(xf, np.float64)
    mg, mo, mf = xa_gpu.mean(0), xa_orc.mean(0), xf.mean(0)
    inc_err = rel_l2(mg - mf, mo - mf)
    mean_err = rel_l2(mg, mo)
    pert_err = rel_l2(xa_gpu - mg, xa_orc - mo)
    return mean_err, inc_err, pert_err


def big_ensemble_state(k, nx, ny, seed, sigma=0.005, u0=0.01):
    """Like ensemble_state but built member by member (FP64 equilibrium per member, stored
    FP32), for full-size grids where a [k, 9, ny, nx] FP64 array would not fit comfortably."""
    ux0, uy0 = synth.taylor_green_velocity(nx, ny, u0)
    out = np.empty((k, 9, ny, nx), dtype=np.float32)
    for m in range(k):
        dux = synth.gaussian((ny, nx), sigma, seed + 10 * m)
        duy = synth.gaussian((ny, nx), sigma, seed + 10 * m + 1)
        out[m] = lbm.equilibrium(np.ones((ny, nx)), ux0 + dux, uy0 + duy)
    return out


def observe_at_points(f32, obs_xy, obs_vars):
    """Oracle h(x) for every member, evaluating only the observation points (same oracle
    function on a 1 x L strip of the grid)."""
    xs, ys = obs_xy[:, 0], obs_xy[:, 1]
    strip = f32[:, :, ys, xs].astype(np.float64)[:, :, None, :]   # [k, 9, 1, L]
    L = len(obs_xy)
    strip_xy = np.stack([np.arange(L), np.zeros(L, dtype=np.int64)], axis=1)
    return oobs.observe(strip, strip_xy, obs_vars)


def oracle_points(f32, Yf, yo, obs_xy, obs_var, radius, obs_vars, points, infl=1.0):
    """Oracle local analyses at the given (x, y) points only (Algorithm 1 per point)."""
    k, _, ny, nx = f32.shape
    ybar, dY = oobs.ensemble_obs(Yf)
    c2 = synth.loc_cutoff2(radius) if math.isfinite(radius) else math.inf
    out = {}
    for (x, y) in points:
        dYl, dl, rl, nloc = oletkf.point_inputs(x, y, Yf, yo.astype(np.float64), obs_xy,
                                                obs_var.astype(np.float64), nx, ny, radius, c2,
                                                obs_vars, ybar=ybar, dY=dY)
        res = oletkf.local_analysis(f32[:, :, y, x].astype(np.float64).T, dYl, dl, rl, infl)
        res["nloc"] = nloc
        out[(x, y)] = res
    return out
