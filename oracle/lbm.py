"""D2Q9 lattice Boltzmann method in FP64 (Sec. II-A).

Restates the paper's lattice Boltzmann equation (Eq. 1)

    f_ij(x + c i dt, y + c j dt, t + dt) = f_ij(x, y, t) + Omega_ij(x, y, t)

with (i, j) in {-1, 0, 1}^2 (D2Q9), lattice units c = dx = dt = 1, the
lattice-BGK collision Omega = -(f - f^eq) / tau and a body force F, and the
moments of Eqs. 2-5: rho = sum f, u = (1/rho) sum c f.

Readings where the paper is silent:
  * population index q = 3 (j + 1) + (i + 1) for c_q = (i, j);
  * f^eq is the standard second-order D2Q9 equilibrium
    w_q rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u), weights 4/9, 1/9, 1/36;
  * the body force enters as F_q = 3 w_q c_q . F added after the BGK
    relaxation, with u = (sum c f) / rho (no half-force shift);
  * the state stored at integer t is the post-streaming f.

Arrays are [..., 9, ny, nx] (member-major structure of arrays, as the
paper's LBM layout X[m, N_v, N_x], Sec. IV-A).
"""
from __future__ import annotations

import numpy as np

# c_q = (i, j) with q = 3 (j + 1) + (i + 1)
CX = np.array([-1, 0, 1, -1, 0, 1, -1, 0, 1], dtype=np.int64)
CY = np.array([-1, -1, -1, 0, 0, 0, 1, 1, 1], dtype=np.int64)
W = np.array([1 / 36, 1 / 9, 1 / 36, 1 / 9, 4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36], dtype=np.float64)
NV = 9


def _bc(a):
    """Broadcast a length-9 vector over [..., 9, ny, nx]."""
    return a.astype(np.float64)[:, None, None]


def equilibrium(rho, ux, uy):
    """Second-order D2Q9 equilibrium f^eq_q(rho, u), shape [..., 9, ny, nx]."""
    rho = np.asarray(rho, dtype=np.float64)
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    cu = _bc(CX) * ux[..., None, :, :] + _bc(CY) * uy[..., None, :, :]
    uu = (ux * ux + uy * uy)[..., None, :, :]
    return _bc(W) * rho[..., None, :, :] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


def moments(f):
    """Density and velocity (Eqs. 2-3): rho = sum_q f_q, u = sum_q c_q f_q / rho."""
    f = np.asarray(f, dtype=np.float64)
    rho = f.sum(axis=-3)
    jx = (f * _bc(CX)).sum(axis=-3)
    jy = (f * _bc(CY)).sum(axis=-3)
    return rho, jx / rho, jy / rho


def force_term(fx, fy):
    """Body-force source F_q = 3 w_q (c_q . F), shape [9, ny, nx]."""
    fx = np.asarray(fx, dtype=np.float64)
    fy = np.asarray(fy, dtype=np.float64)
    return 3.0 * _bc(W) * (_bc(CX) * fx[None] + _bc(CY) * fy[None])


def collide(f, tau, fx=None, fy=None):
    """Post-collision populations f* = f - (f - f^eq(rho, u)) / tau + F_q."""
    rho, ux, uy = moments(f)
    fs = f - (f - equilibrium(rho, ux, uy)) / tau
    if fx is not None:
        fs = fs + force_term(fx, fy)
    return fs


def stream(fs):
    """Periodic streaming: the population q at x moves to x + c_q."""
    out = np.empty_like(fs)
    for q in range(NV):
        out[..., q, :, :] = np.roll(fs[..., q, :, :], shift=(int(CY[q]), int(CX[q])), axis=(-2, -1))
    return out


def step(f, tau, fx=None, fy=None):
    """One time step of Eq. 1: collide then stream."""
    return stream(collide(f, tau, fx, fy))


def run(f, tau, nsteps, fx=None, fy=None):
    """``nsteps`` time steps from the post-streaming state ``f``."""
    f = np.array(f, dtype=np.float64, copy=True)
    for _ in range(int(nsteps)):
        f = step(f, tau, fx, fy)
    return f


def viscosity(tau):
    """Kinematic viscosity of the BGK model in lattice units, (tau - 1/2) / 3."""
    return (tau - 0.5) / 3.0
