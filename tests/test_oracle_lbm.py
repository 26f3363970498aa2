"""Pins of the FP64 LBM oracle against closed forms and invariants (Sec. II-A)."""
import math

import numpy as np
import pytest

from oracle import lbm
from synth import taylor_green_velocity, kolmogorov_force, gaussian

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_population_order_convention():
    # c_q = (i, j) with q = 3 (j + 1) + (i + 1), (i, j) in {-1, 0, 1}^2 (Eq. 1 indices)
    for q in range(9):
        assert lbm.CX[q] == q % 3 - 1
        assert lbm.CY[q] == q // 3 - 1


def test_lattice_isotropy_tensors():
    # Textbook D2Q9 lattice tensors: sum w = 1, sum w c_a = 0, sum w c_a c_b = delta/3,
    # sum w c_a c_b c_c = 0, sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9.
    c = np.stack([lbm.CX, lbm.CY], axis=1).astype(float)
    w = lbm.W
    d = np.eye(2)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("q,qa->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, c, c), d / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    t4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
          + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), t4, atol=1e-15)


def test_equilibrium_moments_exact():
    # sum feq = rho, sum c feq = rho u, sum c_a c_b feq = rho (u_a u_b + delta_ab / 3)
    rho = 1.0 + gaussian((5, 7), 0.05, 1)
    ux = gaussian((5, 7), 0.05, 2)
    uy = gaussian((5, 7), 0.05, 3)
    feq = lbm.equilibrium(rho, ux, uy)
    c = [lbm.CX[:, None, None].astype(float), lbm.CY[:, None, None].astype(float)]
    u = [ux, uy]
    assert np.allclose(feq.sum(0), rho, rtol=1e-14)
    for a in range(2):
        assert np.allclose((c[a] * feq).sum(0), rho * u[a], atol=1e-15)
        for b in range(2):
            expect = rho * (u[a] * u[b] + (1.0 / 3.0 if a == b else 0.0))
            assert np.allclose((c[a] * c[b] * feq).sum(0), expect, atol=1e-15)
    r2, ux2, uy2 = lbm.moments(feq)  # Eqs. 2-3 recover rho and u
    assert np.allclose(r2, rho, rtol=1e-14)
    assert np.allclose(ux2, ux, atol=1e-15)
    assert np.allclose(uy2, uy, atol=1e-15)


def test_rest_state_is_fixed_point():
    f = lbm.equilibrium(np.ones((6, 5)), np.zeros((6, 5)), np.zeros((6, 5)))
    assert np.allclose(lbm.run(f, 0.6, 5), f, atol=1e-16)


def test_force_term_moments():
    fx = gaussian((4, 4), 1e-5, 4)
    fy = gaussian((4, 4), 1e-5, 5)
    F = lbm.force_term(fx, fy)
    assert np.allclose(F.sum(0), 0.0, atol=1e-20)
    assert np.allclose((lbm.CX[:, None, None] * F).sum(0), fx, atol=1e-20)
    assert np.allclose((lbm.CY[:, None, None] * F).sum(0), fy, atol=1e-20)


def test_streaming_moves_along_c():
    # Eq. 1: what leaves x with velocity c_q arrives at x + c_q one step later
    for q in range(9):
        f = np.zeros((9, 6, 7))
        f[q, 2, 3] = 1.0
        g = lbm.stream(f)
        assert g[q, (2 + lbm.CY[q]) % 6, (3 + lbm.CX[q]) % 7] == 1.0
        assert g.sum() == 1.0


def _random_state(ny, nx, seed):
    rho = 1.0 + gaussian((ny, nx), 0.01, seed)
    ux = gaussian((ny, nx), 0.02, seed + 1)
    uy = gaussian((ny, nx), 0.02, seed + 2)
    return lbm.equilibrium(rho, ux, uy) + gaussian((9, ny, nx), 1e-3, seed + 3)


def test_mass_conservation():
    f = _random_state(12, 10, 10)
    m0 = f.sum()
    fx = gaussian((12, 10), 1e-4, 20)
    fy = gaussian((12, 10), 1e-4, 21)
    g = lbm.run(f, 0.55, 30, fx, fy)
    assert abs(g.sum() - m0) < 1e-12 * m0


def test_momentum_changes_by_total_force():
    # BGK conserves momentum locally; each step adds sum_x F(x) to the total
    f = _random_state(9, 11, 30)
    fx = 1e-4 + gaussian((9, 11), 1e-4, 40)
    fy = -2e-4 + gaussian((9, 11), 1e-4, 41)
    def total_momentum(h):
        return np.array([(lbm.CX[:, None, None] * h).sum(), (lbm.CY[:, None, None] * h).sum()])
    p0 = total_momentum(f)
    g = lbm.run(f, 0.7, 3, fx, fy)
    expect = p0 + 3 * np.array([fx.sum(), fy.sum()])
    assert np.allclose(total_momentum(g), expect, rtol=0, atol=1e-13)


def _tgv_decay_error(n, tau, u0, t_end):
    ux0, uy0 = taylor_green_velocity(n, n, u0)
    f = lbm.equilibrium(np.ones((n, n)), ux0, uy0)
    f = lbm.run(f, tau, t_end)
    _, ux, uy = lbm.moments(f)
    amp = float((ux * ux0 + uy * uy0).sum() / (ux0 * ux0 + uy0 * uy0).sum())
    kappa = 2 * math.pi / n
    exact = math.exp(-2.0 * lbm.viscosity(tau) * kappa * kappa * t_end)
    return abs(amp - exact) / exact


def test_taylor_green_decay_matches_closed_form():
    # Closed form: u(t) = u(0) exp(-2 nu kappa^2 t), nu = (tau - 1/2)/3.  Diffusive scaling
    # (t ~ n^2) keeps the decay fixed while the lattice error falls as 1/n^2.
    e32 = _tgv_decay_error(32, 0.8, 0.01, 200)
    e64 = _tgv_decay_error(64, 0.8, 0.005, 800)
    assert e32 < 8e-3, e32
    assert e64 < e32 / 3.5, (e32, e64)   # second order: ratio -> 4


def _kolmogorov_amp_error(n, tau, amp, steps):
    fx, fy = kolmogorov_force(n, n, amp, 1)
    f = lbm.equilibrium(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    f = lbm.run(f, tau, steps, fx, fy)
    _, ux, uy = lbm.moments(f)
    kappa = 2 * math.pi / n
    s = np.sin(kappa * np.arange(n))[:, None]
    got = float((ux * s).sum() / (s * s).sum() / n)
    exact = amp / (lbm.viscosity(tau) * kappa * kappa)   # steady Stokes balance nu u'' = -F
    assert np.abs(uy).max() < 1e-9 * exact
    return abs(got - exact) / exact


def test_kolmogorov_steady_state_matches_closed_form():
    e16 = _kolmogorov_amp_error(16, 0.8, 1e-6, 2500)
    e32 = _kolmogorov_amp_error(32, 0.8, 1e-6, 8000)
    assert e16 < 0.03, e16
    assert e32 < e16 / 3.5, (e16, e32)   # second order: ratio -> 4
