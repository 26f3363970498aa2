"""Pins of the FP64 LETKF oracle (Sec. II-B, Algorithm 1) against independent facts:
brute-force Kalman filter, number-theoretic lattice counts, closed-form spectra, the 3D
convolution behind the Gaspari-Cohn function, a hand-worked scalar case and the transform's
algebraic identities."""
import json
import math
import os

import numpy as np
import pytest

from oracle import lbm, obs, letkf, kalman, jacobi
from synth import gaussian, regular_obs_network, loc_cutoff2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- local obs selection

def _r2(n):
    """Number of ways to write n as a sum of two squares (Jacobi: 4 (d_1(n) - d_3(n)))."""
    if n == 0:
        return 1
    d1 = sum(1 for d in range(1, n + 1) if n % d == 0 and d % 4 == 1)
    d3 = sum(1 for d in range(1, n + 1) if n % d == 0 and d % 4 == 3)
    return 4 * (d1 - d3)


@pytest.mark.parametrize("n,stride,radius", [(32, 4, 3.0), (256, 8, 8.0), (128, 4, 12.0)])
def test_local_count_on_an_obs_point_is_a_lattice_disk_count(n, stride, radius):
    # A grid point on an observation point sees the obs lattice points stride*(i, j) with
    # stride^2 (i^2 + j^2) < c^2: sum of r2(m) over m < c^2 / stride^2.
    c2 = loc_cutoff2(radius)
    net = regular_obs_network(n, n, stride)
    sel, d2 = letkf.local_obs(0, 0, net, n, n, c2)
    expect = sum(_r2(m) for m in range(0, int(math.ceil(c2 / stride ** 2))) if stride ** 2 * m < c2)
    assert len(sel) == expect
    assert (d2 < c2).all()


def test_configured_cutoffs():
    # c = 2 sqrt(10/3) r: c^2 = 120 for r = 3 and 1920 for r = 12
    assert loc_cutoff2(3.0) == pytest.approx(120.0, abs=1e-12)
    assert loc_cutoff2(12.0) == pytest.approx(1920.0, abs=1e-9)


def test_local_obs_matches_brute_force_over_periodic_images():
    nx, ny, c2 = 12, 10, 20.0
    rng = np.random.Generator(np.random.PCG64(7))
    net = np.unique(rng.integers(0, [nx, ny], size=(25, 2)), axis=0).astype(np.int32)
    for y in range(ny):
        for x in range(nx):
            sel, d2 = letkf.local_obs(x, y, net, nx, ny, c2)
            brute = []
            for i, (ox, oy) in enumerate(net):
                best = min((ox + sx * nx - x) ** 2 + (oy + sy * ny - y) ** 2
                           for sx in (-1, 0, 1) for sy in (-1, 0, 1))
                if best < c2:
                    brute.append((i, best))
            assert [int(s) for s in sel] == [b[0] for b in brute]
            assert [int(v) for v in d2] == [b[1] for b in brute]


def test_gaussian_weight_values():
    r = 3.0
    w = letkf.localization_weight(np.array([0.0, r * r, loc_cutoff2(r)]), r)
    assert w[0] == 1.0
    assert w[1] == pytest.approx(math.exp(-0.5), rel=1e-15)
    assert w[2] == pytest.approx(math.exp(-20.0 / 3.0), rel=1e-14)
    assert (letkf.localization_weight(np.array([5.0, 1e9]), math.inf) == 1.0).all()


def _cone_self_convolution(z):
    """3D self-convolution of the radial cone (1 - s)_+ at distance z, normalized to 1 at 0:
    the construction behind the Gaspari-Cohn function, evaluated by quadrature."""
    from scipy import integrate

    def cone(s):
        return max(0.0, 1.0 - s)

    def conv(r):
        if r < 1e-12:
            return 4.0 * math.pi * integrate.quad(lambda s: s * s * cone(s) ** 2, 0.0, 1.0,
                                                  epsabs=1e-14, epsrel=1e-12)[0]

        def inner(s):
            lo, hi = abs(r - s), min(r + s, 1.0)
            if hi <= lo:
                return 0.0
            return integrate.quad(lambda t: t * cone(t), lo, hi, epsabs=1e-14, epsrel=1e-12)[0]
        return 2.0 * math.pi / r * integrate.quad(lambda s: s * cone(s) * inner(s), 0.0, 1.0,
                                                  limit=200, epsabs=1e-14, epsrel=1e-12)[0]
    return conv(z) / conv(0.0)


@pytest.mark.parametrize("z", [0.05, 0.3, 0.7, 1.0, 1.2, 1.6, 1.9])
def test_gaspari_cohn_is_the_self_convolution_of_a_cone(z):
    # Gaspari & Cohn build their fifth-order function as a 3D convolution of compactly
    # supported pieces; the normalized self-convolution of (1 - d/c)_+ reproduces it, which
    # pins every coefficient and both branches of the oracle's piecewise formula.
    pytest.importorskip("scipy")
    assert letkf.gaspari_cohn(np.array([z]))[0] == pytest.approx(_cone_self_convolution(z),
                                                                    abs=1e-9)


def test_gaspari_cohn_weight_support_and_shape():
    r = 3.0
    c = math.sqrt(10.0 / 3.0) * r
    d = np.linspace(0.0, 2.5 * c, 2001)
    w = letkf.localization_weight(d * d, r, "gc")
    assert w[0] == 1.0
    assert (w[d >= 2.0 * c] == 0.0).all()          # zero from the default cutoff on
    assert (np.diff(w[d < 2.0 * c]) < 0.0).all()   # strictly decreasing inside
    # the two branches meet at d = c (value 5/24) without a jump in value or slope
    assert letkf.gaspari_cohn(np.array([1.0]))[0] == pytest.approx(5.0 / 24.0, rel=1e-14)
    g = letkf.gaspari_cohn(np.array([1.0 - 2e-6, 1.0 - 1e-6, 1.0 + 1e-6, 1.0 + 2e-6]))
    assert (g[1] - g[0]) == pytest.approx(g[3] - g[2], rel=1e-4)
    with pytest.raises(ValueError):
        letkf.localization_weight(np.array([1.0]), r, "spline")


# ---------------------------------------------------------------- observation operator

def test_observation_operator_reads_moments():
    ny, nx = 6, 8
    rho = 1.0 + gaussian((ny, nx), 0.01, 1)
    ux = gaussian((ny, nx), 0.01, 2)
    uy = gaussian((ny, nx), 0.01, 3)
    f = lbm.equilibrium(rho, ux, uy)
    net = np.array([[1, 2], [7, 5], [0, 0]], dtype=np.int32)
    y = obs.observe(f, net, obs.VAR_RHO | obs.VAR_U | obs.VAR_V)
    expect = np.stack([rho[net[:, 1], net[:, 0]], ux[net[:, 1], net[:, 0]],
                       uy[net[:, 1], net[:, 0]]], axis=1).ravel()
    assert np.allclose(y, expect, atol=1e-15)
    y2 = obs.observe(f, net, obs.VAR_U | obs.VAR_V)
    assert np.allclose(y2, expect.reshape(3, 3)[:, 1:].ravel(), atol=1e-15)


# ---------------------------------------------------------------- eigensolvers

def _toeplitz_tridiagonal(n):
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


@pytest.mark.parametrize("n", [2, 5, 8, 16])
def test_eigensolvers_on_closed_form_spectrum(n):
    # tridiag(-1, 2, -1) has eigenvalues 2 - 2 cos(pi j / (n + 1)), j = 1..n
    A = _toeplitz_tridiagonal(n)
    exact = np.sort(2.0 - 2.0 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1)))
    for lam, V in (jacobi.jacobi_eigh(A), np.linalg.eigh(A)):
        assert np.allclose(np.sort(lam), exact, atol=1e-13)
        assert np.allclose(V @ np.diag(lam) @ V.T, A, atol=1e-13)
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)


def test_jacobi_matches_lapack_on_random_spd():
    for seed, n in [(1, 8), (2, 16), (3, 24)]:
        B = gaussian((n, n), 1.0, seed)
        A = (n - 1) * np.eye(n) + B @ B.T
        lj, Vj = jacobi.jacobi_eigh(A)
        ll, Vl = np.linalg.eigh(A)
        assert np.allclose(lj, ll, rtol=1e-13)
        # same matrix function from both decompositions
        assert np.allclose((Vj / np.sqrt(lj)) @ Vj.T, (Vl / np.sqrt(ll)) @ Vl.T, atol=1e-13)


# ---------------------------------------------------------------- one local problem

def _random_local_problem(k, p, n=9, seed=0):
    Xb = 0.1 + gaussian((n, k), 0.01, seed)
    Yf = gaussian((k, p), 0.01, seed + 1)
    ybar, dY = obs.ensemble_obs(Yf)
    d = gaussian((p,), 0.01, seed + 2)
    rinv = 1e4 * np.exp(-gaussian((p,), 1.0, seed + 3) ** 2)
    return Xb, dY.T, d, rinv


@pytest.mark.parametrize("k,p", [(8, 47), (16, 5), (32, 84), (64, 20)])
def test_transform_identities(k, p):
    Xb, dY, d, rinv = _random_local_problem(k, p, seed=k + p)
    r = letkf.local_analysis(Xb, dY, d, rinv)
    one = np.ones(k)
    Q, dW, wbar = r["Q"], r["dW"], r["wbar"]
    assert np.allclose(Q, Q.T, atol=0)
    assert np.allclose(Q @ one, (k - 1) * one, rtol=1e-12)          # dY 1 = 0
    assert r["lam"].min() >= (k - 1) * (1 - 1e-12)
    assert np.allclose(dW, dW.T, atol=1e-13)
    assert np.allclose(dW @ one, one, atol=1e-12)                    # dW 1 = 1
    assert np.allclose(dW @ dW, (k - 1) * np.linalg.inv(Q), atol=1e-12)
    assert abs(one @ wbar) < 1e-12 * max(1.0, np.abs(wbar).max())     # 1^T wbar = 0
    dXa = r["Xa"] - r["Xa"].mean(axis=1, keepdims=True)
    assert np.allclose(r["Xa"].mean(axis=1), r["xbar"] + r["dX"] @ wbar, atol=1e-15)
    assert np.allclose(dXa.sum(axis=1), 0.0, atol=1e-14)            # perturbations sum to 0


def test_no_local_observation_is_identity():
    Xb, _, _, _ = _random_local_problem(8, 1)
    r = letkf.local_analysis(Xb, np.zeros((0, 8)), np.zeros(0), np.zeros(0))
    assert np.allclose(r["Xa"], Xb, atol=1e-15)


@pytest.mark.parametrize("rho", [1.0, 1.3])
def test_no_local_observation_with_inflation_scales_perturbations(rho):
    # With no observation Q = (k-1)/rho I, so wbar = 0 and dW = sqrt(k-1) Q^-1/2 = sqrt(rho) I:
    # the mean is kept and every perturbation is scaled by sqrt(rho) (Eqs. letkf_q ..
    # letkf_xa with the inflated Q).
    Xb, _, _, _ = _random_local_problem(12, 1, seed=33)
    r = letkf.local_analysis(Xb, np.zeros((0, 12)), np.zeros(0), np.zeros(0), rho)
    xbar = Xb.mean(axis=1, keepdims=True)
    assert np.allclose(r["Xa"], xbar + math.sqrt(rho) * (Xb - xbar), atol=1e-15)


def test_scalar_two_member_case_matches_hand_worked_kalman():
    g = json.load(open(os.path.join(GOLDEN, "scalar_kalman_k2.json")))
    x = np.array([g["members"]])
    xbar = x.mean()
    r = letkf.local_analysis(x, (x - xbar), np.array([g["yo"] - xbar]),
                             np.array([1.0 / g["obs_error_var"]]))
    assert np.allclose(r["Xa"][0], g["analysis_members"], rtol=1e-14)
    assert r["Xa"].mean() == pytest.approx(g["analysis_mean"], rel=1e-14)
    assert np.var(r["Xa"][0], ddof=1) == pytest.approx(g["analysis_variance"], rel=1e-13)


# ---------------------------------------------------------------- whole-ensemble analysis

def _linear_h(obs_xy, nx, ny):
    """Linear H observing rho = sum f and j_x = sum c_x f at each point (state order q, y, x)."""
    L = len(obs_xy)
    H = np.zeros((2 * L, 9 * ny * nx))
    for l, (ox, oy) in enumerate(obs_xy):
        for q in range(9):
            col = (q * ny + oy) * nx + ox
            H[2 * l, col] = 1.0
            H[2 * l + 1, col] = lbm.CX[q]
    return H


def _small_ensemble(k, nx, ny, seed):
    rho = 1.0 + gaussian((k, ny, nx), 0.01, seed)
    ux = gaussian((k, ny, nx), 0.02, seed + 1)
    uy = gaussian((k, ny, nx), 0.02, seed + 2)
    return lbm.equilibrium(rho, ux, uy) + gaussian((k, 9, ny, nx), 1e-3, seed + 3)


@pytest.mark.parametrize("k", [3, 6, 8])
def test_infinite_localization_equals_brute_force_kalman_filter(k):
    # With G = 1 and every observation local, the LETKF at each grid point uses the same
    # ensemble-space solution; with a linear H it must equal the KF (Eqs. kfx, kfp, kfk)
    # with the ensemble covariance (Eq. enkf_p).
    nx = ny = 4
    f = _small_ensemble(k, nx, ny, 100 + k)
    net = np.array([[0, 0], [2, 1], [3, 3]], dtype=np.int32)
    H = _linear_h(net, nx, ny)
    X = f.reshape(k, -1).T                      # [N, k]
    Yf = (H @ X).T                              # [k, 2L]
    rvar = np.array([1e-4, 4e-4, 2e-4, 1e-4, 3e-4, 1e-4])
    yo = H @ X.mean(axis=1) + gaussian((6,), 0.01, 7)
    Xa, info = letkf.analyze(f, Yf, yo, net, rvar, math.inf, math.inf,
                             obs.VAR_RHO | obs.VAR_U)
    xa_kf, Pa_kf, _ = kalman.kalman_analysis(X.mean(axis=1), kalman.ensemble_covariance(X),
                                             H, np.diag(rvar), yo)
    Xa_flat = Xa.reshape(k, -1).T
    incr = xa_kf - X.mean(axis=1)
    assert np.allclose(Xa_flat.mean(axis=1) - X.mean(axis=1), incr,
                       atol=1e-10 * np.abs(incr).max())
    Pa = kalman.ensemble_covariance(Xa_flat)
    assert np.allclose(Pa, Pa_kf, atol=1e-10 * np.abs(Pa_kf).max())
    # every grid point solved the same (global) ensemble-space problem
    Ws = [r["W"] for r in info.values()]
    assert all(np.allclose(W, Ws[0], atol=1e-12) for W in Ws)


@pytest.mark.parametrize("k,rho", [(4, 1.1), (6, 1.5), (8, 1.1), (8, 1.5)])
def test_inflated_analysis_equals_kalman_filter_on_inflated_covariance(k, rho):
    # Multiplicative inflation rho scales the background covariance: Pf = rho dX dX^T / (k-1)
    # (Eq. enkf_p times rho).  With a linear H and no localization, the LETKF's
    # Q = (k-1)/rho I + dY^T R^-1 dY must then give the KF's mean x^f + K (yo - H x^f) and the
    # KF's covariance (I - K H) rho Pb (Eqs. kfx, kfp, kfk with rho Pb).  A mistaken
    # (k-1) rho, or an inflation of only one of the mean and the perturbations, fails here.
    nx = ny = 4
    f = _small_ensemble(k, nx, ny, 700 + k)
    net = np.array([[1, 0], [3, 2], [0, 3]], dtype=np.int32)
    H = _linear_h(net, nx, ny)
    X = f.reshape(k, -1).T
    Yf = (H @ X).T
    rvar = np.array([2e-4, 1e-4, 1e-4, 5e-4, 3e-4, 2e-4])
    yo = H @ X.mean(axis=1) + gaussian((6,), 0.01, 17)
    Xa, _ = letkf.analyze(f, Yf, yo, net, rvar, math.inf, math.inf,
                          obs.VAR_RHO | obs.VAR_U, infl=rho)
    Pb = kalman.ensemble_covariance(X)
    xa_kf, Pa_kf, _ = kalman.kalman_analysis(X.mean(axis=1), rho * Pb, H, np.diag(rvar), yo)
    Xa_flat = Xa.reshape(k, -1).T
    incr = xa_kf - X.mean(axis=1)
    assert np.allclose(Xa_flat.mean(axis=1) - X.mean(axis=1), incr,
                       atol=1e-10 * np.abs(incr).max())
    Pa = kalman.ensemble_covariance(Xa_flat)
    assert np.allclose(Pa, Pa_kf, atol=1e-10 * np.abs(Pa_kf).max())
    # and it differs from the uninflated analysis by more than rounding
    _, Pa_1, _ = kalman.kalman_analysis(X.mean(axis=1), Pb, H, np.diag(rvar), yo)
    assert np.abs(Pa_kf - Pa_1).max() > 1e-3 * np.abs(Pa_kf).max()


def test_infinite_localization_equals_global_etkf():
    k, nx, ny = 8, 5, 4
    f = _small_ensemble(k, nx, ny, 300)
    net = np.array([[1, 1], [4, 3], [0, 2]], dtype=np.int32)
    Yf = obs.observe(f, net, obs.VAR_U | obs.VAR_V)
    rvar = np.full(6, 1e-4)
    yo = Yf.mean(axis=0) + gaussian((6,), 0.01, 9)
    Xa, _ = letkf.analyze(f, Yf, yo, net, rvar, math.inf, math.inf, obs.VAR_U | obs.VAR_V)
    ybar, dY = obs.ensemble_obs(Yf)
    g = letkf.local_analysis(f.reshape(k, -1).T, dY.T, yo - ybar, 1.0 / rvar)
    assert np.allclose(Xa.reshape(k, -1).T, g["Xa"], atol=1e-14)


def test_localized_analysis_reduces_spread_only_near_observations():
    k, n = 8, 16
    f = _small_ensemble(k, n, n, 500)
    net = np.array([[3, 3]], dtype=np.int32)
    Yf = obs.observe(f, net, obs.VAR_U | obs.VAR_V)
    yo = Yf.mean(axis=0)
    Xa, info = letkf.analyze(f, Yf, yo, net, np.full(2, 1e-6), 2.0, loc_cutoff2(2.0),
                             obs.VAR_U | obs.VAR_V)
    far = (11, 11)                      # distance^2 = 128 >= 53.3: no local obs
    assert info[far]["nloc"] == 0
    assert np.allclose(Xa[:, :, 11, 11], f[:, :, 11, 11], atol=1e-15)
    near = (3, 3)
    assert info[near]["nloc"] == 1
    assert np.var(Xa[:, :, 3, 3], axis=0).sum() < np.var(f[:, :, 3, 3], axis=0).sum()
