"""The EVD-free schedule (LETKF_EIG_RATIONAL) against the FP64 oracle at full size.

The schedule computes Q^-1 c by one tridiagonal solve and Q^-1/2 by Zolotarev's rational
approximation of t^-1/2 (shifted L D L^T solves of the tridiagonal T), after the same
Householder tridiagonalization as the split schedule; no eigenvectors are formed.  Checked:
  * the full-size workloads (256^2 at k = 32, 1024^2 at k = 64) at sampled grid points against
    the oracle's local analyses, FP32 and mixed, at the parity tests' bars (1e-5 relative L2
    over the sampled outputs, 5e-5 per point);
  * points whose condition bound exceeds the largest approximation's range go to the fused
    kernel: with an inflation that makes every observed point's Q that ill-conditioned the
    schedule's output equals the fused schedule's bit for bit there;
  * the cycle through the captured graph equals forecast + analysis on this schedule.
"""
import numpy as np
import pytest

import synth
from oracle import lbm
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

UV = L.LETKF_OBS_U | L.LETKF_OBS_V


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _sampled_points(nx, ny, n, seed):
    rng = synth.generator(seed)
    pts = {(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, ny // 2)}
    while len(pts) < n:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    return sorted(pts)


@pytest.mark.parametrize("name,precision", [("turb256_k32", L.LETKF_FP32),
                                            ("turb256_k32", L.LETKF_MIXED),
                                            ("turb1024_k64", L.LETKF_FP32),
                                            ("turb1024_k64", L.LETKF_MIXED)])
def test_full_size_workload_sampled_points_match_oracle(name, precision):
    w = synth.WORKLOADS[name]
    nx, ny, k = w.nx, w.ny, w.k
    f0 = C.big_ensemble_state(k, nx, ny, seed=141)
    net = w.obs_network()
    var = w.obs_error_var(len(net) * 2).astype(np.float32)
    exp = L.Experiment(nx, ny, k, w.tau, net, var, loc_radius=w.loc_radius,
                       precision=precision, eig_schedule=L.LETKF_EIG_RATIONAL)
    exp.set_state(f0)
    Yf = C.observe_at_points(f0, net, UV)
    yo = (Yf.mean(0) + synth.gaussian(Yf.shape[1], 0.01, 142)).astype(np.float32)
    pts = _sampled_points(nx, ny, 40, 143)
    exp.analyze(yo)
    got = exp.get_deviation()
    assert exp.sync() == 0
    assert exp.stats().eig_schedule == L.LETKF_EIG_RATIONAL
    ref = C.oracle_points(f0, Yf, yo, net, var, w.loc_radius, UV, pts)
    bg, bo, bf, worst = [], [], [], [0.0, 0.0, 0.0]
    for (x, y) in pts:
        r = ref[(x, y)]
        b_g = C.dev64(got[:, :, y, x])
        b_o = r["Xa"].T - lbm.W[None, :]
        b_f = f0[:, :, y, x].astype(np.float64) - lbm.W[None, :]
        bg.append(b_g)
        bo.append(b_o)
        bf.append(b_f)
        worst = [max(a, b) for a, b in zip(worst, C.point_parity(b_g, b_o, b_f))]
    errs = C.point_parity(np.concatenate(bg, 1), np.concatenate(bo, 1), np.concatenate(bf, 1))
    assert max(errs) < 1e-5, errs
    assert max(worst) < 5e-5, worst
    exp.close()


@pytest.mark.parametrize("k", [16, 48])
def test_points_beyond_the_approximations_go_to_the_fused_kernel(k):
    # inflation 1e12 puts the floor (k-1)/rho near 1e-11: every observed point's condition
    # bound is far above 1e6, so the schedule hands every observed point to the fused kernel
    nx = ny = 24
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=151), 1e-4, 152)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    yo = C.observations(C.ensemble_state(1, nx, ny, seed=153), net, UV, 0.01, 154)[0]
    out = {}
    for sch in (L.LETKF_EIG_RATIONAL, L.LETKF_EIG_FUSED):
        exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, infl=1e12,
                           eig_schedule=sch)
        exp.set_state(f0)
        exp.analyze(yo)
        out[sch] = exp.get_deviation()
        exp.sync()
        st = exp.stats()
        exp.close()
    assert st.n_zero_obs == 0
    # Q is numerically singular here, so both may carry non-finite values: in the same places
    assert np.array_equal(out[L.LETKF_EIG_RATIONAL], out[L.LETKF_EIG_FUSED], equal_nan=True)


def test_rational_cycle_equals_forecast_then_analysis():
    nx = ny = 40
    k = 24
    f0 = C.ensemble_state(k, nx, ny, seed=161)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    yos = [C.observations(C.ensemble_state(1, nx, ny, seed=162 + c), net, UV, 0.01, 170 + c)[0]
           for c in range(3)]
    a = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, eig_schedule=L.LETKF_EIG_RATIONAL)
    b = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, eig_schedule=L.LETKF_EIG_RATIONAL)
    a.set_state(f0)
    b.set_state(f0)
    for y in yos:
        a.cycle(5, y)
        b.forecast(5)
        b.analyze(y)
    assert np.array_equal(a.get_deviation(), b.get_deviation())
    assert a.sync() == 0 and b.sync() == 0
