"""Longer chaotic runs, judged by RMSE against the synthetic truth (OSSE, Sec. V).

A forced 2D turbulence nature run on 96 x 96 (tau 0.52, Kolmogorov + band-limited forcing)
is spun up together with an ensemble of k = 40 perturbed copies (k > 32, so the mixed form
builds the Gram matrices on the tensor cores).  Then every 25 steps the nature run is
observed ((u, v) every 4th point, sigma 0.01) and the ensemble assimilates the noisy
observations; a free ensemble from the same start runs without assimilation.  The
velocity RMSE of the ensemble mean against the truth must

  * drop at every analysis (analysis RMSE below the forecast RMSE of the same cycle, in the
    cycle average and in at least 90 % of the cycles),
  * settle well below the free run's (a factor 2 after 30 cycles),
  * settle below the observation error,
and the mixed-precision form must track the FP32 form (same RMSE within 10 %: the runs are
chaotic, so the trajectories are compared by their error statistics, not pointwise).
"""
import numpy as np
import pytest

import synth
from oracle import lbm
from paper_2308_03310_gb300 import _build, letkf as L

pytestmark = pytest.mark.gpu

NX = NY = 96
K = 40
TAU = 0.52
STEPS = 25
CYCLES = 30
SIGMA = 0.01


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _velocity_rmse(f_members, f_truth):
    _, ux, uy = lbm.moments(f_members.astype(np.float64))
    _, tx, ty = lbm.moments(f_truth.astype(np.float64))
    return float(np.sqrt(np.mean((ux.mean(0) - tx) ** 2 + (uy.mean(0) - ty) ** 2)))


def _osse(precision):
    w = synth.Workload(name="rmse96", nx=NX, ny=NY, k=K, tau=TAU, obs_stride=4,
                       obs_sigma=SIGMA, loc_radius=6.0, steps_per_cycle=STEPS, cycles=CYCLES,
                       init="turbulence", truth_noise=1e-3, kolmogorov_amp=1e-5,
                       kolmogorov_n=4, random_rms=1e-5, spinup=3000, seed=4242)
    net = w.obs_network()
    var = w.obs_error_var(len(net) * 2).astype(np.float32)
    fx, fy = w.force()
    force = np.stack([fx, fy]).astype(np.float32)
    kw = dict(loc_radius=w.loc_radius, force=force)
    # members + the nature run (auxiliary member, advanced but never analysed)
    da = L.Experiment(NX, NY, K, TAU, net, var, n_aux=1, precision=precision, **kw)
    free = L.Experiment(NX, NY, K, TAU, net, var, n_aux=1, precision=precision, **kw)
    ux0, uy0 = w.truth_velocity()
    dux, duy = w.member_perturbations()
    rho = np.ones((K + 1, NY, NX), np.float32)
    ux = np.concatenate([ux0[None] + dux, ux0[None]]).astype(np.float32)
    uy = np.concatenate([uy0[None] + duy, uy0[None]]).astype(np.float32)
    for e in (da, free):
        e.set_macro(rho, ux, uy)
        e.forecast(w.spinup)
    LV = len(net) * 2
    fc, an, fr = [], [], []
    for c in range(CYCLES):
        da.forecast(STEPS)
        free.forecast(STEPS)
        y_truth = da.get_obs()[K]                   # the nature run's h(x)
        yo = (y_truth + w.obs_noise(c, LV)).astype(np.float32)
        f = da.get_state()
        fc.append(_velocity_rmse(f[:K], f[K]))
        da.analyze(yo)
        f = da.get_state()
        an.append(_velocity_rmse(f[:K], f[K]))
        g = free.get_state()
        fr.append(_velocity_rmse(g[:K], g[K]))
    assert da.sync() == 0 and free.sync() == 0
    return np.array(fc), np.array(an), np.array(fr)


@pytest.fixture(scope="module")
def runs():
    return {p: _osse(p) for p in (L.LETKF_FP32, L.LETKF_MIXED)}


def test_analysis_reduces_error_every_cycle(runs):
    fc, an, fr = runs[L.LETKF_FP32]
    print("forecast RMSE", np.round(fc, 5), "\nanalysis RMSE", np.round(an, 5),
          "\nfree RMSE", np.round(fr, 5))
    assert an.mean() < fc.mean()
    assert np.mean(an < fc) >= 0.9


def test_assimilation_beats_the_free_run_and_the_observation_error(runs):
    fc, an, fr = runs[L.LETKF_FP32]
    late = slice(CYCLES - 10, CYCLES)
    assert an[late].mean() < 0.5 * fr[late].mean(), (an[late].mean(), fr[late].mean())
    assert an[late].mean() < SIGMA


def test_mixed_precision_tracks_fp32_in_rmse(runs):
    an32 = runs[L.LETKF_FP32][1]
    anmx = runs[L.LETKF_MIXED][1]
    late = slice(CYCLES - 10, CYCLES)
    rel = abs(anmx[late].mean() - an32[late].mean()) / an32[late].mean()
    print("late analysis RMSE fp32", an32[late].mean(), "mixed", anmx[late].mean())
    assert rel < 0.10, rel
