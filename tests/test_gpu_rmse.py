"""Longer runs, judged by RMSE against the synthetic truth (OSSE, Sec. V).

Truth: a decaying 2D flow on 96 x 96 (tau 0.55) from a seeded divergence-free random velocity
field (wavenumbers 2-5, RMS 0.02).  Ensemble (k = 40, so the mixed form builds the Gram
matrices on the tensor cores): truth + a common error field + per-member perturbations
(both divergence-free, RMS 0.005), so the ensemble mean is wrong by about the ensemble
spread.  Every 25 steps the truth is observed ((u, v) every 4th point, sigma 1e-3) and the
ensemble assimilates the noisy observations; a free ensemble from the same start runs without
assimilation.  The velocity RMSE of the ensemble mean against the truth must

  * drop at every analysis (analysis below the forecast of the same cycle: on average and in
    at least 90 % of the cycles),
  * end well below the free run's (a factor 3 over the last 10 of 30 cycles),
and the mixed-precision form must track the FP32 form (the same RMSE within 5 %).
"""
import numpy as np
import pytest

import synth
from oracle import lbm
from paper_2308_03310_gb300 import _build, letkf as L

pytestmark = pytest.mark.gpu

NX = NY = 96
K = 40
TAU = 0.55
STEPS = 25
CYCLES = 30
SIGMA = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _velocity_rmse(f_members, f_truth):
    _, ux, uy = lbm.moments(f_members.astype(np.float64))
    _, tx, ty = lbm.moments(f_truth.astype(np.float64))
    return float(np.sqrt(np.mean((ux.mean(0) - tx) ** 2 + (uy.mean(0) - ty) ** 2)))


def _field(rms, seed):
    """Divergence-free random velocity field (wavenumbers 2..5) with the given RMS."""
    return synth.band_limited_force(NX, NY, 2.0, 5.0, rms, seed)


def _osse(precision):
    net = synth.regular_obs_network(NX, NY, 4)
    LV = len(net) * 2
    var = np.full(LV, SIGMA ** 2, dtype=np.float32)
    # members + the truth (auxiliary member, advanced but never analysed)
    da = L.Experiment(NX, NY, K, TAU, net, var, n_aux=1, precision=precision, loc_radius=6.0)
    free = L.Experiment(NX, NY, K, TAU, net, var, n_aux=1, precision=precision, loc_radius=6.0)
    tx, ty = _field(0.02, 7001)
    ex, ey = _field(0.005, 7002)
    ux = np.empty((K + 1, NY, NX))
    uy = np.empty((K + 1, NY, NX))
    for m in range(K):
        px, py = _field(0.005, 7100 + m)
        ux[m], uy[m] = tx + ex + px, ty + ey + py
    ux[K], uy[K] = tx, ty
    rho = np.ones((K + 1, NY, NX), np.float32)
    for e in (da, free):
        e.set_macro(rho, ux.astype(np.float32), uy.astype(np.float32))
    fc, an, fr = [], [], []
    for c in range(CYCLES):
        da.forecast(STEPS)
        free.forecast(STEPS)
        y_truth = da.get_obs()[K]                   # h(x) of the truth
        yo = (y_truth + synth.gaussian(LV, SIGMA, 7500 + c)).astype(np.float32)
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


def test_assimilation_beats_the_free_run(runs):
    fc, an, fr = runs[L.LETKF_FP32]
    late = slice(CYCLES - 10, CYCLES)
    assert an[late].mean() < fr[late].mean() / 3, (an[late].mean(), fr[late].mean())


def test_mixed_precision_tracks_fp32_in_rmse(runs):
    an32 = runs[L.LETKF_FP32][1]
    anmx = runs[L.LETKF_MIXED][1]
    late = slice(CYCLES - 10, CYCLES)
    rel = abs(anmx[late].mean() - an32[late].mean()) / an32[late].mean()
    print("late analysis RMSE fp32", an32[late].mean(), "mixed", anmx[late].mean())
    assert rel < 0.05, rel
