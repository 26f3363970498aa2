"""Grouped analysis of co-resident ensembles (uneven batching).

Four ensembles with k = 16, 32, 64, 128 share one grid and a clustered observation network
(a dense patch observed every 2nd point over a quarter of the domain, every 8th point
elsewhere, and a band of rows without observations, so that a fifth of the points have no local
observation): local observation counts range from 0 to a few hundred scalars.  One grouped
analysis runs the eigensolve of the points of the ensembles on the fused schedule in one
persistent launch per column class, and the split kernels of those on a split schedule.
Checked:
  * each ensemble's grouped result is bit for bit its own letkf_analyze on the same schedule
    (which the parity tests pin to the oracle), in FP32 and in the mixed form, with every
    ensemble fused, every one split, a mix, and AUTO (each picks at the first group analysis);
  * points without local observations are left untouched;
  * the graph-captured group cycle equals the forecasts followed by the grouped analysis, for
    odd and even step counts and on replay; with AUTO handles the first group cycle picks the
    schedules without capture and the later ones replay a graph;
  * invalid groups are rejected.
"""
import numpy as np
import pytest

import synth
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

UV = L.LETKF_OBS_U | L.LETKF_OBS_V
NX = NY = 48
KS = (16, 32, 64, 128)


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _network(nx=NX, ny=NY):
    return synth.clustered_obs_network(nx, ny, 2, 8, patch=(4, 4, nx // 2, ny // 2),
                                       empty_band=(30, 14))


def _ensembles(precision, schedules=(L.LETKF_EIG_AUTO,) * 4, nx=NX, ny=NY):
    net = _network(nx, ny)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    exps, f0s, yos = [], [], []
    for i, k in enumerate(KS):
        f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=1200 + i), 1e-4, 1300 + i)
        e = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.0, precision=precision,
                         eig_schedule=schedules[i])
        e.set_state(f0)
        truth = C.ensemble_state(1, nx, ny, seed=1400 + i)
        exps.append(e)
        f0s.append(f0)
        yos.append(C.observations(truth, net, UV, 0.01, 1500 + i)[0])
    return exps, f0s, yos


MIX = (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT, L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT)


@pytest.mark.parametrize("precision", [L.LETKF_FP32, L.LETKF_MIXED])
@pytest.mark.parametrize("schedule", ["fused", "split", "mix", "auto"])
def test_group_analysis_equals_each_alone_analysis(precision, schedule):
    scheds = {"fused": (L.LETKF_EIG_FUSED,) * 4, "split": (L.LETKF_EIG_SPLIT,) * 4,
              "mix": MIX, "auto": (L.LETKF_EIG_AUTO,) * 4}[schedule]
    grouped, f0s, yos = _ensembles(precision, scheds)
    st = grouped[0].stats()
    assert 0.15 < st.n_zero_obs / st.n_points < 0.5          # a share of points sees nothing
    L.letkf_group_analyze(grouped, yos)
    picked = tuple(e.stats().eig_schedule for e in grouped)
    assert all(p in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT) for p in picked)
    if schedule != "auto":
        assert picked == scheds
    alone, _, _ = _ensembles(precision, picked)
    for e, y in zip(alone, yos):
        e.analyze(y)
    for g, a, f0 in zip(grouped, alone, f0s):
        got, ref = g.get_deviation(), a.get_deviation()
        assert g.sync() == 0 and a.sync() == 0
        assert np.array_equal(got, ref)
        # points without local observations keep their forecast
        assert not np.array_equal(got, C.to_deviation32(f0))


def test_points_without_observations_are_untouched_in_the_group():
    grouped, f0s, yos = _ensembles(L.LETKF_FP32)
    L.letkf_group_analyze(grouped, yos)
    from oracle import letkf as oletkf
    net = _network()
    c2 = synth.loc_cutoff2(2.0)
    far = [(x, y) for y in range(NY) for x in range(NX)
           if len(oletkf.local_obs(x, y, net, NX, NY, c2)[0]) == 0]
    assert len(far) > 0.15 * NX * NY
    for g, f0 in zip(grouped, f0s):
        got = g.get_deviation()
        ref = C.to_deviation32(f0)
        for (x, y) in far[::7]:
            assert np.array_equal(got[:, :, y, x], ref[:, :, y, x])


@pytest.mark.parametrize("nsteps", [3, 4])
def test_group_cycle_equals_forecast_then_group_analysis(nsteps):
    a, _, yos = _ensembles(L.LETKF_FP32, MIX)
    b, _, _ = _ensembles(L.LETKF_FP32, MIX)
    for c in range(3):                       # capture, then replays (buffer parity flips)
        L.letkf_group_cycle(a, nsteps, yos)
        for e in b:
            e.forecast(nsteps)
        L.letkf_group_analyze(b, yos)
    for x, y in zip(a, b):
        assert np.array_equal(x.get_deviation(), y.get_deviation())
        assert x.sync() == 0 and y.sync() == 0


def test_group_cycle_with_auto_handles_picks_then_captures():
    # AUTO handles pick at the first group cycle, which therefore runs without capture; the
    # later ones replay a graph; all equal group cycles of handles fixed to the same picks
    # a 46 x 46 grid: a chunk size (and so an autotuner key) no other test uses
    a, _, yos = _ensembles(L.LETKF_FP32, nx=46, ny=46)
    assert all(e.stats().eig_schedule == L.LETKF_EIG_AUTO for e in a)
    L.letkf_group_cycle(a, 3, yos)
    assert a[0].stats().cycle_kernels == 0
    picked = tuple(e.stats().eig_schedule for e in a)
    assert all(p in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT) for p in picked)
    b, _, _ = _ensembles(L.LETKF_FP32, picked, nx=46, ny=46)
    L.letkf_group_cycle(b, 3, yos)
    for _ in range(2):
        L.letkf_group_cycle(a, 3, yos)
        L.letkf_group_cycle(b, 3, yos)
    assert a[0].stats().cycle_kernels > 0
    for x, y in zip(a, b):
        assert np.array_equal(x.get_deviation(), y.get_deviation())
        assert x.sync() == 0 and y.sync() == 0


def test_invalid_groups_are_rejected():
    exps, _, yos = _ensembles(L.LETKF_FP32)
    with pytest.raises(L.LetkfError):
        L.letkf_group_analyze([exps[0], exps[0]], yos[:2])   # a handle twice
    with pytest.raises(L.LetkfError):
        L.letkf_group_analyze([], [])
