"""Grouped analysis of co-resident ensembles (uneven batching).

Four ensembles with k = 16, 32, 64, 128 share one grid and a clustered observation network
(a dense patch observed every 2nd point over a quarter of the domain, every 8th point
elsewhere, and a band of rows without observations, so that a fifth of the points have no local
observation): local observation counts range from 0 to a few hundred scalars.  One grouped
analysis runs the eigensolve of the points of the ensembles on the fused schedule in one
persistent launch per column class, and the split kernels of those on a split schedule.
Checked:
  * each ensemble's grouped result matches the FP64 oracle's local analyses at sampled points
    (the densest, points without observations, random ones), FP32 and mixed, with every
    ensemble in the persistent launch and with a mix of fused and split ensembles;
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
# the EVD-free schedule serves k <= 64
RAT = (L.LETKF_EIG_RATIONAL, L.LETKF_EIG_RATIONAL, L.LETKF_EIG_RATIONAL, L.LETKF_EIG_FUSED)
CHEB = (L.LETKF_EIG_CHEBYSHEV, L.LETKF_EIG_CHEBYSHEV, L.LETKF_EIG_CHEBYSHEV, L.LETKF_EIG_FUSED)


@pytest.mark.parametrize("precision", [L.LETKF_FP32, L.LETKF_MIXED])
@pytest.mark.parametrize("schedule", ["fused", "split", "mix", "rational", "chebyshev", "auto"])
def test_group_analysis_equals_each_alone_analysis(precision, schedule):
    scheds = {"fused": (L.LETKF_EIG_FUSED,) * 4, "split": (L.LETKF_EIG_SPLIT,) * 4,
              "mix": MIX, "rational": RAT, "chebyshev": CHEB,
              "auto": (L.LETKF_EIG_AUTO,) * 4}[schedule]
    grouped, f0s, yos = _ensembles(precision, scheds)
    st = grouped[0].stats()
    assert 0.15 < st.n_zero_obs / st.n_points < 0.5          # a share of points sees nothing
    L.letkf_group_analyze(grouped, yos)
    picked = tuple(e.stats().eig_schedule for e in grouped)
    assert all(p in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT, L.LETKF_EIG_RATIONAL,
                     L.LETKF_EIG_CHEBYSHEV)
               for p in picked)
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


def _oracle_sample_points(net, n=32, seed=1600):
    """Sampled grid points for the oracle check: the densest local networks, points without
    local observations and seeded random ones."""
    from oracle import letkf as oletkf
    c2 = synth.loc_cutoff2(2.0)
    counts = {(x, y): len(oletkf.local_obs(x, y, net, NX, NY, c2)[0])
              for y in range(NY) for x in range(NX)}
    order = sorted(counts, key=lambda p: (-counts[p], p))
    pts = set(order[:8]) | set([p for p in order if counts[p] == 0][:6])
    rng = synth.generator(seed)
    while len(pts) < n:
        pts.add((int(rng.integers(NX)), int(rng.integers(NY))))
    return sorted(pts), counts


@pytest.mark.parametrize("precision", [L.LETKF_FP32, L.LETKF_MIXED])
@pytest.mark.parametrize("schedule", ["fused", "mix", "rational", "chebyshev"])
def test_group_analysis_matches_oracle_at_sampled_points(precision, schedule):
    # The grouped analysis (the persistent launch over all fused-schedule ensembles, split
    # kernels for the others) of the k = 16/32/64/128 ensembles on the clustered network,
    # each checked against the FP64 oracle's local analyses (Algorithm 1 per point) at the
    # densest points, at points without observations and at random points, to the parity
    # tests' 1e-5 relative L2 on the mean, the mean increment and the perturbations.
    from oracle import lbm, obs as oobs
    scheds = {"fused": (L.LETKF_EIG_FUSED,) * 4, "mix": MIX, "rational": RAT,
              "chebyshev": CHEB}[schedule]
    grouped, f0s, yos = _ensembles(precision, scheds)
    L.letkf_group_analyze(grouped, yos)
    net = _network()
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    pts, counts = _oracle_sample_points(net)
    assert max(counts.values()) > 40 and min(counts[p] for p in pts) == 0
    for g, f0, yo in zip(grouped, f0s, yos):
        got = g.get_deviation()
        assert g.sync() == 0
        Yf = oobs.observe(f0.astype(np.float64), net, UV)
        ref = C.oracle_points(f0, Yf, yo, net, var, 2.0, UV, pts)
        bg, bo, bf, worst = [], [], [], [0.0, 0.0, 0.0]
        for (x, y) in pts:
            r = ref[(x, y)]
            b_g = C.dev64(got[:, :, y, x])
            b_o = r["Xa"].T - lbm.W[None, :]
            b_f = f0[:, :, y, x].astype(np.float64) - lbm.W[None, :]
            if r["nloc"] == 0:
                assert np.array_equal(got[:, :, y, x],
                                      C.to_deviation32(f0[:, :, y, x][:, :, None, None])[:, :, 0, 0])
                continue
            bg.append(b_g)
            bo.append(b_o)
            bf.append(b_f)
            # per point: the mean and the perturbations relative to themselves; the increment
            # relative to the larger of itself and the analysis spread (a point whose few,
            # distant observations nearly cancel in c has a tiny increment, whose own relative
            # error says nothing about the analysis)
            mg, mo, mf = b_g.mean(0), b_o.mean(0), b_f.mean(0)
            spread = np.linalg.norm(b_o - mo) / np.sqrt(b_o.shape[0])
            inc = np.linalg.norm((mg - mf) - (mo - mf)) / max(np.linalg.norm(mo - mf), spread)
            e = C.point_parity(b_g, b_o, b_f)
            worst = [max(worst[0], e[0]), max(worst[1], inc), max(worst[2], e[2])]
        errs = C.point_parity(np.concatenate(bg, 1), np.concatenate(bo, 1), np.concatenate(bf, 1))
        assert max(errs) < 1e-5, (g.k, errs)
        assert max(worst) < 5e-5, (g.k, worst)


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
    assert all(p in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT, L.LETKF_EIG_RATIONAL,
                     L.LETKF_EIG_CHEBYSHEV)
               for p in picked)
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


def test_sixteen_small_ensembles_in_one_group():
    # the largest group: 16 handles of mixed k on small grids, every one on the FUSED
    # schedule, so the eigensolve of all their points is one persistent launch per column
    # class; each grouped result equals its own analysis bit for bit; 17 handles are rejected
    nx = ny = 20
    ks = (16, 24, 32, 40, 48, 56, 64, 20) * 2
    net = _network(nx, ny)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)

    def build():
        exps, f0s, yos = [], [], []
        for i, k in enumerate(ks):
            f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=1800 + i), 1e-4,
                                          1850 + i)
            e = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.0,
                             eig_schedule=L.LETKF_EIG_FUSED)
            e.set_state(f0)
            exps.append(e)
            f0s.append(f0)
            yos.append(C.observations(C.ensemble_state(1, nx, ny, seed=1900 + i), net, UV,
                                      0.01, 1950 + i)[0])
        return exps, f0s, yos

    grouped, _, yos = build()
    L.letkf_group_analyze(grouped, yos)
    alone, _, _ = build()
    for e, y in zip(alone, yos):
        e.analyze(y)
    for g, a in zip(grouped, alone):
        assert np.array_equal(g.get_deviation(), a.get_deviation())
        assert g.sync() == 0 and a.sync() == 0
    extra = L.Experiment(nx, ny, 8, 0.6, net, var, loc_radius=2.0)
    with pytest.raises(L.LetkfError):
        L.letkf_group_analyze(grouped + [extra], yos + [yos[0]])
