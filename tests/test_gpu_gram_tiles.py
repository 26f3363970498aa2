"""The FP32 Gram's two tile schedules for k >= 17 and their autotuner (LETKF_GRAM_*).

PIPE runs one CTA per SM over 7 x 2 points (8 x 6 at k <= 32, 3 x 1 at k <= 128) with
per-point compacted entries and cp.async double buffering; TEAM runs two CTAs per SM over 4 x 2
points with the chunk's weights in shared memory.  Checked:
  * both schedules' analyses match the FP64 oracle at every grid point (1e-5 relative L2) and
    their Gram matrices agree with each other to FP32 rounding, k = 24, 48, 100;
  * AUTO resolves at the first analysis to one of the two, and a handle configured with that
    schedule computes the same bits;
  * a cycle on AUTO runs eagerly the first time and is captured the second.
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


def _flat(a):
    return np.asarray(a).transpose(0, 2, 3, 1).reshape(a.shape[0], -1)


def _case(k, nx, ny, seed):
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=seed), 1e-4, seed + 1)
    net = synth.regular_obs_network(nx, ny, 3)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    yo = C.observations(C.ensemble_state(1, nx, ny, seed=seed + 2), net, UV, 0.01, seed + 3)[0]
    return f0, net, var, yo


def _analyze(f0, net, var, yo, k, nx, ny, tile, pts):
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.5, gram_tile=tile,
                       eig_schedule=L.LETKF_EIG_FUSED)
    exp.set_state(f0)
    pr = exp.analyze_probe(yo, pts, want=("gram",))
    dev = exp.get_deviation()
    assert exp.sync() == 0
    st = exp.stats()
    exp.close()
    return dev, pr["gram"], st


@pytest.mark.parametrize("k,nx,ny", [(24, 26, 20), (48, 22, 16), (100, 12, 10)])
def test_both_tile_schedules_match_oracle_and_each_other(k, nx, ny):
    f0, net, var, yo = _case(k, nx, ny, 700 + k)
    pts = np.array([0, nx * ny // 2 + 3, nx * ny - 1])
    out = {}
    for tile in (L.LETKF_GRAM_PIPE, L.LETKF_GRAM_TEAM):
        dev, gram, st = _analyze(f0, net, var, yo, k, nx, ny, tile, pts)
        assert st.gram_tile == tile
        out[tile] = (dev, gram)
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, 2.5, UV)
    Wb = lbm.W[None, :, None, None]
    fb = _flat(f0.astype(np.float64) - Wb)
    for tile, (dev, _) in out.items():
        errs = C.point_parity(_flat(C.dev64(dev)), _flat(Xa_ref - Wb), fb)
        assert max(errs) < 1e-5, (tile, errs)
    ga, gb = out[L.LETKF_GRAM_PIPE][1], out[L.LETKF_GRAM_TEAM][1]
    assert np.abs(ga - gb).max() <= 1e-6 * np.abs(ga).max()


def test_auto_picks_a_schedule_and_computes_its_bits():
    k, nx, ny = 40, 30, 24
    f0, net, var, yo = _case(k, nx, ny, 811)
    pts = np.array([5, 300])
    dev_a, gram_a, st = _analyze(f0, net, var, yo, k, nx, ny, L.LETKF_GRAM_AUTO, pts)
    assert st.gram_tile in (L.LETKF_GRAM_PIPE, L.LETKF_GRAM_TEAM)
    dev_b, gram_b, st_b = _analyze(f0, net, var, yo, k, nx, ny, st.gram_tile, pts)
    assert np.array_equal(dev_a, dev_b) and np.array_equal(gram_a, gram_b)
    # a later AUTO handle of the same shape takes the process' pick at letkf_init
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.5, eig_schedule=L.LETKF_EIG_FUSED)
    assert exp.stats().gram_tile == st.gram_tile
    exp.close()


def test_auto_cycle_runs_eagerly_first_then_captures():
    k, nx, ny = 36, 28, 22
    f0, net, var, yo = _case(k, nx, ny, 911)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.5, gram_tile=L.LETKF_GRAM_AUTO,
                       eig_schedule=L.LETKF_EIG_FUSED)
    exp.set_state(f0)
    exp.cycle(4, yo)
    first = exp.stats()
    exp.cycle(4, yo)
    second = exp.stats()
    assert exp.sync() == 0
    exp.close()
    assert first.gram_tile in (L.LETKF_GRAM_PIPE, L.LETKF_GRAM_TEAM)
    assert first.cycle_kernels == 0 and second.cycle_kernels > 0


def test_mixed_and_small_ensembles_report_their_fixed_gram():
    net = synth.regular_obs_network(16, 16, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    a = L.Experiment(16, 16, 48, 0.6, net, var, loc_radius=2.0, precision=L.LETKF_MIXED)
    b = L.Experiment(16, 16, 12, 0.6, net, var, loc_radius=2.0)
    assert a.stats().gram_tile == L.LETKF_GRAM_TENSOR
    assert b.stats().gram_tile == L.LETKF_GRAM_TEAM
    a.close()
    b.close()
