"""The paper's own LETKF workloads (Sec. V) against the FP64 oracle.

Both observe rho, u and v (V = 3) of a 128 x 128 D2Q9 flow with ensembles of M = 4, 16 and 64:
  * dense (Sec. V-A): every grid point observed and only its own observation local
    (l_max = 1: the cutoff admits d = 0 alone);
  * sparse (Sec. V-B): observations every 4th point (L = 32^2), Gaspari-Cohn localization with
    the cutoff distance 2 (p - 1) = 6 cells (support 2c = 6, so c = 3 and r = c / sqrt(10/3)).
Observation errors are 20 % of each observed variable's fluctuation (the paper's "~20 %
Gaussian observation noise", read per variable).  Checked at sampled grid points: the local
observation counts exactly, the analysis mean, mean increment and perturbations at the
parity bar (1e-5 relative L2), FP32 and mixed, on the schedule AUTO picks.
"""
import math

import numpy as np
import pytest

import synth
from oracle import lbm, obs as oobs
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

RUV = L.LETKF_OBS_RHO | L.LETKF_OBS_U | L.LETKF_OBS_V
N = 128


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _ensemble(k, seed):
    """FP32 f of k members: a band-limited flow (RMS 0.03) with N(0, 0.005^2) velocity and
    N(0, 0.002^2) density perturbations, equilibria from the oracle.  The density fluctuations
    are of the size the weakly compressible D2Q9 flow itself has at these speeds
    (rho - 1 ~ u^2 / c_s^2 = 3 u^2 ~ 3e-3)."""
    tx, ty = synth.band_limited_force(N, N, 2.0, 6.0, 0.03, seed)
    rho = 1.0 + synth.gaussian((k, N, N), 2e-3, seed + 1)
    ux = tx[None] + synth.gaussian((k, N, N), 0.005, seed + 2)
    uy = ty[None] + synth.gaussian((k, N, N), 0.005, seed + 3)
    return lbm.equilibrium(rho, ux, uy).astype(np.float32), (tx, ty)


def _setup(case, k, seed):
    f0, (tx, ty) = _ensemble(k, seed)
    stride = 1 if case == "dense" else 4
    net = synth.regular_obs_network(N, N, stride)
    truth = lbm.equilibrium(1.0 + synth.gaussian((N, N), 2e-3, seed + 4), tx, ty)
    ytrue = oobs.observe(truth, net, RUV)
    # 20 % of each variable's fluctuation: rho about 1, u and v about 0
    sig = 0.2 * np.array([np.std(ytrue[0::3] - 1.0), np.std(ytrue[1::3]), np.std(ytrue[2::3])])
    var = np.tile(sig ** 2, len(net)).astype(np.float32)
    yo = (ytrue + np.tile(sig, len(net)) * synth.gaussian(ytrue.shape, 1.0, seed + 5))
    if case == "dense":
        loc = dict(loc_radius=1.0, loc_cutoff2=1.0, loc_kind=L.LETKF_LOC_GAUSS)
        oloc = dict(radius=1.0, cutoff2=1.0, kind="gauss")
    else:
        r = 3.0 / math.sqrt(10.0 / 3.0)
        loc = dict(loc_radius=r, loc_cutoff2=36.0, loc_kind=L.LETKF_LOC_GC)
        oloc = dict(radius=r, cutoff2=36.0, kind="gc")
    return f0, net, var, yo.astype(np.float32), loc, oloc


@pytest.mark.parametrize("case", ["dense", "sparse"])
@pytest.mark.parametrize("k", [4, 16, 64])
@pytest.mark.parametrize("precision", [L.LETKF_FP32, L.LETKF_MIXED])
def test_paper_workload_matches_oracle_at_sampled_points(case, k, precision):
    from oracle import letkf as oletkf
    f0, net, var, yo, loc, oloc = _setup(case, k, 1700 + k)
    exp = L.Experiment(N, N, k, 0.52, net, var, obs_vars=RUV, precision=precision, **loc)
    exp.set_state(f0)
    st = exp.stats()
    assert st.max_local_obs == (1 if case == "dense" else 9)
    exp.analyze(yo)
    got = exp.get_deviation()
    assert exp.sync() == 0
    Yf = C.observe_at_points(f0, net, RUV)
    ybar, dY = oobs.ensemble_obs(Yf)
    rng = synth.generator(1750 + k)
    pts = sorted({(0, 0), (N - 1, N - 1), (5, 7)} |
                 {(int(rng.integers(N)), int(rng.integers(N))) for _ in range(24)})
    bg, bo, bf = [], [], []
    for (x, y) in pts:
        dYl, dl, rl, nloc = oletkf.point_inputs(x, y, Yf, yo.astype(np.float64), net,
                                                var.astype(np.float64), N, N, oloc["radius"],
                                                oloc["cutoff2"], RUV, ybar=ybar, dY=dY,
                                                loc=oloc["kind"])
        res = oletkf.local_analysis(f0[:, :, y, x].astype(np.float64).T, dYl, dl, rl)
        bg.append(C.dev64(got[:, :, y, x]))
        bo.append(res["Xa"].T - lbm.W[None, :])
        bf.append(f0[:, :, y, x].astype(np.float64) - lbm.W[None, :])
    errs = C.point_parity(np.concatenate(bg, 1), np.concatenate(bo, 1), np.concatenate(bf, 1))
    assert max(errs) < 1e-5, errs
    exp.close()
