"""Gaspari-Cohn localization (the paper's choice, Sec. II-B) on the GPU against the oracle.

LETKF_LOC_GC weights an observation at distance d by GC(d / c), c = sqrt(10/3) r, the
fifth-order piecewise rational function of Gaspari & Cohn (1999, Eq. 4.10), zero from d = 2c
on (the Gaussian form's default cutoff, so the local observation sets are the same).  Checked
against the oracle, which the CPU tests pin to the 3D self-convolution of a cone:
  * the localized Gram matrix, c, the local counts and the eigenvalues at sampled points, in
    the FP32 form and in the mixed form (sqrt(GC) on the tensor-core path);
  * the whole analysis (mean, mean increment, perturbations) at the 1e-5 bar;
  * the Gaspari-Cohn analysis differs from the Gaussian one (the weights are really used).
"""
import math

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


def _case(k, nx, ny, stride, radius, seed, precision, loc_kind=L.LETKF_LOC_GC):
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=seed), 1e-4, seed + 1)
    truth = C.ensemble_state(1, nx, ny, seed=seed + 7)
    net = synth.regular_obs_network(nx, ny, stride)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=radius, precision=precision,
                       loc_kind=loc_kind)
    yo = C.observations(truth, net, UV, 0.01, seed + 9)[0]
    exp.set_state(f0)
    return exp, f0, yo, net, var


def _flat(a):
    return np.asarray(a).transpose(0, 2, 3, 1).reshape(a.shape[0], -1)


CASES = [
    (8, 32, 32, 4, 3.0, L.LETKF_FP32),     # the single-cycle shape
    (32, 24, 22, 4, 4.0, L.LETKF_FP32),
    (40, 21, 19, 3, 3.0, L.LETKF_MIXED),   # tensor-core Gram, ragged tiles
    (64, 16, 16, 2, 3.0, L.LETKF_MIXED),
    (128, 12, 10, 3, 3.0, L.LETKF_MIXED),
]


@pytest.mark.parametrize("k,nx,ny,stride,radius,precision", CASES)
def test_gc_gram_cvec_counts_eigenvalues_match_oracle(k, nx, ny, stride, radius, precision):
    exp, f0, yo, net, var = _case(k, nx, ny, stride, radius, 400 + k, precision)
    pts = np.array(sorted({0, 1, nx - 1, nx + 1, (ny // 2) * nx + nx // 2, nx * ny - 1}))
    pr = exp.analyze_probe(yo, pts, want=("nloc", "gram", "cvec", "eigval"))
    assert exp.sync() == 0
    ref = C.oracle_analysis(f0, yo, net, var, radius, UV, loc="gc",
                            points=[(p % nx, p // nx) for p in pts])[1]
    for i, p in enumerate(pts):
        r = ref[(p % nx, p // nx)]
        assert pr["nloc"][i] == r["nloc"]
        assert C.rel_l2(pr["gram"][i], r["A"]) < 1e-5, (p, C.rel_l2(pr["gram"][i], r["A"]))
        assert C.rel_l2(pr["cvec"][i], r["c"]) < 1e-5, (p, C.rel_l2(pr["cvec"][i], r["c"]))
        assert np.abs(pr["eigval"][i] - r["lam"]).max() < 1e-5 * r["lam"].max()


@pytest.mark.parametrize("k,nx,ny,stride,radius,precision", CASES)
def test_gc_analysis_matches_oracle(k, nx, ny, stride, radius, precision):
    exp, f0, yo, net, var = _case(k, nx, ny, stride, radius, 500 + k, precision)
    exp.analyze(yo)
    dev = C.dev64(exp.get_deviation())
    assert exp.sync() == 0
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, radius, UV, loc="gc")
    Wb = lbm.W[None, :, None, None]
    errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), _flat(f0.astype(np.float64) - Wb))
    assert max(errs) < 1e-5, errs


def test_gc_and_gaussian_analyses_differ():
    out = []
    for kind in (L.LETKF_LOC_GC, L.LETKF_LOC_GAUSS):
        exp, f0, yo, net, var = _case(16, 24, 24, 4, 3.0, 601, L.LETKF_FP32, kind)
        exp.analyze(yo)
        out.append(C.dev64(exp.get_deviation()))
        assert exp.sync() == 0
    f = C.dev64(C.to_deviation32(f0))
    inc = [o - f for o in out]
    assert C.rel_l2(inc[0], inc[1]) > 1e-3


def test_gc_needs_a_radius():
    net = synth.regular_obs_network(8, 8, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    with pytest.raises(L.LetkfError):
        L.Experiment(8, 8, 4, 0.6, net, var, loc_radius=0.0, loc_kind=L.LETKF_LOC_GC)
