"""Mixed precision (LETKF_MIXED): the tensor-core Gram path against the FP64 oracle.

For 17 <= k <= 128 the mixed form builds A = Yb^T R_loc^-1 Yb and c on the tcgen05 tensor
cores from split FP16 operands (hi + lo, ~22 significant bits) with FP32 accumulation; the
rest of the analysis is the FP32 path.  Its stated error against the oracle, per output:
  Gram matrix A, vector c            1e-5 relative L2 (measured ~1e-6)
  local observation counts            exact (integer decision on integer distances)
  eigenvalues of Q                    1e-5 of the largest
  analysis mean, mean increment,
  analysis perturbations              1e-5 relative L2 (the bar of the FP32 form)
The cases cover the three tile shapes of the kernel (k padded to 32: 4x2 points per tile,
two points per operand tile; k padded to 64: 2x2 points per tile; k padded to 128: one point
per tile), members beyond k in the padding, ragged tiles, tiles
whose candidates fill several segments, points and whole tiles without local observations,
row-chunked launches, and bitwise reproducibility.
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


def _case(k, nx, ny, stride, radius, seed, precision=L.LETKF_MIXED, obs_xy=None,
          chunk_bytes=0, obs_vars=UV):
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=seed), 1e-4, seed + 1)
    truth = C.ensemble_state(1, nx, ny, seed=seed + 7)
    net = synth.regular_obs_network(nx, ny, stride) if obs_xy is None else obs_xy
    V = bin(obs_vars).count("1")
    var = np.full(len(net) * V, 1e-4, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, obs_vars=obs_vars,
                       loc_radius=radius if math.isfinite(radius) else None,
                       precision=precision, chunk_bytes=chunk_bytes)
    yo = C.observations(truth, net, obs_vars, 0.01, seed + 9)[0]
    exp.set_state(f0)
    return exp, f0, yo, net, var


def _flat(a):
    return np.asarray(a).transpose(0, 2, 3, 1).reshape(a.shape[0], -1)


def _parity(exp, f0, yo, net, var, radius, obs_vars=UV, tol=1e-5):
    exp.analyze(yo)
    dev = C.dev64(exp.get_deviation())
    assert exp.sync() == 0
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, radius, obs_vars)
    Wb = lbm.W[None, :, None, None]
    errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), _flat(f0.astype(np.float64) - Wb))
    assert max(errs) < tol, errs
    return dev


@pytest.mark.parametrize("k,nx,ny,stride,radius", [
    (17, 22, 19, 3, 3.0),     # smallest k of the form; 15 padded members; ragged 4x2 tiles
    (24, 20, 18, 2, 2.5),     # two points per operand tile
    (32, 16, 16, 2, 3.0),     # no padding in the 32-member form
    (33, 21, 19, 3, 3.0),     # 31 padded members; ragged 2x2 tiles
    (50, 20, 20, 2, 2.5),     # k not a multiple of 4 (scalar epilogue stores)
    (64, 16, 16, 2, 3.0),     # no padding, ~110 local observation scalars
    (65, 13, 11, 3, 2.0),     # first k of the 128-member tile
    (100, 12, 12, 2, 2.0),
    (128, 12, 10, 3, 3.0),    # largest ensemble
])
def test_mixed_gram_cvec_counts_eigenvalues_match_oracle(k, nx, ny, stride, radius):
    exp, f0, yo, net, var = _case(k, nx, ny, stride, radius, seed=200 + k)
    pts = np.array(sorted({0, 1, nx - 1, nx, nx + 1, (ny // 2) * nx + nx // 2, nx * ny - 1,
                           nx * (ny - 1)}))
    pr = exp.analyze_probe(yo, pts, want=("nloc", "gram", "cvec", "eigval"))
    assert exp.sync() == 0
    ref = C.oracle_analysis(f0, yo, net, var, radius, UV,
                            points=[(p % nx, p // nx) for p in pts])[1]
    for i, p in enumerate(pts):
        r = ref[(p % nx, p // nx)]
        assert pr["nloc"][i] == r["nloc"]
        assert C.rel_l2(pr["gram"][i], r["A"]) < 1e-5, (p, C.rel_l2(pr["gram"][i], r["A"]))
        assert C.rel_l2(pr["cvec"][i], r["c"]) < 1e-5, (p, C.rel_l2(pr["cvec"][i], r["c"]))
        assert np.abs(pr["eigval"][i] - r["lam"]).max() < 1e-5 * r["lam"].max()


@pytest.mark.parametrize("k,nx,ny,stride,radius", [
    (20, 23, 17, 3, 3.0),
    (32, 18, 18, 2, 3.0),
    (48, 18, 17, 3, 3.0),
    (64, 16, 16, 2, 3.0),
    (96, 12, 12, 3, 2.5),
    (128, 10, 10, 2, 2.0),
])
def test_mixed_analysis_matches_oracle(k, nx, ny, stride, radius):
    exp, f0, yo, net, var = _case(k, nx, ny, stride, radius, seed=300 + k)
    _parity(exp, f0, yo, net, var, radius)


def test_mixed_and_fp32_forms_agree():
    outs = []
    for prec in (L.LETKF_FP32, L.LETKF_MIXED):
        exp, f0, yo, net, var = _case(64, 16, 16, 2, 3.0, seed=401, precision=prec)
        exp.analyze(yo)
        outs.append(C.dev64(exp.get_deviation()))
        assert exp.sync() == 0
    fb = C.dev64(C.to_deviation32(f0))
    errs = C.point_parity(_flat(outs[1]), _flat(outs[0]), _flat(fb))
    assert max(errs) < 1e-5, errs


def test_mixed_without_localization_spans_many_segments():
    # every observation is local to every point: 400 points x 2 variables = 800 candidate
    # slots per tile, several segments of the candidate ring
    nx = ny = 20
    exp, f0, yo, net, var = _case(64, nx, ny, 1, math.inf, seed=501)
    dev = _parity(exp, f0, yo, net, var, math.inf)
    # one global transform: the analysis perturbations of every point are X_b' dW
    assert np.isfinite(dev).all()


def test_mixed_points_and_tiles_without_observations_are_unchanged():
    nx = ny = 24
    net = np.array([[2, 2], [3, 2], [15, 4]], dtype=np.int32)
    exp, f0, yo, _, var = _case(64, nx, ny, 4, 2.0, seed=601, obs_xy=net)
    st = exp.stats()
    assert st.n_zero_obs > 0.4 * nx * ny        # whole 2x2 tiles without a candidate too
    g0 = exp.get_deviation()
    _parity(exp, f0, yo, net, var, 2.0)
    g1 = exp.get_deviation()
    assert exp.sync() == 0
    c2 = synth.loc_cutoff2(2.0)
    from oracle import letkf as oletkf
    for y in range(ny):
        for x in range(nx):
            if len(oletkf.local_obs(x, y, net, nx, ny, c2)[0]) == 0:
                assert np.array_equal(g1[:, :, y, x], g0[:, :, y, x])


def test_mixed_chunked_launches_and_repeats_are_bitwise_identical():
    outs = []
    for chunk in (0, 16 * 64 * 64 * 4 * 3, 0):   # whole grid, 3-row chunks, whole grid again
        exp, f0, yo, net, var = _case(64, 16, 16, 2, 3.0, seed=701, chunk_bytes=chunk)
        exp.analyze(yo)
        outs.append(exp.get_state())
        assert exp.sync() == 0
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


def test_mixed_full_size_workload_sampled_points_match_oracle():
    # the 1024 x 1024, k = 64 workload (obs every 4th point, r = 12) in its mixed form
    w = synth.WORKLOADS["turb1024_k64"]
    nx, ny, k = w.nx, w.ny, w.k
    f0 = C.big_ensemble_state(k, nx, ny, seed=831)
    net = w.obs_network()
    var = w.obs_error_var(len(net) * 2).astype(np.float32)
    exp = L.Experiment(nx, ny, k, w.tau, net, var, loc_radius=w.loc_radius,
                       precision=L.LETKF_MIXED)
    exp.set_state(f0)
    Yf = C.observe_at_points(f0, net, UV)
    yo = (Yf.mean(0) + synth.gaussian(Yf.shape[1], 0.01, 832)).astype(np.float32)
    rng = synth.generator(833)
    pts = {(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, ny // 2)}
    while len(pts) < 32:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    pts = sorted(pts)
    lin = np.array([y * nx + x for (x, y) in pts])
    pr = exp.analyze_probe(yo, lin, want=("nloc", "gram", "eigval"))
    got = exp.get_deviation()
    assert exp.sync() == 0
    ref = C.oracle_points(f0, Yf, yo, net, var, w.loc_radius, UV, pts)
    bg, bo, bf = [], [], []
    for i, (x, y) in enumerate(pts):
        r = ref[(x, y)]
        assert pr["nloc"][i] == r["nloc"]
        assert np.abs(pr["eigval"][i] - r["lam"]).max() < 1e-5 * r["lam"].max()
        bg.append(C.dev64(got[:, :, y, x]))
        bo.append(r["Xa"].T - lbm.W[None, :])
        bf.append(f0[:, :, y, x].astype(np.float64) - lbm.W[None, :])
    errs = C.point_parity(np.concatenate(bg, 1), np.concatenate(bo, 1), np.concatenate(bf, 1))
    assert max(errs) < 1e-5, errs
