"""The eigensolve schedules against the FP64 oracle and against each other.

FUSED runs every phase of a point's analysis in one warp; SPLIT runs the tridiagonalization
(warp per point), the QL recurrence (thread per point, rotations recorded) and the replay,
back-transform and update (warp per point) as three launches; SPLIT_CHECK is SPLIT with a
rotation record of one sweep, so that nearly every point is handed back to the fused kernel,
which recomputes it from the Gram matrix the split kernels left intact; RATIONAL (k <= 64)
forms no eigenvectors (tridiagonal solves and a rational approximation of Q^-1/2), its
probe eigenvalues come from an eigenvalue-only QL; CHEBYSHEV (k <= 64) applies polynomial
approximations of Q^-1/2 and Q^-1, passing ill-conditioned points to RATIONAL.  All of them must meet
the analysis bar (1e-5 relative L2 on mean, mean increment and perturbations) and SPLIT must
agree with FUSED to within FP32 rounding of the two summation orders.
"""
import numpy as np
import pytest

import synth
from oracle import lbm
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

UV = L.LETKF_OBS_U | L.LETKF_OBS_V
SCHEDULES = [L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT, L.LETKF_EIG_SPLIT_CHECK, L.LETKF_EIG_RATIONAL,
             L.LETKF_EIG_CHEBYSHEV]
EVD_FREE = (L.LETKF_EIG_RATIONAL, L.LETKF_EIG_CHEBYSHEV)   # k <= 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _flat(a):
    return np.asarray(a).transpose(0, 2, 3, 1).reshape(a.shape[0], -1)


def _run(k, nx, ny, stride, radius, seed, schedule, precision=L.LETKF_FP32):
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=seed), 1e-4, seed + 1)
    truth = C.ensemble_state(1, nx, ny, seed=seed + 7)
    net = synth.regular_obs_network(nx, ny, stride)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=radius, precision=precision,
                       eig_schedule=schedule)
    yo = C.observations(truth, net, UV, 0.01, seed + 9)[0]
    exp.set_state(f0)
    pts = np.array([0, nx * ny // 2 + nx // 3, nx * ny - 1])
    pr = exp.analyze_probe(yo, pts, want=("eigval",))
    dev = C.dev64(exp.get_deviation())
    assert exp.sync() == 0
    return f0, yo, net, var, dev, pr["eigval"], pts


@pytest.mark.parametrize("k,nx,ny,stride,radius", [
    (5, 14, 12, 3, 2.5),
    (16, 16, 16, 4, 3.0),
    (32, 20, 18, 4, 3.0),
    (64, 14, 14, 2, 3.0),
    (100, 10, 10, 2, 2.0),
    (128, 10, 9, 3, 2.5),
])
def test_schedules_match_oracle_and_each_other(k, nx, ny, stride, radius):
    outs = {}
    for sch in SCHEDULES:
        if sch in EVD_FREE and k > 64:
            continue
        f0, yo, net, var, dev, lam, pts = _run(k, nx, ny, stride, radius, 900 + k, sch)
        outs[sch] = (dev, lam)
    Xa_ref, ref = C.oracle_analysis(f0, yo, net, var, radius, UV,
                                    points=[(p % nx, p // nx) for p in pts])
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, radius, UV)
    Wb = lbm.W[None, :, None, None]
    fb = _flat(f0.astype(np.float64) - Wb)
    for sch, (dev, lam) in outs.items():
        errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), fb)
        assert max(errs) < 1e-5, (sch, errs)
        for i, p in enumerate(pts):
            r = ref[(p % nx, p // nx)]
            assert np.abs(np.sort(lam[i]) - r["lam"]).max() < 1e-5 * r["lam"].max(), sch
    # split and fused: the same algorithm and recurrence, different summation orders only
    fused, split = outs[L.LETKF_EIG_FUSED][0], outs[L.LETKF_EIG_SPLIT][0]
    errs = C.point_parity(_flat(split), _flat(fused), fb)
    assert max(errs) < 2e-6, errs
    lf, ls = np.sort(outs[L.LETKF_EIG_FUSED][1], 1), np.sort(outs[L.LETKF_EIG_SPLIT][1], 1)
    assert np.abs(lf - ls).max() <= 1e-6 * np.abs(lf).max()


@pytest.mark.parametrize("k,n,precision", [(32, 136, L.LETKF_FP32), (24, 128, L.LETKF_MIXED),
                                         (64, 128, L.LETKF_MIXED)])
def test_split_schedule_on_two_streams_matches_fused_and_oracle(k, n, precision):
    # chunks of >= 16384 points (k <= 32) run the split kernels as two overlapping halves on two
    # streams (the second half's points listed at their chunk index); the analysis must equal
    # the fused schedule to FP32 rounding and the oracle at sampled points, including the
    # points at the seam between the halves
    net = synth.regular_obs_network(n, n, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    f0 = C.big_ensemble_state(k, n, n, seed=961 + k)
    Yf = C.observe_at_points(f0, net, UV)
    yo = (Yf.mean(0) + synth.gaussian(Yf.shape[1], 0.01, 962)).astype(np.float32)
    outs = {}
    for sch in (L.LETKF_EIG_SPLIT, L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT_CHECK):
        exp = L.Experiment(n, n, k, 0.6, net, var, loc_radius=3.0, precision=precision,
                           eig_schedule=sch)
        exp.set_state(f0)
        exp.analyze(yo)
        outs[sch] = C.dev64(exp.get_deviation())
        assert exp.sync() == 0
    Wb = lbm.W[None, :, None, None]
    fb = _flat(f0.astype(np.float64) - Wb)
    # the same algorithm; at 33 <= k <= 64 the split tridiagonalization sums its dot products
    # over two warps (another summation order), and the increment's rounding difference
    # scales with Q's condition number (up to ~80 here: 80 x FP32 epsilon ~ 5e-6)
    for sch in (L.LETKF_EIG_SPLIT, L.LETKF_EIG_SPLIT_CHECK):
        errs = C.point_parity(_flat(outs[sch]), _flat(outs[L.LETKF_EIG_FUSED]), fb)
        assert max(errs) < 5e-6, (sch, errs)
    half = (n * n // 2 + 63) // 64 * 64
    pts = sorted({0, half - 1, half, half + 1, n * n - 1, n * n // 3})
    ref = C.oracle_points(f0, Yf, yo, net, var, 3.0, UV, [(p % n, p // n) for p in pts])
    bg, bo, bf = [], [], []
    for p in pts:
        x, y = p % n, p // n
        bg.append(outs[L.LETKF_EIG_SPLIT][:, :, y, x])
        bo.append(ref[(x, y)]["Xa"].T - lbm.W[None, :])
        bf.append(f0[:, :, y, x].astype(np.float64) - lbm.W[None, :])
    errs = C.point_parity(np.concatenate(bg, 1), np.concatenate(bo, 1), np.concatenate(bf, 1))
    assert max(errs) < 1e-5, errs


def test_split_schedule_in_mixed_precision_matches_oracle():
    f0, yo, net, var, dev, _, _ = _run(64, 16, 16, 2, 3.0, 951, L.LETKF_EIG_SPLIT,
                                       precision=L.LETKF_MIXED)
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, 3.0, UV)
    Wb = lbm.W[None, :, None, None]
    errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), _flat(f0.astype(np.float64) - Wb))
    assert max(errs) < 1e-5, errs


def test_split_schedule_is_reproducible():
    runs = [_run(32, 16, 16, 4, 3.0, 961, L.LETKF_EIG_SPLIT)[4] for _ in range(2)]
    assert np.array_equal(runs[0], runs[1])


def _auto_case(k, schedule, seed):
    nx = ny = 12
    net = synth.regular_obs_network(nx, ny, 3)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=seed), 1e-4, seed + 1)
    yo = C.observations(C.ensemble_state(1, nx, ny, seed=seed + 2), net, UV, 0.01, seed + 3)[0]
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.0, eig_schedule=schedule)
    exp.set_state(f0)
    return exp, yo


def test_auto_schedule_resolves_at_the_first_analysis_once_per_process():
    # k = 47 is a shape no other test uses, so the process has no pick for it yet
    exp, yo = _auto_case(47, L.LETKF_EIG_AUTO, 971)
    assert exp.stats().eig_schedule == L.LETKF_EIG_AUTO         # unresolved before analysing
    exp.analyze(yo)
    pick = exp.stats().eig_schedule
    assert pick in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT) + EVD_FREE
    got = exp.get_deviation()
    assert exp.sync() == 0
    # the timed runs worked on scratch: the analysis is the picked schedule's, bit for bit
    ref, _ = _auto_case(47, pick, 971)
    ref.analyze(yo)
    assert np.array_equal(got, ref.get_deviation()) and ref.sync() == 0
    # a later handle of the same shape takes the pick at letkf_init
    later, _ = _auto_case(47, L.LETKF_EIG_AUTO, 972)
    assert later.stats().eig_schedule == pick and later.sync() == 0


def test_auto_schedule_first_cycle_runs_eagerly_then_captures():
    # k = 45: unused elsewhere.  The first cycle times the schedules (no graph), the next
    # ones replay a captured graph; all equal the picked schedule's cycles bit for bit.
    a, yo = _auto_case(45, L.LETKF_EIG_AUTO, 975)
    a.cycle(3, yo)
    assert a.stats().cycle_kernels == 0                        # eager: no graph yet
    pick = a.stats().eig_schedule
    assert pick in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT) + EVD_FREE
    b, _ = _auto_case(45, pick, 975)
    b.cycle(3, yo)
    for _ in range(2):
        a.cycle(3, yo)
        b.cycle(3, yo)
    assert a.stats().cycle_kernels > 0
    assert a.stats().cycle_kernels == b.stats().cycle_kernels
    assert np.array_equal(a.get_deviation(), b.get_deviation())
    assert a.sync() == 0 and b.sync() == 0


@pytest.mark.parametrize("k_big,k_small", [(16, 8), (128, 100), (64, 33)])
def test_handles_of_different_k_coexist(k_big, k_small):
    # the kernels' shared-memory caps are process-wide: a later handle with a smaller k
    # must not lower them under an earlier handle with a larger k
    for sch in (L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT) + EVD_FREE:
        if sch in EVD_FREE and k_big > 64:
            continue
        first = _run(k_big, 10, 10, 2, 2.0, 980 + k_big, sch)          # builds handle 1
        nx = ny = 10
        net = synth.regular_obs_network(nx, ny, 2)
        var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
        f0 = C.perturb_nonequilibrium(C.ensemble_state(k_big, nx, ny, seed=981), 1e-4, 982)
        a = L.Experiment(nx, ny, k_big, 0.6, net, var, loc_radius=2.0, eig_schedule=sch)
        b = L.Experiment(nx, ny, k_small, 0.6, net, var, loc_radius=2.0, eig_schedule=sch)
        a.set_state(f0)
        truth = C.ensemble_state(1, nx, ny, seed=983)
        yo = C.observations(truth, net, UV, 0.01, 984)[0]
        a.analyze(yo)                                   # after b lowered nothing
        dev = C.dev64(a.get_deviation())
        assert a.sync() == 0 and b.sync() == 0
        Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, 2.0, UV)
        Wb = lbm.W[None, :, None, None]
        errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), _flat(f0.astype(np.float64) - Wb))
        assert max(errs) < 1e-5, (sch, errs)
        del first


@pytest.mark.parametrize("sch", [L.LETKF_EIG_FUSED, L.LETKF_EIG_SPLIT])
def test_large_ensemble_with_rank_deficient_gram_converges(sch):
    # k = 128 with ~84 local observed scalars and sigma = 1e-3: Q = 127 I + a rank-84 term
    # with eigenvalues in the thousands (the case that exhausted the QL iteration cap when
    # deflation was tested against the local diagonal only)
    nx = ny = 24
    k = 128
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=991), 2e-3, 992)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-6, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=4.0, eig_schedule=sch)
    exp.set_state(f0)
    truth = C.ensemble_state(1, nx, ny, seed=993)
    yo = C.observations(truth, net, UV, 1e-3, 994)[0]
    exp.analyze(yo)
    dev = C.dev64(exp.get_deviation())
    assert exp.sync() == 0
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, 4.0, UV)
    Wb = lbm.W[None, :, None, None]
    errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), _flat(f0.astype(np.float64) - Wb))
    assert max(errs) < 1e-5, errs
