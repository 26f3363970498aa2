"""The Chebyshev schedule (LETKF_EIG_CHEBYSHEV) against the FP64 oracle.

The schedule replaces Q^-1/2 and Q^-1 by Chebyshev interpolants of t^-1/2 and t^-1 on
[1, kappa] (S = Q rho / (k-1), kappa from the least of the Gershgorin, Frobenius and trace
bounds of A) applied to [dX; c^T] by Clenshaw's recurrence; no factorization is formed.  A point
whose bound needs a degree above 9k/16 (kappa 16 at k = 64) goes to the rational schedule
through a list.  Checked:
  * the full-size workloads (256^2 at k = 32, 1024^2 at k = 64) at sampled grid points against
    the oracle's local analyses, FP32 and mixed, at the parity tests' bars (1e-5 relative L2
    over the sampled outputs, 5e-5 per point);
  * a network whose observation error variances differ 1000-fold between the two halves of a
    48 x 16 domain, so that some points are transformed by the polynomials and others are passed on
    (both counted by letkf_get_work_counts), against the oracle at every grid point, k = 16
    and 48;
  * the products counted match the degrees of the table, point by point from the probed Gram
    matrices (the condition bound of each point selects its set);
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
CHEB = L.LETKF_EIG_CHEBYSHEV


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _flat(a):
    return np.asarray(a).transpose(0, 2, 3, 1).reshape(a.shape[0], -1)


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
                       precision=precision, eig_schedule=CHEB)
    exp.set_state(f0)
    Yf = C.observe_at_points(f0, net, UV)
    yo = (Yf.mean(0) + synth.gaussian(Yf.shape[1], 0.01, 142)).astype(np.float32)
    pts = _sampled_points(nx, ny, 40, 143)
    exp.analyze(yo)
    got = exp.get_deviation()
    assert exp.sync() == 0
    assert exp.stats().eig_schedule == CHEB
    counts = exp.work_counts()
    assert counts["cheb_points"] + counts["cheb_handed_on"] == nx * ny - exp.stats().n_zero_obs
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
    assert max(errs) < 1e-5, (errs, counts)
    assert max(worst) < 5e-5, (worst, counts)
    exp.close()


@pytest.mark.parametrize("k", [16, 48])
def test_polynomial_and_passed_on_points_match_oracle(k):
    # observation error variance 1e-2 on the left half of a 48-wide domain, 1e-5 on the right:
    # the Gram matrices of points that see right-half observations are ~1000 times larger,
    # beyond the Chebyshev sets in use; the middle of the left half (cutoff 7.3) sees none
    nx, ny = 48, 16
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=181), 1e-4, 182)
    net = synth.regular_obs_network(nx, ny, 3)
    right = (net[:, 0] >= nx // 2)
    var = np.repeat(np.where(right, 1e-5, 1e-2), 2).astype(np.float32)
    yo = C.observations(C.ensemble_state(1, nx, ny, seed=183), net, UV, 0.01, 184)[0]
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=2.0, eig_schedule=CHEB)
    exp.set_state(f0)
    exp.analyze(yo)
    dev = C.dev64(exp.get_deviation())
    assert exp.sync() == 0
    counts = exp.work_counts()
    exp.close()
    assert counts["cheb_points"] > 0 and counts["cheb_handed_on"] > 0, counts
    Xa_ref, _ = C.oracle_analysis(f0, yo, net, var, 2.0, UV)
    Wb = lbm.W[None, :, None, None]
    fb = _flat(f0.astype(np.float64) - Wb)
    errs = C.point_parity(_flat(dev), _flat(Xa_ref - Wb), fb)
    assert max(errs) < 1e-5, (errs, counts)


# the approximations' kappa_max, in the order the transform tries them (chebyshev.cu)
CHEB_KAPPA_MAX = (1.0002, 1.005, 1.035, 1.1, 1.2, 1.35, 1.5, 1.75, 2.0, 2.5, 3.0, 4.0, 6.0, 10.0,
                  16.0)


def _table_degree(kappa_max):
    # the least degree whose interpolants reach 2e-8 on [1, kappa_max]
    n = 1
    while L.letkf_chebyshev_coefficients(kappa_max, n)[2] > 2e-8:
        n += 1
    return n


def _degree_for(kappa, degrees):
    for km, n in zip(CHEB_KAPPA_MAX, degrees):
        if kappa <= km:
            return n
    return None


def test_products_follow_the_degree_table():
    # Every observed point's bound kappa = 1 + min(Gershgorin, Frobenius, trace)(A) / d picks the
    # first approximation that covers it, and its degree is the number of products.  Checked
    # point by point against the probed Gram matrices of the same analysis; a bound within the
    # device's FP32 rounding margin of a set's edge may take either neighbour.
    nx = ny = 16
    k = 32
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=191), 1e-5, 192)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-2, dtype=np.float32)
    yo = C.observations(C.ensemble_state(1, nx, ny, seed=193), net, UV, 0.1, 194)[0]
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, eig_schedule=CHEB)
    exp.set_state(f0)
    pts = np.arange(nx * ny)
    pr = exp.analyze_probe(yo, pts, want=("nloc", "gram"))
    assert exp.sync() == 0
    counts = exp.work_counts()
    exp.close()
    degrees = [_table_degree(km) for km in CHEB_KAPPA_MAX]
    assert degrees[:4] == [1, 2, 3, 4]
    d = float(k - 1)
    lo = hi = observed = exact = 0
    seen = set()
    for i in range(pts.size):
        if pr["nloc"][i] == 0:
            continue
        observed += 1
        A = pr["gram"][i].astype(np.float64)
        e = max(min(np.abs(A).sum(axis=1).max(), np.sqrt((A * A).sum()), np.trace(A)), 0.0)
        n_lo = _degree_for(1.0 + (e / d) * (1.0 - 1e-4), degrees)
        n_hi = _degree_for(1.0 + (e / d) * (1.0 + 1e-3) + 2e-6, degrees)
        assert n_lo is not None and n_hi is not None
        lo += n_lo
        hi += n_hi
        exact += n_lo == n_hi
        seen.add(n_lo)
    assert counts["cheb_points"] == observed and counts["cheb_handed_on"] == 0, counts
    assert lo <= counts["cheb_products"] <= hi, (counts, lo, hi)
    assert exact >= 0.9 * observed                # the check is point by point, not a range
    assert min(seen) < 4                          # the sets below kappa 1.1 are in use


def test_chebyshev_cycle_equals_forecast_then_analysis():
    nx = ny = 40
    k = 24
    f0 = C.ensemble_state(k, nx, ny, seed=161)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    yos = [C.observations(C.ensemble_state(1, nx, ny, seed=162 + c), net, UV, 0.01, 170 + c)[0]
           for c in range(3)]
    a = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, eig_schedule=CHEB)
    b = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=3.0, eig_schedule=CHEB)
    a.set_state(f0)
    b.set_state(f0)
    for y in yos:
        a.cycle(5, y)
        b.forecast(5)
        b.analyze(y)
    assert np.array_equal(a.get_deviation(), b.get_deviation())
    assert a.sync() == 0 and b.sync() == 0
