"""letkf_local_analysis_noalloc: the analysis for callers that cannot allocate device memory.

Such callers (plugin code that only receives its input/output buffers, processes whose
device memory is reserved by another allocator, allocation-free real-time loops) cannot
create a handle, so this entry point takes the padded per-point local data and keeps its
scratch in a static device array.  Checked here, through the C ABI:
  * two calls in a row against the handle-based letkf_analyze on the same forecast and
    observations, for every Gram tile width the entry point instantiates (k = 5, 16, 32, 64,
    128) and with and without inflation;
  * against the FP64 oracle's local analysis on the same padded inputs (ragged local counts,
    points without observations, garbage in the padding rows), for k >= 33;
  * the size limit: the largest problem the scratch holds is accepted and analysed
    correctly, one point more is rejected.
The tolerance is the parity tests' 1e-5 relative L2 on the analysis mean, the mean increment
and the perturbations.  The file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import synth
from oracle import letkf as oletkf
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

UV = L.LETKF_OBS_U | L.LETKF_OBS_V
SCRATCH_FLOATS = L.LETKF_NOALLOC_SCRATCH_BYTES // 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _max_points(k):
    """Largest npts whose Gram matrices, c vectors, counts and status fit in the scratch."""
    return (SCRATCH_FLOATS - 64) // (k * k + k + 1)


def _padded_local_data(Yf, yo, net, var, nx, ny, radius):
    """Padded local layout (dy_loc [N][lmaxV][k], d_loc, r_loc) built from the handle's
    forecast observations with the oracle's localization rule."""
    k = Yf.shape[0]
    Yf = Yf.astype(np.float64)
    ybar = Yf.mean(0)
    dY = Yf - ybar
    c2 = synth.loc_cutoff2(radius)
    per = []
    for y in range(ny):
        for x in range(nx):
            sel, d2 = oletkf.local_obs(x, y, net, nx, ny, c2)
            g = oletkf.localization_weight(d2, radius)
            idx = (sel[:, None] * 2 + np.arange(2)[None, :]).ravel()
            per.append((idx, np.repeat(g, 2)))
    lmaxv = max(len(i) for i, _ in per)
    n = nx * ny
    dy_loc = np.zeros((n, lmaxv, k), np.float32)
    d_loc = np.zeros((n, lmaxv), np.float32)
    r_loc = np.zeros((n, lmaxv), np.float32)
    for p, (idx, g) in enumerate(per):
        m = len(idx)
        dy_loc[p, :m] = dY[:, idx].T
        d_loc[p, :m] = yo[idx] - ybar[idx]
        r_loc[p, :m] = g / var[idx]
    return dy_loc, d_loc, r_loc, lmaxv


def _random_padded_problems(npts, k, lmaxv, seed):
    """Independent local problems in the padded layout: ragged counts in [0, lmaxv] (about a
    tenth of the points without observations), perturbation rows with zero member mean,
    padding rows filled with garbage that a correct kernel ignores (r = 0 marks them)."""
    rng = synth.generator(seed)
    counts = rng.integers(0, lmaxv + 1, size=npts)
    counts[rng.random(npts) < 0.1] = 0
    x = (0.1 + synth.gaussian((npts, 9, k), 0.01, seed + 1)).astype(np.float32)
    yf = synth.gaussian((npts, lmaxv, k), 0.01, seed + 2)
    dy = (yf - yf.mean(axis=2, keepdims=True)).astype(np.float32)
    d = synth.gaussian((npts, lmaxv), 0.01, seed + 3).astype(np.float32)
    r = (1e4 * np.exp(-synth.gaussian((npts, lmaxv), 1.0, seed + 4) ** 2)).astype(np.float32)
    pad = np.arange(lmaxv)[None, :] >= counts[:, None]
    r[pad] = 0.0
    dy[pad] = 7.0                     # garbage: must not reach the result
    d[pad] = -3.0
    return x, dy, d, r, counts


def _noalloc(npts, k, lmaxv, dy, d, r, infl, x):
    """One call through the C ABI on torch's current stream; returns (rc, analysis blocks)."""
    import torch

    dev = torch.device("cuda")
    t_dy, t_d, t_r = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (dy, d, r))
    t_x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    torch.cuda.synchronize()
    rc = L.letkf_local_analysis_noalloc(npts, k, lmaxv, t_dy.data_ptr(), t_d.data_ptr(),
                                        t_r.data_ptr(), infl, t_x.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    return rc, t_x.cpu().numpy()


def _oracle_blocks(x, dy, d, r, counts, infl, points):
    out = []
    for p in points:
        m = int(counts[p])
        res = oletkf.local_analysis(x[p].astype(np.float64), dy[p, :m].astype(np.float64),
                                    d[p, :m].astype(np.float64), r[p, :m].astype(np.float64),
                                    infl)
        out.append(res["Xa"])
    return np.stack(out)                     # [n, 9, k]


def _block_parity(got, ref, xf):
    """point_parity of [n, 9, k] analysis blocks (members on the last axis)."""
    k = got.shape[-1]
    flat = [np.asarray(a, np.float64).transpose(2, 0, 1).reshape(k, -1) for a in (got, ref, xf)]
    return C.point_parity(*flat)


@pytest.mark.parametrize("k,infl", [(5, 1.0), (16, 1.0), (32, 1.1), (64, 1.0), (128, 1.1)])
def test_noalloc_matches_handle_analysis_on_two_calls_in_a_row(k, infl):
    nx = ny = 32 if k <= 64 else 24           # 24^2 points at k = 128 fit the scratch
    radius = 3.0
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=501), 1e-4, 502)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=radius, infl=infl)
    exp.set_state(f0)
    g0 = exp.get_deviation()                       # [k, 9, ny, nx]
    Yf = exp.get_obs()[:k]
    x0 = np.ascontiguousarray(g0.transpose(2, 3, 1, 0).reshape(nx * ny, 9, k))
    for call, seed in enumerate((503, 504)):      # two calls in a row share the scratch
        truth = C.ensemble_state(1, nx, ny, seed=seed)
        yo = C.observations(truth, net, UV, 0.01, seed + 1)[0]
        exp.set_deviation(g0)
        exp.analyze(yo)
        ga = exp.get_deviation()
        assert exp.sync() == 0
        ref = ga.transpose(2, 3, 1, 0).reshape(nx * ny, 9, k)
        dy_loc, d_loc, r_loc, lmaxv = _padded_local_data(Yf, yo, net, var, nx, ny, radius)
        rc, got = _noalloc(nx * ny, k, lmaxv, dy_loc, d_loc, r_loc, infl, x0)
        assert rc == L.LETKF_OK, L.strerror(rc)
        errs = _block_parity(got, ref, x0)
        assert max(errs) < 1e-5, (call, errs)
    exp.close()


@pytest.mark.parametrize("k,infl,lmaxv", [(40, 1.1, 60), (64, 1.0, 150), (64, 1.5, 33)])
def test_noalloc_matches_oracle_local_analysis(k, infl, lmaxv):
    npts = 300
    x, dy, d, r, counts = _random_padded_problems(npts, k, lmaxv, seed=900 + k + lmaxv)
    for call in range(2):                    # the second call reuses the scratch as left
        rc, got = _noalloc(npts, k, lmaxv, dy, d, r, infl, x)
        assert rc == L.LETKF_OK, L.strerror(rc)
        ref = _oracle_blocks(x, dy, d, r, counts, infl, range(npts))
        errs = _block_parity(got, ref, x)
        assert max(errs) < 1e-5, (call, errs)
        empty = counts == 0
        assert empty.any()
        if infl == 1.0:                      # without inflation such points stay as they are
            assert np.array_equal(got[empty], x[empty])


def test_noalloc_accepts_the_largest_problem_and_rejects_one_point_more():
    k, lmaxv = 64, 4
    n_max = _max_points(k)
    assert n_max == 4032                     # (64 MiB / 4 - 64) // (64^2 + 64 + 1)
    x, dy, d, r, counts = _random_padded_problems(n_max + 1, k, lmaxv, seed=977)
    # one point too many: rejected before any launch, with valid device buffers
    rc, got = _noalloc(n_max + 1, k, lmaxv, dy, d, r, 1.0, x)
    assert rc == L.LETKF_EINVAL
    assert np.array_equal(got, x)
    # the largest problem that fits: accepted, and every point analysed correctly
    rc, got = _noalloc(n_max, k, lmaxv, dy[:n_max], d[:n_max], r[:n_max], 1.0, x[:n_max])
    assert rc == L.LETKF_OK, L.strerror(rc)
    sample = np.r_[0:8, n_max - 8:n_max, synth.generator(978).integers(0, n_max, 48)]
    ref = _oracle_blocks(x, dy, d, r, counts, 1.0, sample)
    errs = _block_parity(got[sample], ref, x[sample])
    assert max(errs) < 1e-5, errs
    # an ensemble size beyond the kernels' range
    x2, dy2, d2, r2, _ = _random_padded_problems(4, 129, 2, seed=979)
    rc, got = _noalloc(4, 129, 2, dy2, d2, r2, 1.0, x2)
    assert rc == L.LETKF_EINVAL
    assert np.array_equal(got, x2)
