"""letkf_local_analysis_noalloc: the analysis for callers that cannot allocate device memory.

Such callers (plugin code that only receives its input/output buffers, processes whose
device memory is reserved by another allocator, allocation-free real-time loops) cannot
create a handle, so this entry point takes the padded per-point local data and keeps its
scratch in a static device array.  Here it is called through the C ABI twice in a row and
checked against the handle-based letkf_analyze on the same forecast and observations, to
the tolerance the parity tests use (1e-5 relative L2 on the analysis mean, mean increment
and perturbations).  The file is collected last so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest

import synth
from oracle import letkf as oletkf
from paper_2308_03310_gb300 import _build, letkf as L
from tests import _cases as C

pytestmark = pytest.mark.gpu

UV = L.LETKF_OBS_U | L.LETKF_OBS_V


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _padded_local_data(Yf, yo, net, var, nx, ny, radius):
    """The padded local layout of Algorithm 1 (dy_loc [N][lmaxV][k], d_loc, r_loc), built
    from the handle's forecast observations with the same localization rule."""
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


def test_noalloc_matches_handle_analysis_on_two_calls_in_a_row():
    import torch

    nx = ny = 32
    k, radius = 16, 3.0
    f0 = C.perturb_nonequilibrium(C.ensemble_state(k, nx, ny, seed=501), 1e-4, 502)
    net = synth.regular_obs_network(nx, ny, 4)
    var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
    exp = L.Experiment(nx, ny, k, 0.6, net, var, loc_radius=radius)
    exp.set_state(f0)
    g0 = exp.get_deviation()                       # [k, 9, ny, nx]
    Yf = exp.get_obs()[:k]
    x0 = np.ascontiguousarray(g0.transpose(2, 3, 1, 0).reshape(nx * ny, 9, k))
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((503, 504)):      # two calls in a row share the scratch
        truth = C.ensemble_state(1, nx, ny, seed=seed)
        yo = C.observations(truth, net, UV, 0.01, seed + 1)[0]
        exp.set_deviation(g0)
        exp.analyze(yo)
        ga = exp.get_deviation()
        assert exp.sync() == 0
        ref = ga.transpose(2, 3, 1, 0).reshape(nx * ny, 9, k).astype(np.float64)

        dy_loc, d_loc, r_loc, lmaxv = _padded_local_data(Yf, yo, net, var, nx, ny, radius)
        t_dy = torch.from_numpy(dy_loc).to(dev)
        t_d = torch.from_numpy(d_loc).to(dev)
        t_r = torch.from_numpy(r_loc).to(dev)
        t_x = torch.from_numpy(x0.copy()).to(dev)
        torch.cuda.synchronize()
        rc = L.letkf_local_analysis_noalloc(nx * ny, k, lmaxv, t_dy.data_ptr(), t_d.data_ptr(),
                                            t_r.data_ptr(), 1.0, t_x.data_ptr(),
                                            stream.cuda_stream)
        assert rc == L.LETKF_OK, L.strerror(rc)
        got = t_x.cpu().numpy().astype(np.float64)
        # [N, 9, k] blocks -> [k, N*9] for the member-axis comparison
        errs = C.point_parity(got.transpose(2, 0, 1).reshape(k, -1),
                              ref.transpose(2, 0, 1).reshape(k, -1),
                              x0.astype(np.float64).transpose(2, 0, 1).reshape(k, -1))
        assert max(errs) < 1e-5, (call, errs)


def test_noalloc_rejects_problems_larger_than_its_scratch():
    k = 64
    too_many = L.LETKF_NOALLOC_SCRATCH_BYTES // 4 // (k * k + k + 1) + 1
    rc = L.letkf_local_analysis_noalloc(too_many, k, 4, 1, 1, 1, 1.0, 1, 0)
    assert rc == L.LETKF_EINVAL
    assert L.letkf_local_analysis_noalloc(10, 129, 4, 1, 1, 1, 1.0, 1, 0) == L.LETKF_EINVAL
