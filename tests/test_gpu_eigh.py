"""letkf_eigh_batch (one warp per matrix) and letkf_eigh_batch_ws (the split schedule, caller
workspace): the analysis' batched symmetric eigensolver against numpy.linalg.eigh.

Pins (FP64 eigh of the same FP32 matrices is the reference):
  * eigenvalues within 1e-5 of the largest magnitude, orthonormal eigenvectors (max entry of
    V^T V - I below 1e-5), residual ||Q V - V L|| / ||Q|| below 1e-5, for k = 2..128;
  * a degenerate spectrum (31 I + a rank-3 term: k - 3 equal eigenvalues) and a tightly
    clustered one: orthonormality and residual still hold, and the FP64 refinement sweep
    (modified Gram-Schmidt within clusters, Rayleigh quotients) keeps the matrix functions the
    analysis needs, W = V L^-1/2 V^T and V L^-1 V^T, at least as accurate as without it;
  * the upper triangle and the diagonal of the input are left bit for bit.
"""
import numpy as np
import pytest

from paper_2308_03310_gb300 import _build, letkf as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _random_spd(n, k, seed, scale=None):
    rng = np.random.default_rng(seed)
    out = np.empty((n, k, k), np.float32)
    for p in range(n):
        Y = 0.7 * (rng.random((k, 2 * k)) - 0.5)
        out[p] = ((k - 1) * np.eye(k) + Y @ Y.T).astype(np.float32)
    return out


def _from_spectrum(lams, seed):
    rng = np.random.default_rng(seed)
    k = len(lams)
    U, _ = np.linalg.qr(rng.standard_normal((k, k)))
    Q = (U * np.asarray(lams)) @ U.T
    return ((Q + Q.T) / 2).astype(np.float32)


SOLVERS = ["fused", "split"]


def _solve(Q, refine, solver="fused"):
    import torch
    n, k, _ = Q.shape
    dev = torch.device("cuda")
    tq = torch.from_numpy(Q.copy()).to(dev)
    lam = torch.empty((n, k), dtype=torch.float32, device=dev)
    vec = torch.empty((n, k, k), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    if solver == "fused":
        rc = L.letkf_eigh_batch(n, k, tq.data_ptr(), lam.data_ptr(), vec.data_ptr(), refine,
                                stream)
    else:
        nb = L.letkf_eigh_workspace_bytes(n, k)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        base = (ws.data_ptr() + 255) // 256 * 256
        rc = L.letkf_eigh_batch_ws(n, k, tq.data_ptr(), lam.data_ptr(), vec.data_ptr(), refine,
                                   base, nb, stream)
    assert rc == L.LETKF_OK, L.strerror(rc)
    return tq.cpu().numpy(), lam.cpu().numpy().astype(np.float64), \
        vec.cpu().numpy().astype(np.float64)


def _check_pairs(Q, lam, vec, tol=1e-5):
    for p in range(Q.shape[0]):
        q = Q[p].astype(np.float64)
        ref = np.linalg.eigvalsh(q)
        scale = np.abs(ref).max()
        assert np.abs(np.sort(lam[p]) - ref).max() < tol * scale
        V = vec[p].T                                   # columns = eigenvectors
        assert np.abs(V.T @ V - np.eye(len(ref))).max() < tol
        assert np.linalg.norm(q @ V - V * lam[p]) / np.linalg.norm(q) < tol


def _matfun_errors(Q, lam, vec):
    """Relative errors of V L^-1/2 V^T and V L^-1 V^T against FP64 eigh, worst over the batch."""
    e_half, e_inv = 0.0, 0.0
    for p in range(Q.shape[0]):
        q = Q[p].astype(np.float64)
        w, U = np.linalg.eigh(q)
        V = vec[p].T
        for f, name in ((lambda x: x ** -0.5, "half"), (lambda x: 1.0 / x, "inv")):
            ref = (U * f(w)) @ U.T
            got = (V * f(lam[p])) @ V.T
            e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            if name == "half":
                e_half = max(e_half, e)
            else:
                e_inv = max(e_inv, e)
    return e_half, e_inv


@pytest.mark.parametrize("k", [2, 5, 31, 32, 33, 64, 100, 128])
@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("solver", SOLVERS)
def test_eigenpairs_match_eigh(k, refine, solver):
    Q = _random_spd(24, k, 1000 + k)
    Qout, lam, vec = _solve(Q, refine, solver)
    _check_pairs(Q, lam, vec)
    iu = np.triu_indices(k)
    assert np.array_equal(Qout[:, iu[0], iu[1]], Q[:, iu[0], iu[1]])


@pytest.mark.parametrize("k", [32, 64, 128])
@pytest.mark.parametrize("solver", SOLVERS)
def test_degenerate_spectrum(k, solver):
    rng = np.random.default_rng(7 + k)
    Q = np.empty((8, k, k), np.float32)
    for p in range(8):
        Y = rng.standard_normal((k, 3)) * 0.5
        Q[p] = ((k - 1) * np.eye(k) + Y @ Y.T).astype(np.float32)
    for refine in (0, 1):
        _, lam, vec = _solve(Q, refine, solver)
        _check_pairs(Q, lam, vec)


@pytest.mark.parametrize("k", [32, 64])
def test_refinement_on_clustered_spectra(k):
    # a cluster of 8 eigenvalues 2e-6 apart (relative ~6e-8) next to well separated ones
    mats = []
    for s in range(8):
        lams = np.concatenate([31.0 + 2e-6 * np.arange(8), 31.5 + 0.25 * np.arange(k - 8)])
        mats.append(_from_spectrum(lams, 500 + s))
    Q = np.stack(mats)
    errs = {}
    for refine in (0, 1):
        _, lam, vec = _solve(Q, refine)
        _check_pairs(Q, lam, vec)
        errs[refine] = _matfun_errors(Q, lam, vec)
    print("clustered k", k, "W, Pinv errors without / with refinement:", errs[0], errs[1])
    # measured on GB300: W 1.63e-6 -> 1.54e-6 (k = 32), 3.48e-6 -> 3.27e-6 (k = 64); the rest
    # of the error is the FP32 accuracy of the well separated pairs (~k eps)
    for i in range(2):
        assert errs[1][i] <= 1.02 * errs[0][i] + 1e-8, errs
        assert errs[1][i] < 1e-5, errs


@pytest.mark.parametrize("k,rank,top", [(128, 84, 2000.0), (64, 40, 5000.0), (32, 20, 1e4)])
@pytest.mark.parametrize("solver", SOLVERS)
def test_small_cluster_next_to_large_eigenvalues_converges(k, rank, top, solver):
    # (k-1) I + a rank-r term with eigenvalues up to `top`: k - r equal eigenvalues beside
    # large ones.  QL must deflate the equal block although every sweep through the large
    # entries leaves rounding of order eps ||Q|| on its couplings (threshold eps ||T||).
    rng = np.random.default_rng(k + rank)
    Q = np.empty((6, k, k), np.float32)
    for p in range(6):
        U, _ = np.linalg.qr(rng.standard_normal((k, rank)))
        lam = np.geomspace(1.0, top, rank)
        Q[p] = ((k - 1) * np.eye(k) + (U * lam) @ U.T).astype(np.float32)
    for refine in (0, 1):
        _, lam, vec = _solve(Q, refine, solver)         # LETKF_OK, not ENOTCONV
        _check_pairs(Q, lam, vec)


def test_split_solver_rejects_a_short_or_misaligned_workspace():
    import torch
    n, k = 8, 32
    dev = torch.device("cuda")
    q = torch.eye(k, device=dev).repeat(n, 1, 1).contiguous()
    lam = torch.empty((n, k), device=dev)
    nb = L.letkf_eigh_workspace_bytes(n, k)
    assert nb > 8 * n * k * k
    ws = torch.empty(nb + 512, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) // 256 * 256
    s = torch.cuda.current_stream().cuda_stream
    assert L.letkf_eigh_batch_ws(n, k, q.data_ptr(), lam.data_ptr(), 0, 0, base, nb - 1, s) \
        == L.LETKF_ENOMEM
    assert L.letkf_eigh_batch_ws(n, k, q.data_ptr(), lam.data_ptr(), 0, 0, base + 4, nb, s) \
        == L.LETKF_ENOMEM
    assert L.letkf_eigh_batch_ws(n, k, q.data_ptr(), lam.data_ptr(), 0, 0, base, nb, s) \
        == L.LETKF_OK
    assert np.allclose(lam.cpu().numpy(), 1.0)
