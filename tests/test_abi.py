"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/letkf.h declares, and its host-side validation rejects bad problems."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2308_03310_gb300 import _build, letkf as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "letkf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;{]*\)\s*;", src, flags=re.M)
    return [n for n in names if n != "if"]


def test_header_declarations_match_binding():
    declared = _declared_functions()
    assert len(declared) >= 14
    assert sorted(declared) == sorted(L.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_strerror_names_every_code(lib):
    for code in range(0, -8, -1):
        assert L.strerror(code) and L.strerror(code) != "unknown status code"
    assert L.strerror(-99) == "unknown status code"


def _cfg(nx=32, ny=32, k=8, **kw):
    obs = np.array([[0, 0], [4, 4]], dtype=np.int32)
    var = np.full(4, 1e-4, dtype=np.float32)
    cfg = L.letkf_config()
    cfg.nx, cfg.ny, cfg.k, cfg.n_aux = nx, ny, k, 0
    cfg.tau = 0.6
    cfg.n_obs = 2
    cfg.obs_xy = obs.ctypes.data_as(C.POINTER(C.c_int32))
    cfg.obs_vars = L.LETKF_OBS_U | L.LETKF_OBS_V
    cfg.obs_err_var = var.ctypes.data_as(C.POINTER(C.c_float))
    cfg.loc_kind = L.LETKF_LOC_GAUSS
    cfg.loc_radius = 3.0
    cfg.infl = 1.0
    for key, val in kw.items():
        setattr(cfg, key, val)
    cfg._keep = (obs, var)
    return cfg


def test_workspace_size_is_host_only_and_scales(lib):
    small = L.letkf_workspace_size(_cfg())
    big = L.letkf_workspace_size(_cfg(nx=64, ny=64))
    assert small > 0 and big > 3 * small
    # state double buffer + grid-point-major copy at least
    assert small >= (2 * 8 * 9 + 9 * 8) * 32 * 32 * 4


@pytest.mark.parametrize("field,value", [
    ("k", 1), ("k", 129), ("nx", 0), ("tau", 0.5), ("obs_vars", 0), ("obs_vars", 8),
    ("loc_radius", 0.0), ("infl", 0.0), ("n_aux", 5), ("precision", 7), ("loc_kind", 3),
    ("chunk_bytes", -1)])
def test_invalid_configurations_are_rejected(lib, field, value):
    with pytest.raises(L.LetkfError) as e:
        L.letkf_workspace_size(_cfg(**{field: value}))
    assert e.value.code == L.LETKF_EINVAL


def test_observation_outside_grid_is_rejected(lib):
    cfg = _cfg()
    bad = np.array([[0, 0], [32, 4]], dtype=np.int32)
    cfg.obs_xy = bad.ctypes.data_as(C.POINTER(C.c_int32))
    with pytest.raises(L.LetkfError):
        L.letkf_workspace_size(cfg)


def test_nonpositive_error_variance_is_rejected(lib):
    cfg = _cfg()
    var = np.array([1e-4, 0.0, 1e-4, 1e-4], dtype=np.float32)
    cfg.obs_err_var = var.ctypes.data_as(C.POINTER(C.c_float))
    with pytest.raises(L.LetkfError):
        L.letkf_workspace_size(cfg)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.letkf_sync(None) == L.LETKF_EINVAL
    assert lib.letkf_destroy(None) == L.LETKF_OK
    assert lib.lbm_forecast(None, 1) == L.LETKF_EINVAL
    assert lib.letkf_analyze(None, None, 0) == L.LETKF_EINVAL


def test_header_constants_match_the_binding():
    src = open(os.path.join(ROOT, "include", "letkf.h")).read()
    defines = dict(re.findall(r"^#define\s+(LETKF_\w+)\s+\(?(-?\d+)\)?\s*(?:/\*|$)", src,
                              flags=re.M))
    checked = 0
    for name, value in defines.items():
        if hasattr(L, name):
            assert getattr(L, name) == int(value), name
            checked += 1
    for name in ("LETKF_LOC_GC", "LETKF_EIG_SPLIT", "LETKF_MIXED", "LETKF_ENOMEM"):
        assert name in defines and hasattr(L, name), name
    assert checked >= 20
    scratch = re.search(r"#define\s+LETKF_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", src)
    assert int(scratch.group(1)) << int(scratch.group(2)) == L.LETKF_NOALLOC_SCRATCH_BYTES


def test_gaspari_cohn_localization_needs_a_radius(lib):
    assert L.letkf_workspace_size(_cfg(loc_kind=L.LETKF_LOC_GC)) > 0
    with pytest.raises(L.LetkfError):
        L.letkf_workspace_size(_cfg(loc_kind=L.LETKF_LOC_GC, loc_radius=0.0))


def test_eigensolver_workspace_query_and_argument_checks(lib):
    # host-side checks only: none of these calls reaches the device
    small = L.letkf_eigh_workspace_bytes(1000, 32)
    assert small > 1000 * (32 * 32 + 4 * 32) * 8
    assert L.letkf_eigh_workspace_bytes(4000, 32) > 3 * small
    assert L.letkf_eigh_workspace_bytes(-1, 32) == 0
    assert L.letkf_eigh_workspace_bytes(10, 1) == 0
    assert L.letkf_eigh_workspace_bytes(10, 129) == 0
    fake = 1 << 20                                    # never dereferenced by these calls
    assert L.letkf_eigh_batch_ws(0, 32, fake, fake, 0, 0, 0, 0, None) == L.LETKF_OK
    assert L.letkf_eigh_batch_ws(4, 1, fake, fake, 0, 0, fake, 1 << 20, None) == L.LETKF_EINVAL
    assert L.letkf_eigh_batch_ws(4, 32, fake, fake, 0, 2, fake, 1 << 20, None) == L.LETKF_EINVAL
    assert L.letkf_eigh_batch_ws(4, 32, 0, fake, 0, 0, fake, 1 << 20, None) == L.LETKF_EINVAL
    need = L.letkf_eigh_workspace_bytes(4, 32)
    assert L.letkf_eigh_batch_ws(4, 32, fake, fake, 0, 0, fake, need - 1, None) \
        == L.LETKF_ENOMEM
    assert L.letkf_eigh_batch_ws(4, 32, fake, fake, 0, 0, fake + 8, need, None) \
        == L.LETKF_ENOMEM
    assert L.letkf_eigh_batch_ws(4, 32, fake, fake, 0, 0, 0, need, None) == L.LETKF_ENOMEM


@pytest.mark.parametrize("kappa,n,bound", [(1e2, 8, 5e-9), (1e3, 10, 1e-8), (1e4, 12, 2e-8),
                                           (1e5, 14, 3e-8), (1e6, 16, 4e-8)])
def test_rational_coefficients_are_zolotarevs(lib, kappa, n, bound):
    # The EVD-free schedule's coefficients (host code in the library): poles and residues of
    # the n-term approximation of t^-1/2 on [1/kappa, 1].  Checked against Zolotarev's
    # construction evaluated with scipy's Jacobi elliptic functions (poles c_{2l-1} =
    # delta^2 sn^2 / cn^2 at u = (2l-1) K'/(2n), parameter 1 - delta^2) and against the
    # approximation error measured here on a finer grid.
    scipy_special = pytest.importorskip("scipy.special")
    poles, res, err = L.letkf_rational_coefficients(kappa, n)
    d2 = 1.0 / kappa
    m = 1.0 - d2
    Kp = scipy_special.ellipk(m)
    sn, cn, _, _ = scipy_special.ellipj(np.arange(1, 2 * n, 2) * Kp / (2 * n), m)
    assert np.allclose(poles, d2 * sn ** 2 / cn ** 2, rtol=1e-10, atol=0)
    assert (poles > 0).all() and (res > 0).all()
    t = np.logspace(-np.log10(kappa), 0, 300001)
    approx = (res[None, :] / (t[:, None] + poles[None, :])).sum(1)
    measured = np.abs(np.sqrt(t) * approx - 1.0).max()
    assert measured < bound and abs(measured - err) < 0.05 * measured + 1e-12
    # equioscillation: the error reaches +-max at both ends of the interval
    ends = np.sqrt(t[[0, -1]]) * approx[[0, -1]] - 1.0
    assert np.allclose(np.abs(ends), measured, rtol=0.05)


def test_rational_coefficients_reject_bad_arguments(lib):
    for kappa, n in [(1.0, 8), (1e13, 8), (100.0, 0), (100.0, 17)]:
        with pytest.raises(L.LetkfError):
            L.letkf_rational_coefficients(kappa, n)


@pytest.mark.parametrize("kappa,n,bound", [(1.0002, 1, 1e-8), (1.005, 2, 2e-8), (1.035, 3, 2e-8),
                                           (1.1, 4, 2e-8), (2.0, 10, 2e-8), (16.0, 36, 2e-8),
                                           (3.0, 6, 1e-3)])
def test_chebyshev_coefficients_interpolate_rsqrt_and_inverse(lib, kappa, n, bound):
    # The Chebyshev schedule's coefficients (host code in the library): the degree-n
    # interpolants of t^-1/2 and t^-1 on [1, kappa] at the first-kind Chebyshev points, in
    # s = (2t - kappa - 1) / (kappa - 1).  Checked against numpy's chebinterpolate (the same
    # definition, an independent implementation) and against the error measured here.
    cheb = np.polynomial.chebyshev
    ca, cb, err = L.letkf_chebyshev_coefficients(kappa, n)
    t_of = lambda s: 1.0 + 0.5 * (s + 1.0) * (kappa - 1.0)
    ra = cheb.chebinterpolate(lambda s: t_of(s) ** -0.5, n)
    rb = cheb.chebinterpolate(lambda s: 1.0 / t_of(s), n)
    assert np.allclose(ca, ra, rtol=0, atol=1e-13) and np.allclose(cb, rb, rtol=0, atol=1e-13)
    t = np.linspace(1.0, kappa, 200001)
    s = (2 * t - kappa - 1) / (kappa - 1)
    measured = max(np.abs(cheb.chebval(s, ca) * np.sqrt(t) - 1).max(),
                   np.abs(cheb.chebval(s, cb) * t - 1).max())
    assert measured < bound and abs(measured - err) < 0.05 * measured + 1e-15
    # the degrees the schedule uses are the smallest that reach 2e-8
    if bound == 2e-8:
        assert L.letkf_chebyshev_coefficients(kappa, n - 1)[2] > 2e-8


def test_chebyshev_coefficients_reject_bad_arguments(lib):
    for kappa, n in [(1.0, 8), (1e7, 8), (2.0, 0), (2.0, 257)]:
        with pytest.raises(L.LetkfError):
            L.letkf_chebyshev_coefficients(kappa, n)
