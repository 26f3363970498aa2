"""Thin ctypes binding of libletkf (``include/letkf.h``), same names as the C entry points.

Only argument marshalling happens here: every step of the forecast and the
analysis runs in the library's CUDA kernels.  PyTorch supplies device memory
(the handle's workspace) and the CUDA stream.  There is no CPU fallback: if the
shared library has not been built, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB

LETKF_OK = 0
LETKF_EINVAL = -1
LETKF_ENOMEM = -2
LETKF_ENOTCONV = -3
LETKF_ENONFINITE = -4
LETKF_ETIMEOUT = -5
LETKF_ECUDA = -6
LETKF_ESTATE = -7

LETKF_HOST = 0
LETKF_DEVICE = 1

LETKF_OBS_RHO = 1
LETKF_OBS_U = 2
LETKF_OBS_V = 4

LETKF_LOC_NONE = 0
LETKF_LOC_GAUSS = 1
LETKF_LOC_GC = 2

LETKF_FP32 = 0
LETKF_MIXED = 1
LETKF_EIG_AUTO = 0
LETKF_EIG_FUSED = 1
LETKF_EIG_SPLIT = 2
LETKF_EIG_SPLIT_CHECK = 3
LETKF_EIG_RATIONAL = 4
LETKF_EIG_CHEBYSHEV = 5
LETKF_GRAM_AUTO = 0
LETKF_GRAM_PIPE = 1
LETKF_GRAM_TEAM = 2
LETKF_GRAM_TENSOR = 3

# Every symbol include/letkf.h declares, in declaration order.
EXPORTED = (
    "letkf_workspace_size", "letkf_init", "letkf_sync", "letkf_destroy", "letkf_strerror",
    "letkf_get_stats", "letkf_enable_timing", "letkf_get_timings", "letkf_set_state", "letkf_get_state", "letkf_set_deviation",
    "letkf_get_deviation", "letkf_set_macro", "lbm_forecast",
    "letkf_get_obs", "letkf_analyze", "letkf_analyze_probe", "letkf_cycle",
    "letkf_local_analysis_noalloc", "letkf_eigh_batch", "letkf_eigh_workspace_bytes",
    "letkf_eigh_batch_ws", "letkf_group_analyze", "letkf_group_cycle",
    "letkf_fp32_peak_grid", "letkf_fp32_peak_run", "letkf_rational_coefficients",
    "letkf_chebyshev_coefficients", "letkf_get_work_counts",
)

LETKF_NOALLOC_SCRATCH_BYTES = 64 << 20


class letkf_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("k", C.c_int32), ("n_aux", C.c_int32),
        ("tau", C.c_float), ("force", C.POINTER(C.c_float)),
        ("n_obs", C.c_int32), ("obs_xy", C.POINTER(C.c_int32)), ("obs_vars", C.c_int32),
        ("obs_err_var", C.POINTER(C.c_float)), ("loc_kind", C.c_int32),
        ("loc_radius", C.c_float), ("loc_cutoff2", C.c_float), ("infl", C.c_float),
        ("precision", C.c_int32), ("eig_schedule", C.c_int32), ("gram_tile", C.c_int32),
        ("chunk_bytes", C.c_int64),
        ("stream", C.c_void_p),
    ]


class letkf_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_points", C.c_int32), ("n_zero_obs", C.c_int32),
                ("max_local_obs", C.c_int32), ("mean_local_obs", C.c_double),
                ("n_chunks", C.c_int32), ("eig_schedule", C.c_int32), ("cuda_error", C.c_int32),
                ("cycle_kernels", C.c_int32), ("gram_tile", C.c_int32)]


class letkf_timings(C.Structure):
    _fields_ = [("forecast_ms", C.c_float), ("forecast_steps", C.c_int32), ("obs_ms", C.c_float),
                ("transpose_in_ms", C.c_float), ("gram_ms", C.c_float), ("eigen_ms", C.c_float),
                ("transpose_out_ms", C.c_float), ("n_chunks", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class letkf_probe(C.Structure):
    _fields_ = [("n_points", C.c_int32), ("points", C.POINTER(C.c_int32)),
                ("nloc", C.POINTER(C.c_int32)), ("gram", C.POINTER(C.c_float)),
                ("cvec", C.POINTER(C.c_float)), ("eigval", C.POINTER(C.c_float)),
                ("xf", C.POINTER(C.c_float))]


class LetkfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


_lib = None


def load(path: str = LIB):
    """Load libletkf.so (built in tree by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libletkf.so not found at {path}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "letkf_workspace_size": (C.c_int, [C.POINTER(letkf_config), C.POINTER(C.c_size_t)]),
        "letkf_init": (C.c_int, [C.POINTER(letkf_config), P, C.c_size_t, C.POINTER(P)]),
        "letkf_sync": (C.c_int, [P]),
        "letkf_destroy": (C.c_int, [P]),
        "letkf_strerror": (C.c_char_p, [C.c_int]),
        "letkf_get_stats": (C.c_int, [P, C.POINTER(letkf_stats)]),
        "letkf_enable_timing": (C.c_int, [P, C.c_int32]),
        "letkf_get_timings": (C.c_int, [P, C.POINTER(letkf_timings)]),
        "letkf_set_state": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32]),
        "letkf_get_state": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32]),
        "letkf_set_deviation": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32]),
        "letkf_get_deviation": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32]),
        "letkf_set_macro": (C.c_int, [P, P, P, P, C.c_int32, C.c_int32, C.c_int32]),
        "lbm_forecast": (C.c_int, [P, C.c_int32]),
        "letkf_get_obs": (C.c_int, [P, P, C.c_int32]),
        "letkf_analyze": (C.c_int, [P, P, C.c_int32]),
        "letkf_analyze_probe": (C.c_int, [P, P, C.c_int32, C.POINTER(letkf_probe)]),
        "letkf_cycle": (C.c_int, [P, C.c_int32, P, C.c_int32]),
        "letkf_local_analysis_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P, P,
                                                   C.c_float, P, P]),
        "letkf_eigh_batch": (C.c_int, [C.c_int32, C.c_int32, P, P, P, C.c_int32, P]),
        "letkf_eigh_workspace_bytes": (C.c_size_t, [C.c_int32, C.c_int32]),
        "letkf_eigh_batch_ws": (C.c_int, [C.c_int32, C.c_int32, P, P, P, C.c_int32, P,
                                          C.c_size_t, P]),
        "letkf_group_analyze": (C.c_int, [P, P, C.c_int32, C.c_int32]),
        "letkf_group_cycle": (C.c_int, [P, C.c_int32, C.c_int32, P, C.c_int32]),
        "letkf_fp32_peak_grid": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "letkf_fp32_peak_run": (C.c_int, [C.c_int32, P, C.POINTER(C.c_int64), P]),
        "letkf_rational_coefficients": (C.c_double, [C.c_double, C.c_int32,
                                                     C.POINTER(C.c_double),
                                                     C.POINTER(C.c_double)]),
        "letkf_chebyshev_coefficients": (C.c_double, [C.c_double, C.c_int32,
                                                      C.POINTER(C.c_double),
                                                      C.POINTER(C.c_double)]),
        "letkf_get_work_counts": (C.c_int, [P, C.POINTER(C.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().letkf_strerror(int(code)).decode()


def _check(rc, where):
    if rc != LETKF_OK:
        raise LetkfError(rc, where)


# ---------------------------------------------------------------- raw ABI, same names

def letkf_workspace_size(cfg: letkf_config) -> int:
    n = C.c_size_t(0)
    _check(load().letkf_workspace_size(C.byref(cfg), C.byref(n)), "letkf_workspace_size")
    return n.value


def letkf_init(cfg: letkf_config, workspace_ptr: int = 0, workspace_bytes: int = 0) -> int:
    h = C.c_void_p(0)
    _check(load().letkf_init(C.byref(cfg), C.c_void_p(workspace_ptr or None), workspace_bytes,
                             C.byref(h)), "letkf_init")
    return h.value


def letkf_sync(h: int) -> int:
    return load().letkf_sync(C.c_void_p(h))


def letkf_destroy(h: int) -> None:
    load().letkf_destroy(C.c_void_p(h))


def letkf_get_stats(h: int) -> letkf_stats:
    st = letkf_stats()
    _check(load().letkf_get_stats(C.c_void_p(h), C.byref(st)), "letkf_get_stats")
    return st


def letkf_enable_timing(h, on):
    _check(load().letkf_enable_timing(C.c_void_p(h), int(bool(on))), "letkf_enable_timing")


def letkf_get_timings(h) -> letkf_timings:
    t = letkf_timings()
    _check(load().letkf_get_timings(C.c_void_p(h), C.byref(t)), "letkf_get_timings")
    return t


def letkf_set_state(h, ptr, m0, count, where):
    _check(load().letkf_set_state(C.c_void_p(h), C.c_void_p(ptr), m0, count, where), "letkf_set_state")


def letkf_get_state(h, ptr, m0, count, where):
    _check(load().letkf_get_state(C.c_void_p(h), C.c_void_p(ptr), m0, count, where), "letkf_get_state")


def letkf_set_deviation(h, ptr, m0, count, where):
    _check(load().letkf_set_deviation(C.c_void_p(h), C.c_void_p(ptr), m0, count, where),
           "letkf_set_deviation")


def letkf_get_deviation(h, ptr, m0, count, where):
    _check(load().letkf_get_deviation(C.c_void_p(h), C.c_void_p(ptr), m0, count, where),
           "letkf_get_deviation")


def letkf_set_macro(h, rho, ux, uy, m0, count, where):
    _check(load().letkf_set_macro(C.c_void_p(h), C.c_void_p(rho), C.c_void_p(ux), C.c_void_p(uy),
                                  m0, count, where), "letkf_set_macro")


def lbm_forecast(h, nsteps):
    _check(load().lbm_forecast(C.c_void_p(h), int(nsteps)), "lbm_forecast")


def letkf_get_obs(h, ptr, where):
    _check(load().letkf_get_obs(C.c_void_p(h), C.c_void_p(ptr), where), "letkf_get_obs")


def letkf_analyze(h, yo_ptr, where):
    _check(load().letkf_analyze(C.c_void_p(h), C.c_void_p(yo_ptr), where), "letkf_analyze")


def letkf_analyze_probe(h, yo_ptr, where, probe: letkf_probe):
    _check(load().letkf_analyze_probe(C.c_void_p(h), C.c_void_p(yo_ptr), where, C.byref(probe)),
           "letkf_analyze_probe")


def letkf_cycle(h, nsteps, yo_ptr, where):
    _check(load().letkf_cycle(C.c_void_p(h), int(nsteps), C.c_void_p(yo_ptr), where), "letkf_cycle")


def letkf_local_analysis_noalloc(npts, k, lmaxv, dy_ptr, d_ptr, rinv_ptr, infl, x_ptr, stream):
    """Local analyses of npts padded local problems with no device allocation (device pointers).
    Returns the status code (LETKF_OK, LETKF_EINVAL, LETKF_ENOTCONV, ...) without raising."""
    return load().letkf_local_analysis_noalloc(int(npts), int(k), int(lmaxv), C.c_void_p(dy_ptr),
                                               C.c_void_p(d_ptr), C.c_void_p(rinv_ptr),
                                               float(infl), C.c_void_p(x_ptr), C.c_void_p(stream))


def letkf_eigh_batch(npts, k, q_ptr, eigval_ptr, evec_ptr, refine, stream):
    """Eigenpairs of npts symmetric k x k matrices (device pointers; evec may be 0).
    Returns the status code without raising."""
    return load().letkf_eigh_batch(int(npts), int(k), C.c_void_p(q_ptr), C.c_void_p(eigval_ptr),
                                   C.c_void_p(evec_ptr or None), int(refine),
                                   C.c_void_p(stream))


def letkf_eigh_workspace_bytes(npts, k):
    """Device bytes letkf_eigh_batch_ws needs for npts matrices of order k (0: invalid)."""
    return int(load().letkf_eigh_workspace_bytes(int(npts), int(k)))


def letkf_eigh_batch_ws(npts, k, q_ptr, eigval_ptr, evec_ptr, refine, ws_ptr, ws_bytes, stream):
    """letkf_eigh_batch on the split schedule with a caller workspace (device pointers).
    Returns the status code without raising."""
    return load().letkf_eigh_batch_ws(int(npts), int(k), C.c_void_p(q_ptr),
                                      C.c_void_p(eigval_ptr), C.c_void_p(evec_ptr or None),
                                      int(refine), C.c_void_p(ws_ptr or None), int(ws_bytes),
                                      C.c_void_p(stream))


def letkf_fp32_peak_grid():
    """(blocks, threads) of the FP32 FMA microbenchmark launch on the current device."""
    b, t = C.c_int32(0), C.c_int32(0)
    _check(load().letkf_fp32_peak_grid(C.byref(b), C.byref(t)), "letkf_fp32_peak_grid")
    return b.value, t.value


def letkf_fp32_peak_run(iters, out_ptr, stream):
    """Launch the FP32 FMA microbenchmark on stream; returns the flops it executes."""
    n = C.c_int64(0)
    _check(load().letkf_fp32_peak_run(int(iters), C.c_void_p(out_ptr), C.byref(n),
                                      C.c_void_p(stream)), "letkf_fp32_peak_run")
    return n.value


def letkf_rational_coefficients(kappa_max, n):
    """(poles, residues, max relative error) of the library's n-term rational approximation
    of t^-1/2 on [1/kappa_max, 1] (host computation, no GPU needed)."""
    p = (C.c_double * int(n))()
    r = (C.c_double * int(n))()
    err = load().letkf_rational_coefficients(float(kappa_max), int(n), p, r)
    if err < 0:
        raise LetkfError(LETKF_EINVAL, "letkf_rational_coefficients")
    return np.array(p[:]), np.array(r[:]), float(err)


def letkf_chebyshev_coefficients(kappa_max, n):
    """(c_rsqrt, c_inv, max relative error): the library's degree-n Chebyshev interpolants of
    t^-1/2 and t^-1 on [1, kappa_max] (host computation, no GPU needed)."""
    a = (C.c_double * (int(n) + 1))()
    b = (C.c_double * (int(n) + 1))()
    err = load().letkf_chebyshev_coefficients(float(kappa_max), int(n), a, b)
    if err < 0:
        raise LetkfError(LETKF_EINVAL, "letkf_chebyshev_coefficients")
    return np.array(a[:]), np.array(b[:]), float(err)


def _group_arrays(exps, yos):
    hs = (C.c_void_p * len(exps))(*[e.h for e in exps])
    wheres, ptrs, keep = set(), [], []
    for y in yos:
        y = _f32(y) if isinstance(y, np.ndarray) else y
        keep.append(y)
        ptr, where = _ptr_where(y)
        ptrs.append(ptr)
        wheres.add(where)
    if len(wheres) > 1:
        raise ValueError("observations of a group must all be on the host or all on the device")
    where = wheres.pop() if wheres else LETKF_HOST
    return hs, (C.c_void_p * len(ptrs))(*ptrs), where, keep


def letkf_group_analyze(exps, yos):
    """One grouped analysis of the Experiments `exps` with observations `yos` (see letkf.h)."""
    hs, ys, where, keep = _group_arrays(exps, yos)
    _check(load().letkf_group_analyze(hs, ys, len(exps), where), "letkf_group_analyze")


def letkf_group_cycle(exps, nsteps, yos):
    """One grouped cycle (forecasts + grouped analysis), replayed from a CUDA graph."""
    hs, ys, where, keep = _group_arrays(exps, yos)
    _check(load().letkf_group_cycle(hs, len(exps), int(nsteps), ys, where), "letkf_group_cycle")


# ---------------------------------------------------------------- marshalling helpers

def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _ptr_where(t):
    """(address, LETKF_HOST/DEVICE) of a float32 numpy array or torch tensor (kept alive by caller)."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32 or not t.flags.c_contiguous:
            raise ValueError("expected a C-contiguous float32 array")
        return t.ctypes.data, LETKF_HOST
    import torch
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 tensor")
    return t.data_ptr(), (LETKF_DEVICE if t.is_cuda else LETKF_HOST)


class Experiment:
    """One DA experiment: owns a libletkf handle, its torch-allocated workspace and stream.

    nx, ny, k, tau          periodic grid, ensemble size, BGK relaxation time
    obs_xy, obs_err_var     [L][2] observation points and the [L*V] diagonal of R
    obs_vars                LETKF_OBS_* bits (rho, u, v)
    loc_radius, loc_kind    radius r and LETKF_LOC_GAUSS / LETKF_LOC_GC; loc_radius=None
                            means no localization; loc_cutoff2 overrides the default cutoff
                            (40/3) r^2
    force, n_aux, infl      [2][ny][nx] body force, auxiliary members (never analysed, e.g. a
                            nature run), multiplicative inflation
    precision, eig_schedule LETKF_FP32 / LETKF_MIXED, LETKF_EIG_*
    gram_tile               LETKF_GRAM_* (FP32 Gram tile schedule for k >= 17; AUTO tunes)
    chunk_bytes, stream, device   Gram chunk budget (0: library default), torch stream, device
    """

    def __init__(self, nx, ny, k, tau, obs_xy, obs_err_var, obs_vars=LETKF_OBS_U | LETKF_OBS_V,
                 loc_radius=None, loc_cutoff2=0.0, force=None, n_aux=0, infl=1.0,
                 precision=LETKF_FP32, chunk_bytes=0, stream=None, device=None,
                 eig_schedule=LETKF_EIG_AUTO, loc_kind=LETKF_LOC_GAUSS,
                 gram_tile=LETKF_GRAM_AUTO):
        import torch
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.nx, self.ny, self.k, self.n_aux = int(nx), int(ny), int(k), int(n_aux)
        self.nmem = self.k + self.n_aux
        self._obs_xy = np.ascontiguousarray(np.asarray(obs_xy, dtype=np.int32).reshape(-1, 2))
        self._obs_var = _f32(obs_err_var).reshape(-1)
        self._force = None if force is None else _f32(force).reshape(2, ny, nx)
        self.V = bin(int(obs_vars) & 7).count("1")
        self.L = self._obs_xy.shape[0]
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        cfg = letkf_config()
        cfg.nx, cfg.ny, cfg.k, cfg.n_aux = self.nx, self.ny, self.k, self.n_aux
        cfg.tau = float(tau)
        cfg.force = (self._force.ctypes.data_as(C.POINTER(C.c_float)) if self._force is not None
                     else C.POINTER(C.c_float)())
        cfg.n_obs = self.L
        cfg.obs_xy = self._obs_xy.ctypes.data_as(C.POINTER(C.c_int32))
        cfg.obs_vars = int(obs_vars)
        cfg.obs_err_var = self._obs_var.ctypes.data_as(C.POINTER(C.c_float))
        if loc_radius is None:
            cfg.loc_kind, cfg.loc_radius = LETKF_LOC_NONE, 0.0
        else:
            cfg.loc_kind, cfg.loc_radius = int(loc_kind), float(loc_radius)
        cfg.loc_cutoff2 = float(loc_cutoff2)
        cfg.infl = float(infl)
        cfg.precision = int(precision)
        cfg.eig_schedule = int(eig_schedule)
        cfg.gram_tile = int(gram_tile)
        cfg.chunk_bytes = int(chunk_bytes)
        cfg.stream = self.stream.cuda_stream
        self.cfg = cfg
        self.workspace_bytes = letkf_workspace_size(cfg)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self.h = letkf_init(cfg, self.workspace.data_ptr(), self.workspace_bytes)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            letkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self) -> int:
        return letkf_sync(self.h)

    def stats(self) -> letkf_stats:
        return letkf_get_stats(self.h)

    def work_counts(self) -> dict:
        """Cumulative counts of the Chebyshev transform (waits for the handle's stream)."""
        c = (C.c_int64 * 3)()
        _check(load().letkf_get_work_counts(self.h, c), "letkf_get_work_counts")
        return {"cheb_points": c[0], "cheb_products": c[1], "cheb_handed_on": c[2]}

    def enable_timing(self, on=True):
        letkf_enable_timing(self.h, on)

    def timings(self) -> dict:
        return letkf_get_timings(self.h).as_dict()

    # -- state
    def set_state(self, f, m0=0):
        f = _f32(f) if isinstance(f, np.ndarray) else f
        ptr, where = _ptr_where(f)
        count = int(np.prod(f.shape)) // (9 * self.nx * self.ny)
        letkf_set_state(self.h, ptr, m0, count, where)

    def get_state(self, m0=0, count=None):
        count = self.nmem - m0 if count is None else count
        out = np.empty((count, 9, self.ny, self.nx), dtype=np.float32)
        letkf_get_state(self.h, out.ctypes.data, m0, count, LETKF_HOST)
        return out

    def get_deviation(self, m0=0, count=None):
        """Device state g = f - w_q (FP32 weights), [count, 9, ny, nx] float32."""
        count = self.nmem - m0 if count is None else count
        out = np.empty((count, 9, self.ny, self.nx), dtype=np.float32)
        letkf_get_deviation(self.h, out.ctypes.data, m0, count, LETKF_HOST)
        return out

    def set_deviation(self, g, m0=0):
        g = _f32(g) if isinstance(g, np.ndarray) else g
        ptr, where = _ptr_where(g)
        count = int(np.prod(g.shape)) // (9 * self.nx * self.ny)
        letkf_set_deviation(self.h, ptr, m0, count, where)

    def set_macro(self, rho, ux, uy, m0=0):
        arrs = [_f32(a) for a in (rho, ux, uy)]
        count = arrs[0].size // (self.nx * self.ny)
        letkf_set_macro(self.h, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                        m0, count, LETKF_HOST)

    # -- hot path
    def forecast(self, nsteps):
        lbm_forecast(self.h, nsteps)

    def get_obs(self):
        out = np.empty((self.nmem, self.L * self.V), dtype=np.float32)
        letkf_get_obs(self.h, out.ctypes.data, LETKF_HOST)
        return out

    def analyze(self, yo):
        yo = _f32(yo) if isinstance(yo, np.ndarray) else yo
        ptr, where = _ptr_where(yo)
        letkf_analyze(self.h, ptr, where)

    def analyze_probe(self, yo, points, want=("nloc", "gram", "cvec", "eigval", "xf")):
        yo = _f32(yo) if isinstance(yo, np.ndarray) else yo
        ptr, where = _ptr_where(yo)
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1))
        n, k = pts.size, self.k
        out = {"nloc": np.zeros(n, np.int32), "gram": np.zeros((n, k, k), np.float32),
               "cvec": np.zeros((n, k), np.float32), "eigval": np.zeros((n, k), np.float32),
               "xf": np.zeros((n, 9, k), np.float32)}
        pr = letkf_probe()
        pr.n_points = n
        pr.points = pts.ctypes.data_as(C.POINTER(C.c_int32))
        for name in ("nloc", "gram", "cvec", "eigval", "xf"):
            typ = C.c_int32 if name == "nloc" else C.c_float
            setattr(pr, name, out[name].ctypes.data_as(C.POINTER(typ)) if name in want
                    else C.POINTER(typ)())
        letkf_analyze_probe(self.h, ptr, where, pr)
        return {name: out[name] for name in want}

    def cycle(self, nsteps, yo):
        yo = _f32(yo) if isinstance(yo, np.ndarray) else yo
        ptr, where = _ptr_where(yo)
        letkf_cycle(self.h, nsteps, ptr, where)
