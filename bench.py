#!/usr/bin/env python3
"""Benchmark of the LBM-LETKF hot path on one GB300 (or N independent replicas).

One step = one data-assimilation cycle of the forced-turbulence workload: 100 D2Q9
steps of the k-member ensemble, then one LETKF analysis at every grid point
(observation operator, transpose, localized Gram, eigensolve/transform/update,
transpose back), replayed as one CUDA graph through the C ABI.

value   LETKF grid-point analyses per second, whole job (sum over ranks), inputs
        resident in HBM, L2 flushed (256 MiB write) between timed cycles.
e2e     the same metric through the public API with host buffers: the cycle's
        observations copied from pinned host memory each step and the analysis
        ensemble in observation space read back to the host.
The observations are those of a nature run stored in advance (the paper's OSSE,
Sec. V), so the truth is not advanced inside the timed region.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the oracle is the reference implementation for this method).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LETKF grid-pt analyses/s + p99 cycle latency, mixed vs FP32 at stated error"
UNIT = "grid-pt analyses/s"
FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128
SMS = 152

# Algorithmic work per unit:
#   lbm_step      72 B per node and member per launch (one FP32 read and one write of the nine
#                 populations; two time steps per launch) + 8 B per node of force
#   transpose     2 x 36 k B per grid point (read + write of the 9 x k block)
#   obs_operator  36 B per (observation point, member) read + 4 V B per (point, member) written x2
#   gram          k (k + 1) flops per local observed scalar per grid point (the upper triangle
#                 of the symmetric A, one multiply-add per entry) + 2 k for c
#   eigen_update  eigenvector schedules (FUSED, SPLIT): 11 k^3 flops per grid point (symmetric
#                 EVD with vectors ~9 k^3, transform ~2 k^3); EVD-free schedule (RATIONAL):
#                 4/3 k^3 (Householder tridiagonalization) + 40 k^2 (the reflectors applied to
#                 the 10 rows [dX; c] twice) + 36 k (n + 1) (n shifted solves of 9 rows and the
#                 mean's solve, forward and back; n = 8 poles below condition 1e2)


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed cycles (default per workload)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="turb1024_k64")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--chunk-mb", type=float, default=0.0,
                   help="Gram buffer per analysis chunk in MiB (0: the library default)")
    p.add_argument("--eig-schedule", choices=sorted(EIG_SCHEDULES), default="auto",
                   help="eigensolve schedule (auto: the handle's autotuner picks)")
    p.add_argument("--cpu-sample-seconds", type=float, default=12.0)
    p.add_argument("--precision", choices=["fp32", "mixed", "both"], default="both",
                   help="fp32: the plain form only; mixed: the split-precision form only; "
                        "both: fp32 as the headline value, mixed reported beside it")
    p.add_argument("--serve-requests", type=int, default=60,
                   help="serve_cfg5: requests in the Poisson stream")
    p.add_argument("--serve-compare-priority", action="store_true",
                   help="serve_cfg5: also serve the FP32 stream with one stream priority for "
                        "every slot, for comparison")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="serve_cfg5: wall-time cap of each form's run (unfinished work is "
                        "counted by completed cycles)")
    p.add_argument("--serve-budget-gb", type=float, default=200.0,
                   help="serve_cfg5: HBM budget for resident experiments")
    p.add_argument("--serve-max-active", type=int, default=8,
                   help="serve_cfg5: most experiments on the GPU at once")
    p.add_argument("--no-error-check", action="store_true",
                   help="skip the error measurement against the FP64 oracle")
    p.add_argument("--_oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--_oracle-steps", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--_oracle-error-prep", default=None, help=argparse.SUPPRESS)
    return p.parse_args(argv)


DEFAULT_STEPS = {"turb256_k32": 200, "turb1024_k64": 10, "tgv32_k8": 200, "turb256_k64": 50}


# ----------------------------------------------------------------------------- ranks

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, device=None) -> float:
    """Max of a float over ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_per_rank: float, world: int) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    return units_per_rank * world / seconds_per_rank


# ----------------------------------------------------------------------------- clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        text = open(self.path).read()
        os.unlink(self.path)
        return parse_clock_csv(text)


def parse_clock_csv(text: str) -> dict:
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    sm, smax, reasons, power = [], [], set(), []
    for line in text.strip().splitlines():
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
            power.append(float(parts[3]))
        except ValueError:
            continue
        for name, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks / roofline

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs"), "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


EIG_SCHEDULES = {"auto": 0, "fused": 1, "split": 2, "rational": 4, "chebyshev": 5}
EIG_NAMES = {1: "fused", 2: "split", 3: "split_check", 4: "rational", 5: "chebyshev"}
GRAM_NAMES = {0: "auto", 1: "pipe", 2: "team", 3: "tensor"}
PEAK_NAMES = {"hbm": "hbm_gbs", "alu": "FP32 FMA peak from the unit counts at max SM clock",
              "tensor": "bf16_tflops_sustained (FP16 operands, same nominal rate)"}


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock (unit counts of the GB300 recipe)."""
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def eigen_flops_per_point(k, schedule):
    """Algorithmic flops of the eigensolve phase per grid point for the schedule in use."""
    if schedule in (4, 5):   # RATIONAL: tridiagonalization, reflector passes, shifted solves
        return 4.0 / 3.0 * k ** 3 + 40.0 * k * k + 36.0 * k * 9
    return 11.0 * k ** 3


def cheb_flops(k, counts):
    """Flops of the CHEBYSHEV schedule for the given counts (points, products, handed on):
    each product R A of the ten rows with the k x k Gram matrix is 20 k^2 flops, the final
    increment and combination 4 k per row; the points passed on cost the RATIONAL count."""
    return (20.0 * k * k * counts["cheb_products"] + 36.0 * k * counts["cheb_points"]
            + eigen_flops_per_point(k, 4) * counts["cheb_handed_on"])


def kernel_work(w, k, npts, mean_local_obs, V, nobs_pts, chunks, steps, schedule=1,
                cheb_counts=None):
    """Algorithmic work of one cycle per kernel: (unit, amount, launches).  For the CHEBYSHEV
    schedule the eigen phase's work follows the device counters of the cycle (cheb_counts);
    without them it falls back to the RATIONAL count."""
    eig = (cheb_flops(k, cheb_counts) if schedule == 5 and cheb_counts
           else eigen_flops_per_point(k, schedule) * npts)
    return {
        # two steps per launch: one read and one write of the state (+ the force) per launch
        "lbm_step": ("GB", (72.0 * npts * k + 8.0 * npts) * (steps // 2 + steps % 2) / 1e9,
                     steps // 2 + steps % 2),
        "obs_operator": ("GB", (36.0 + 8.0 * V) * nobs_pts * k / 1e9, 1),
        "transpose_in": ("GB", 72.0 * k * npts / 1e9, 1),
        "gram": ("TFLOP", (k * (k + 1) + 2 * k) * V * mean_local_obs * npts / 1e12, chunks),
        "eigen_update": ("TFLOP", eig / 1e12, chunks),
        "transpose_out": ("GB", 72.0 * k * npts / 1e9, 1),
    }


def lbm_rates(w, forecast_ms, peaks):
    """D2Q9 throughput of the forecast: million lattice updates per second (all members and
    per member), and the HBM rate a kernel taking one step per launch would need for it
    (72 B per update + the force), as a fraction of the measured copy bandwidth: above 1 only
    with temporal blocking."""
    updates = float(w.n_points) * w.k * w.steps_per_cycle
    mlups = updates / (forecast_ms * 1e-3) / 1e6
    eq_gbs = (72.0 * updates + 8.0 * w.n_points * w.steps_per_cycle) / (forecast_ms * 1e-3) / 1e9
    return {"mlups": mlups, "mlups_per_member": mlups / w.k, "steps_per_launch": 2,
            "single_step_equivalent_gbs": eq_gbs,
            "single_step_equivalent_frac": eq_gbs / peaks["hbm_gbs"]}


def roofline_table(work, ms, peaks, sm_mhz, tensor_gram=False):
    """Per kernel: achieved = algorithmic work / device time against its peak.  The mixed
    form's Gram runs on the tensor cores (FP16 operands: the measured sustained BF16 GEMM
    rate, FP16 and BF16 have the same nominal dense rate); its split form executes 2 tensor
    flops per algorithmic flop ([Xl; Xh] Xh^T), so frac <= 0.5 even at the tensor peak."""
    out = {}
    total = sum(ms.values())
    for name, (unit, amount, launches) in work.items():
        t = ms.get(name, 0.0)
        if t <= 0:
            continue
        if unit == "GB":
            achieved = amount / (t / 1e3)
            peak = peaks["hbm_gbs"]
            out[name] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak}
        elif name == "gram" and tensor_gram:
            achieved = amount / (t / 1e3)
            peak = peaks["bf16_tflops_sustained"]
            out[name] = {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak}
        else:
            achieved = amount / (t / 1e3)
            peak = peaks.get("fp32_tflops") or fp32_peak_tflops(sm_mhz)
            out[name] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak}
        out[name].update({"ms_per_cycle": t, "share": t / total, "launches_per_cycle": launches,
                          "ms_per_launch": t / launches})
    return out


def traffic_for(kernel: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if its source hash still matches."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    ent = d.get(workload, {}).get(kernel)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2308_03310_gb300", "csrc", ent["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent["sha"]:
        return None
    return ent["bytes_per_launch"]


# ----------------------------------------------------------------------------- workload set-up

def spin_up(w, device):
    """Spin up truth + ensemble together on the GPU.  Returns the spin-up experiment (the
    truth is its auxiliary member), a device copy of the members' state at the end of the
    spin-up, and the network, error variances and force of the workload."""
    import numpy as np
    import torch

    from paper_2308_03310_gb300 import letkf as L

    net = w.obs_network()
    V = len(w.obs_vars)
    var = w.obs_error_var(len(net) * V).astype(np.float32)
    fx, fy = w.force()
    force = np.stack([fx, fy]).astype(np.float32)
    kw = dict(obs_vars=L.LETKF_OBS_U | L.LETKF_OBS_V, loc_radius=w.loc_radius, force=force)
    spin = L.Experiment(w.nx, w.ny, w.k, w.tau, net, var, n_aux=1, device=device, **kw)
    ux0, uy0 = w.truth_velocity()
    dux, duy = w.member_perturbations()
    n = w.k + 1
    rho = np.ones((n, w.ny, w.nx), np.float32)
    ux = np.concatenate([ux0[None] + dux, ux0[None]]).astype(np.float32)
    uy = np.concatenate([uy0[None] + duy, uy0[None]]).astype(np.float32)
    spin.set_macro(rho, ux, uy)
    spin.forecast(w.spinup)
    members = torch.empty((w.k, 9, w.ny, w.nx), dtype=torch.float32, device=device)
    torch.cuda.synchronize(device)
    L.letkf_get_deviation(spin.h, members.data_ptr(), 0, w.k, L.LETKF_DEVICE)
    truth = torch.empty((1, 9, w.ny, w.nx), dtype=torch.float32, device=device)
    L.letkf_get_deviation(spin.h, truth.data_ptr(), w.k, 1, L.LETKF_DEVICE)
    torch.cuda.synchronize(device)
    assert spin.sync() == 0
    return spin, members, (net, var, kw), truth


def rmse_run(w, members, truth, setup, device, precision, ncycles, seed_offset=0):
    """Assimilation quality against the synthetic truth (OSSE, Sec. V): the spun-up ensemble and
    its truth (an auxiliary member, advanced but never analysed) cycled ncycles times with
    noisy observations of the truth.  Per cycle the velocity RMSE of the ensemble mean against
    the truth over the whole grid, before (forecast) and after (analysis) the update, and the
    ensemble spread.  Diagnostics only: the moments are formed with torch from the device
    state after each phase."""
    import numpy as np
    import torch

    from paper_2308_03310_gb300 import letkf as L
    net, var, kw = setup
    k = w.k
    exp = L.Experiment(w.nx, w.ny, k, w.tau, net, var, n_aux=1, device=device,
                       precision=precision, **kw)
    torch.cuda.synchronize(device)
    L.letkf_set_deviation(exp.h, members.data_ptr(), 0, k, L.LETKF_DEVICE)
    L.letkf_set_deviation(exp.h, truth.data_ptr(), k, 1, L.LETKF_DEVICE)
    buf = torch.empty((k + 1, 9, w.ny, w.nx), dtype=torch.float32, device=device)
    LV = exp.L * exp.V

    def diag():
        L.letkf_get_deviation(exp.h, buf.data_ptr(), 0, k + 1, L.LETKF_DEVICE)
        torch.cuda.synchronize(device)
        g = buf.double()
        rho = 1.0 + g.sum(1)
        ux = (g[:, [2, 5, 8]].sum(1) - g[:, [0, 3, 6]].sum(1)) / rho
        uy = (g[:, [6, 7, 8]].sum(1) - g[:, [0, 1, 2]].sum(1)) / rho
        err = (ux[:k].mean(0) - ux[k]) ** 2 + (uy[:k].mean(0) - uy[k]) ** 2
        spread = ux[:k].var(0) + uy[:k].var(0)
        return float(err.mean().sqrt()), float(spread.mean().sqrt())

    fc, an, sp = [], [], []
    for c in range(ncycles):
        exp.forecast(w.steps_per_cycle)
        y = exp.get_obs()[k] + w.obs_noise(seed_offset + 5000 + c, LV)
        e, s_ = diag()
        fc.append(e)
        sp.append(s_)
        exp.analyze(y.astype(np.float32))
        an.append(diag()[0])
    rc = exp.sync()
    exp.close()
    if rc:
        raise RuntimeError(f"RMSE cycles failed: {L.strerror(rc)}")
    late = slice(ncycles // 2, ncycles)
    return {"forecast_rmse": float(np.mean(fc[late])), "analysis_rmse": float(np.mean(an[late])),
            "forecast_spread": float(np.mean(sp[late])), "first_forecast_rmse": fc[0],
            "analysis_below_forecast_fraction": float(np.mean(np.array(an) < np.array(fc)))}


def make_experiment(w, members, setup, device, precision, eig_schedule=0, chunk_bytes=0):
    """A fresh experiment of the workload starting from the spun-up members."""
    import torch

    from paper_2308_03310_gb300 import letkf as L
    net, var, kw = setup
    exp = L.Experiment(w.nx, w.ny, w.k, w.tau, net, var, device=device, precision=precision,
                       eig_schedule=eig_schedule, chunk_bytes=chunk_bytes, **kw)
    torch.cuda.synchronize(device)
    L.letkf_set_deviation(exp.h, members.data_ptr(), 0, w.k, L.LETKF_DEVICE)
    assert exp.sync() == 0
    return exp


def nature_observations(spin, w, ncycles, seed_offset=0):
    import numpy as np
    LV = spin.L * spin.V
    yos = []
    for c in range(ncycles):
        spin.forecast(w.steps_per_cycle)
        y = spin.get_obs()[w.k]                      # the nature run is the auxiliary member
        if not np.all(np.isfinite(y)):
            raise RuntimeError("nature run produced non-finite observations")
        yos.append((y + w.obs_noise(c + seed_offset, LV)).astype(np.float32))
    return yos


# ----------------------------------------------------------------------------- CPU oracle leg
#
# Everything below that touches oracle/ runs in a CPU subprocess of this script (the CPU
# baseline, the reference arm and the oracle side of the error measurement); the GPU process
# never imports the oracle.

SUB_EDGE = 256          # the oracle's D2Q9 step and moments are timed on a sub-block this wide


class OracleSample:
    """The FP64 oracle, as it stands, on a bounded sample of one cycle of a workload.

    One cycle = steps_per_cycle D2Q9 steps of the k members, the observation operator and one
    local analysis per grid point.  Sampled: the oracle's D2Q9 step and its moments on a
    periodic sub-block of at most 256 x 256 nodes (the cost per node is the same on any grid),
    scaled by the node count; the oracle's local analysis (local observation search over the
    full network, Gram matrix, eigendecomposition, transform, update) at random grid points of
    the full grid, scaled by the point count."""

    def __init__(self, wname: str):
        import numpy as np

        import synth
        from oracle import lbm, obs as oobs
        self.np, self.lbm, self.oobs = np, lbm, oobs
        w = self.w = synth.WORKLOADS[wname]
        k = w.k
        sx, sy = min(w.nx, SUB_EDGE), min(w.ny, SUB_EDGE)
        self.sub = (sx, sy)
        self.scale = w.n_points / (sx * sy)
        ux0, uy0 = synth.taylor_green_velocity(sx, sy, 0.05)
        self.f = np.empty((k, 9, sy, sx))
        for m in range(k):
            self.f[m] = lbm.equilibrium(np.ones((sy, sx)), ux0 + synth.gaussian((sy, sx), 5e-3, m),
                                        uy0 + synth.gaussian((sy, sx), 5e-3, 1000 + m))
        fx, fy = w.force()
        self.fx, self.fy = fx[:sy, :sx], fy[:sy, :sx]
        self.net_sub = synth.regular_obs_network(sx, sy, w.obs_stride)
        # forecast observations of the full network (a random flow's equilibria at the
        # observation points), for the local analyses
        self.net = w.obs_network()
        L = len(self.net)
        rx = synth.gaussian((k, 1, L), 0.02, 21)
        ry = synth.gaussian((k, 1, L), 0.02, 22)
        strip = lbm.equilibrium(np.ones((k, 1, L)), rx, ry)
        strip_xy = np.stack([np.arange(L), np.zeros(L, dtype=np.int64)], axis=1)
        self.Yf = oobs.observe(strip, strip_xy, oobs.VAR_U | oobs.VAR_V)
        self.yo = self.Yf.mean(0) + synth.gaussian(self.Yf.shape[1], w.obs_sigma, 7)
        self.var = w.obs_error_var(self.Yf.shape[1])
        self.ybar, self.dY = oobs.ensemble_obs(self.Yf)
        self.c2 = synth.loc_cutoff2(w.loc_radius)
        self.rng = synth.generator(11)

    def step(self, seconds: float) -> dict:
        """One sample of about `seconds` of CPU work, extrapolated to one cycle."""
        from oracle import letkf as oletkf
        np, lbm, oobs, w = self.np, self.lbm, self.oobs, self.w
        sx, sy = self.sub
        t0 = time.perf_counter()
        nl = 0
        while nl < 1 or (time.perf_counter() - t0 < 0.2 * seconds and nl < 5):
            self.f = lbm.step(self.f, w.tau, self.fx, self.fy)
            nl += 1
        t_lbm = (time.perf_counter() - t0) / nl * self.scale
        t0 = time.perf_counter()
        oobs.observe(self.f, self.net_sub, oobs.VAR_U | oobs.VAR_V)
        t_obs = (time.perf_counter() - t0) * self.scale
        t0 = time.perf_counter()
        npt = 0
        while npt < 8 or time.perf_counter() - t0 < 0.7 * seconds:
            x, y = int(self.rng.integers(w.nx)), int(self.rng.integers(w.ny))
            dYl, dl, rl, _ = oletkf.point_inputs(x, y, self.Yf, self.yo, self.net, self.var,
                                                 w.nx, w.ny, w.loc_radius, self.c2,
                                                 oobs.VAR_U | oobs.VAR_V, ybar=self.ybar,
                                                 dY=self.dY)
            oletkf.local_analysis(self.f[:, :, y % sy, x % sx].T, dYl, dl, rl)
            npt += 1
        t_pt = (time.perf_counter() - t0) / npt
        t_cycle = w.steps_per_cycle * t_lbm + t_obs + w.n_points * t_pt
        return {"value": w.n_points / t_cycle, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": (f"{nl} D2Q9 step(s) and the moments of the {w.k} members on a "
                           f"{sx}x{sy} periodic sub-block (x{self.scale:g} nodes to the "
                           f"{w.nx}x{w.ny} grid) and {npt} local analyses at random points of "
                           f"the {w.n_points} (FP64 NumPy, one thread), extrapolated to one "
                           f"cycle of {w.steps_per_cycle} steps + {w.n_points} analyses"),
                "lbm_mlups_per_member": w.n_points / t_lbm / 1e6,
                "seconds_per_cycle": t_cycle}


def oracle_sample(wname: str, seconds: float) -> dict:
    return OracleSample(wname).step(seconds)


def oracle_steps(wname: str, steps: int, warmup: int, seconds: float) -> dict:
    """The reference arm's steps in one process: the set-up once, then warmup + steps bounded
    samples of one cycle each."""
    s = OracleSample(wname)
    for _ in range(warmup):
        s.step(seconds)
    runs = [s.step(seconds) for _ in range(steps)]
    return {"seconds_per_cycle": [r["seconds_per_cycle"] for r in runs],
            "sample": runs[-1]["sample"]}


def _oracle_env():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    for key in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(key, None)
    return env


def _run_self(extra, timeout=900):
    r = subprocess.run([sys.executable, os.path.abspath(__file__), *extra], capture_output=True,
                       text=True, env=_oracle_env(), timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(f"oracle subprocess {extra[:2]} failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_subprocess(wname: str, seconds: float) -> dict:
    return _run_self(["--_oracle-sample", "--workload", wname, "--cpu-sample-seconds",
                      str(seconds)])


def run_oracle_all_cores(wname: str, seconds: float) -> dict:
    """The oracle on every host core at once: one single-threaded sample process per core
    (grid points are independent), the aggregate rate their sum.  The process count is
    capped so that the samples' FP64 arrays take at most half the host memory."""
    import concurrent.futures as cf

    import synth
    w = synth.WORKLOADS[wname]
    cores = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError, AttributeError):
        mem = 0
    sub = min(w.nx, SUB_EDGE) * min(w.ny, SUB_EDGE)
    # the sub-block ensemble and its D2Q9 temporaries, plus the full network's observations
    per_proc = 6 * 8 * 9 * w.k * sub + 4 * 8 * 9 * w.k * len(w.obs_network())
    n = cores if mem <= 0 else max(1, min(cores, int(0.5 * mem // per_proc)))
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        runs = list(ex.map(lambda _: run_oracle_subprocess(wname, seconds), range(n)))
    return {"value": sum(r["value"] for r in runs), "unit": UNIT, "cores": n,
            "kind": "oracle", "host_cores": cores,
            "sample": f"{n} concurrent single-threaded samples, each: " + runs[0]["sample"]}


def reference_main(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wname = args.workload
    steps = args.steps if args.steps is not None else 3
    per = max(1.0, min(args.cpu_sample_seconds, 150.0 / max(1, steps + args.warmup)))
    r = _run_self(["--_oracle-steps", "--workload", wname, "--steps", str(steps), "--warmup",
                   str(args.warmup), "--cpu-sample-seconds", str(per)], timeout=1800)
    secs = r["seconds_per_cycle"]
    import synth
    w = synth.WORKLOADS[wname]
    value = w.n_points * steps / sum(secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": (f"each step a bounded sample of about {per:g} s, "
                                        "extrapolated to one cycle (ms_per_step is that "
                                        "extrapolated cycle time, not wall time): " +
                                        r["sample"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- error vs oracle

ERR_POINTS = 32


def oracle_error_prep(wname: str, outdir: str, npoints: int = ERR_POINTS) -> dict:
    """Oracle side of the error measurement (CPU subprocess).  Writes to outdir:
      f0.npy      FP32 [k, 9, ny, nx] forecast ensemble: the oracle's equilibria of a seeded
                  band-limited flow (RMS 0.05, wavenumbers 2-6) plus N(0, member_sigma^2)
                  velocity perturbations per member and node; the GPU's input
      yo.npy      FP32 [L*V] observations: the flow's (u, v) at the observation points plus
                  N(0, obs_sigma^2)
      points.npy  [n, 2] sampled grid points (the four corners, the centre, seeded others)
      ref.npy     [n, k, 9] the oracle's analysis blocks there (Algorithm 1 per point, FP64,
                  as deviations f - w from rest)
      xf.npy      [n, k, 9] the forecast blocks there (f0 - w, FP64)
      nloc.npy    [n] local observation points"""
    import numpy as np

    import synth
    from oracle import lbm, obs as oobs, letkf as oletkf
    w = synth.WORKLOADS[wname]
    k, nx, ny = w.k, w.nx, w.ny
    tx, ty = synth.band_limited_force(nx, ny, 2.0, 6.0, 0.05, w.seed + 71)
    f0 = np.lib.format.open_memmap(os.path.join(outdir, "f0.npy"), mode="w+", dtype=np.float32,
                                   shape=(k, 9, ny, nx))
    for m in range(k):
        ux = tx + synth.gaussian((ny, nx), w.member_sigma, w.seed + 100 + 2 * m)
        uy = ty + synth.gaussian((ny, nx), w.member_sigma, w.seed + 101 + 2 * m)
        f0[m] = lbm.equilibrium(np.ones((ny, nx)), ux, uy)
    f0.flush()
    net = w.obs_network()
    L = len(net)
    xs, ys = net[:, 0], net[:, 1]
    strip_xy = np.stack([np.arange(L), np.zeros(L, dtype=np.int64)], axis=1)
    truth = lbm.equilibrium(np.ones((1, L)), tx[ys, xs][None], ty[ys, xs][None])
    uv = oobs.VAR_U | oobs.VAR_V
    yo = (oobs.observe(truth, strip_xy, uv) + synth.gaussian(2 * L, w.obs_sigma, w.seed + 72))
    yo = yo.astype(np.float32)
    np.save(os.path.join(outdir, "yo.npy"), yo)
    Yf = oobs.observe(np.asarray(f0[:, :, ys, xs], np.float64)[:, :, None, :], strip_xy, uv)
    ybar, dY = oobs.ensemble_obs(Yf)
    var = w.obs_error_var(2 * L)
    c2 = synth.loc_cutoff2(w.loc_radius)
    rng = synth.generator(w.seed + 73)
    pts = {(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, ny // 2)}
    while len(pts) < npoints:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny))))
    pts = sorted(pts)
    ref, xf, nloc = [], [], []
    for (x, y) in pts:
        dYl, dl, rl, n = oletkf.point_inputs(x, y, Yf, yo.astype(np.float64), net, var, nx, ny,
                                             w.loc_radius, c2, uv, ybar=ybar, dY=dY)
        xb = np.asarray(f0[:, :, y, x], np.float64)          # [k, 9]
        res = oletkf.local_analysis(xb.T, dYl, dl, rl)
        ref.append(res["Xa"].T - lbm.W[None, :])
        xf.append(xb - lbm.W[None, :])
        nloc.append(n)
    np.save(os.path.join(outdir, "points.npy"), np.asarray(pts, dtype=np.int64))
    np.save(os.path.join(outdir, "ref.npy"), np.stack(ref))
    np.save(os.path.join(outdir, "xf.npy"), np.stack(xf))
    np.save(os.path.join(outdir, "nloc.npy"), np.asarray(nloc, dtype=np.int64))
    return {"points": len(pts), "mean_local_obs": float(np.mean(nloc))}


def block_errors(got, ref, xf):
    """Relative L2 errors of analysis blocks [n, k, 9] against the reference: the ensemble mean
    (over all sampled points and populations), the mean increment (mean - forecast mean), the
    perturbations about the mean; and the worst single point of each."""
    import numpy as np

    def rel(a, b):
        d = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))

    got, ref, xf = (np.asarray(a, np.float64) for a in (got, ref, xf))
    mg, mo, mf = got.mean(1), ref.mean(1), xf.mean(1)         # [n, 9]
    out = {"mean": rel(mg, mo), "increment": rel(mg - mf, mo - mf),
           "perturbations": rel(got - mg[:, None], ref - mo[:, None])}
    worst = [0.0, 0.0, 0.0]
    for i in range(got.shape[0]):
        e = (rel(mg[i], mo[i]), rel(mg[i] - mf[i], mo[i] - mf[i]),
             rel(got[i] - mg[i], ref[i] - mo[i]))
        worst = [max(a, b) for a, b in zip(worst, e)]
    out.update({"worst_point_mean": worst[0], "worst_point_increment": worst[1],
                "worst_point_perturbations": worst[2]})
    return out


def workload_config(w, precision="fp32"):
    return {"workload": w.name, "grid": f"{w.nx}x{w.ny}", "k": w.k, "tau": w.tau,
            "obs_stride": w.obs_stride, "obs_vars": "u,v", "loc_radius": w.loc_radius,
            "loc": "gaussian, cutoff 2*sqrt(10/3)*r", "steps_per_cycle": w.steps_per_cycle,
            "precision": precision, "l2": "flushed between timed cycles (256 MiB write)",
            "parallelism": "independent replica per GPU"}


# ----------------------------------------------------------------------------- GPU leg

def main(argv=None):
    args = parse_args(argv)
    if args._oracle_sample:
        print(json.dumps(oracle_sample(args.workload, args.cpu_sample_seconds)))
        return 0
    if args._oracle_steps:
        print(json.dumps(oracle_steps(args.workload, args.steps, args.warmup,
                                      args.cpu_sample_seconds)))
        return 0
    if args._oracle_error_prep:
        print(json.dumps(oracle_error_prep(args.workload, args._oracle_error_prep)))
        return 0
    if args.impl == "reference":
        return reference_main(args)

    import numpy as np
    import torch

    import synth
    from paper_2308_03310_gb300 import _build, letkf as L

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
    dist_init("nccl" if world > 1 else "gloo")
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)
    if rank == 0:
        _build.build()
    barrier()
    L.load()

    if args.workload == "serve_cfg5":
        return serve_main(args, device, rank, world)
    if args.workload == "group_cfg4":
        return group_main(args, device, rank, world)
    if args.workload == "group_small":
        return group_small_main(args, device, rank, world)
    if args.workload == "evd_table1":
        return evd_main(args, device, rank, world)
    if args.workload in ("paper_dense", "paper_sparse"):
        return paper_main(args, device, rank, world)
    w = synth.WORKLOADS[args.workload]
    steps = args.steps if args.steps is not None else DEFAULT_STEPS.get(args.workload, 20)
    warm = max(3, args.warmup)
    spin, members, setup, truth = spin_up(w, device)
    yos = nature_observations(spin, w, warm + 2 * steps, seed_offset=1000 * rank)
    spin.close()
    forms = {"fp32": [L.LETKF_FP32], "mixed": [L.LETKF_MIXED],
             "both": [L.LETKF_FP32, L.LETKF_MIXED]}[args.precision]
    sched = EIG_SCHEDULES[args.eig_schedule]
    chunk = int(args.chunk_mb * (1 << 20))
    peak32 = measure_fp32_peak(device)
    results = [measure(w, members, setup, yos, device, prec, steps, warm, world, sched, chunk,
                       peak32) for prec in forms]
    head = results[0]
    ncyc = 20
    rmse = {"cycles": ncyc, "averaged_over": f"cycles {ncyc // 2}..{ncyc - 1}",
            "unit": "lattice velocity", "field": "(u, v) of the ensemble mean vs the truth, all "
                                                   "grid points"}
    for prec in forms:
        rmse["mixed" if prec == L.LETKF_MIXED else "fp32"] = rmse_run(
            w, members, truth, setup, device, prec, ncyc, seed_offset=1000 * rank)
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, head["precision"]),
        "p50_cycle_ms": head["p50_cycle_ms"], "p99_cycle_ms": head["p99_cycle_ms"],
        "roofline": head["roofline"], "kernels": head["kernels"], "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"], "eig_schedule": head["eig_schedule"],
        "gram_tile": head["gram_tile"],
        "chunks_per_analysis": head["chunks_per_analysis"],
        "lbm": head["lbm"],
        "clocks": head["clocks"],
        "local_obs": head["local_obs"],
        **({"chebyshev_per_cycle": head["chebyshev_per_cycle"]}
           if "chebyshev_per_cycle" in head else {}),
        "rmse_vs_truth": rmse,
        "mixed": None,
    }
    if len(results) > 1:
        mx = results[1]
        line["mixed"] = {k: mx[k] for k in ("precision", "value", "ms_per_step", "p50_cycle_ms",
                                             "p99_cycle_ms", "e2e", "gpu_launches", "eig_schedule",
                                             "gram_tile", "clocks")}
        line["mixed"]["kernels"] = {n: {"ms_per_cycle": d["ms_per_cycle"], "frac": d["frac"],
                                         "unit": d["unit"]} for n, d in mx["kernels"].items()}
        line["mixed"]["speedup_vs_fp32"] = mx["value"] / head["value"]
    line["fp32_peak"] = peak32
    if rank == 0 and world == 1 and not args.no_error_check:
        # outside the timed region: one analysis of each form on a seeded synthetic ensemble
        # of the workload's shape, compared with the FP64 oracle at sampled grid points
        try:
            err = measure_error(w, setup, device, forms, sched, chunk)
        except Exception as e:  # the timing stands; say why the error is missing
            err = {"error": str(e)[-300:]}
        line["error_vs_oracle"] = err
        if line["mixed"] is not None:
            line["mixed"]["error"] = err.get("mixed", err.get("error"))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = run_oracle_subprocess(args.workload, args.cpu_sample_seconds)
            line["cpu_baseline"].pop("seconds_per_cycle", None)
        except Exception as e:  # the GPU number stands; say why the baseline is missing
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "kind": "oracle",
                                    "error": str(e)[-300:]}
        try:
            line["cpu_baseline_all_cores"] = run_oracle_all_cores(args.workload,
                                                                  args.cpu_sample_seconds)
        except Exception as e:
            line["cpu_baseline_all_cores"] = {"value": None, "unit": UNIT, "kind": "oracle",
                                              "error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line))
    return 0


# Table 1 of the paper (A100, ms per batch of 128^2 matrices), context for evd_table1
PAPER_TABLE1_MS = {16: (0.7, 1.3), 32: (4.1, 2.4), 48: (922.8, 7.8), 64: (927.4, 14.2)}


def evd_main(args, device, rank, world):
    """Batched symmetric EVD at the shapes of the paper's Table 1: a batch of 128^2 matrices
    Q = (k-1) I + Yb^T R^-1 Yb from the LETKF of a 128 x 128 ensemble (k = 16, 32, 48, 64;
    (u, v) observed every 4th point, sigma 0.01, r = 3; members = a band-limited flow + N(0,
    0.005^2) velocity perturbations after 50 steps), eigenvalues and eigenvectors in FP32.
    Timed: letkf_eigh_batch (one warp per matrix), letkf_eigh_batch_ws (split schedule) and,
    as a library comparator only (not product code), torch.linalg.eigh on the same device.
    The paper's A100 numbers (cuSOLVER syevjBatched, EigenG) are printed beside them."""
    import numpy as np
    import torch

    import synth
    from paper_2308_03310_gb300 import letkf as L

    n = 128
    reps = args.steps if args.steps is not None else 5
    warm = max(3, args.warmup)
    rows = []
    for k in (16, 32, 48, 64):
        net = synth.regular_obs_network(n, n, 4)
        var = np.full(len(net) * 2, 1e-4, dtype=np.float32)
        e = L.Experiment(n, n, k, 0.6, net, var, loc_radius=3.0, device=device)
        tx, ty = synth.band_limited_force(n, n, 2.0, 5.0, 0.02, 51)
        ux = (tx[None] + synth.gaussian((k, n, n), 0.005, 52)).astype(np.float32)
        uy = (ty[None] + synth.gaussian((k, n, n), 0.005, 53)).astype(np.float32)
        e.set_macro(np.ones((k, n, n), np.float32), ux, uy)
        e.forecast(50)
        yo = (e.get_obs()[:k].mean(0) + synth.gaussian(len(net) * 2, 0.01, 54)).astype(np.float32)
        A = e.analyze_probe(yo, np.arange(n * n), want=("gram",))["gram"].astype(np.float64)
        assert e.sync() == 0
        e.close()
        up = np.triu(A)
        Q = (up + np.transpose(np.triu(A, 1), (0, 2, 1)) + (k - 1) * np.eye(k)).astype(np.float32)
        npts = Q.shape[0]
        q = torch.from_numpy(Q).to(device)
        lam = torch.empty((npts, k), dtype=torch.float32, device=device)
        vec = torch.empty((npts, k, k), dtype=torch.float32, device=device)
        nb = L.letkf_eigh_workspace_bytes(npts, k)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device=device)
        wbase = (ws.data_ptr() + 255) // 256 * 256
        stream = torch.cuda.current_stream(device).cuda_stream

        def fused():
            return L.letkf_eigh_batch(npts, k, q.data_ptr(), lam.data_ptr(), vec.data_ptr(), 0,
                                      stream)

        def split():
            return L.letkf_eigh_batch_ws(npts, k, q.data_ptr(), lam.data_ptr(), vec.data_ptr(),
                                         0, wbase, nb, stream)

        def timed(fn, slow_s=1.0):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize(device)
            once = time.perf_counter() - t0
            for _ in range(warm - 1 if once < slow_s else 0):
                fn()
            torch.cuda.synchronize(device)
            out = []
            for _ in range(reps if once < slow_s else 1):  # a call over a second: timed once
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                rc = fn()
                b.record()
                torch.cuda.synchronize(device)
                if isinstance(rc, int) and rc != 0:
                    raise RuntimeError(f"eigensolver failed: {L.strerror(rc)}")
                out.append(a.elapsed_time(b))
            return min(out), statistics.median(out)

        t_fused = timed(fused)
        lam_f = np.sort(lam.cpu().numpy().astype(np.float64), axis=1)
        t_split = timed(split)
        lam_s = np.sort(lam.cpu().numpy().astype(np.float64), axis=1)
        # our solvers leave Householder vectors in the strictly lower triangle of q: the
        # comparator gets its own copy of the symmetric matrices
        qt = torch.from_numpy(Q).to(device)
        t_torch = timed(lambda: torch.linalg.eigh(qt))
        lam_t = torch.linalg.eigh(qt)[0].double().cpu().numpy()
        scale = np.abs(lam_t).max()
        pc, pe = PAPER_TABLE1_MS[k]
        rows.append({"k": k, "batch": npts,
                     "ours_split_ms": t_split[1], "ours_fused_ms": t_fused[1],
                     "torch_linalg_eigh_ms": t_torch[1],
                     "max_eigenvalue_diff_vs_torch": float(max(np.abs(lam_f - lam_t).max(),
                                                               np.abs(lam_s - lam_t).max())
                                                           / scale),
                     "paper_a100_cusolver_syevj_batched_ms": pc, "paper_a100_eigeng_ms": pe})
        del q, qt, lam, vec, ws
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"metric": "batched symmetric EVD time per batch of 128^2 matrices "
                                    "(eigenvalues and eigenvectors, FP32)",
                          "unit": "ms", "higher_is_better": False, "n_gpus": world,
                          "data": "synthetic", "config": {"workload": "evd_table1",
                                                          "batch": n * n, "k": [16, 32, 48, 64]},
                          "comparator": "torch.linalg.eigh: library, context only",
                          "paper_hardware": "A100 40 GB (context, not a target)",
                          "results": rows}))
    return 0


# The paper's LETKF time per cycle at M = 64 on one A100 for its naive parallelization (case A,
# every GPU analyses every grid point): 39.5 ms (dense), and the total cycle times 73.0 ms
# (sparse, case A) and 19.2 ms (sparse, case C on 64 GPUs).  Context, not targets.
PAPER_DENSE_LETKF_MS_M64 = 39.5
PAPER_SPARSE_CYCLE_MS_M64 = {"case_A": 73.0, "case_C": 19.2}


def paper_main(args, device, rank, world):
    """The paper's own workloads (Sec. V): a 128 x 128 D2Q9 turbulence (tau 0.52, the
    Kolmogorov plus band-limited forcing of the 256^2 workload, 5,000-step spin-up of the truth
    and of every member from perturbed copies of it), rho, u and v observed (V = 3) with 20 %
    noise per variable, 100 steps per cycle, ensembles of M = 4, 16 and 64.
      paper_dense   every grid point observed, only its own observation local (l_max = 1)
      paper_sparse  every 4th point observed (L = 32^2), Gaspari-Cohn with cutoff 6 cells
    Timed: graph-captured cycles of each form, and the analysis alone (obs operator,
    transposes, Gram, eigensolve/transform/update) from the cycle's phase events."""
    import numpy as np
    import torch

    import synth
    from paper_2308_03310_gb300 import letkf as L

    n = 128
    dense = args.workload == "paper_dense"
    steps = args.steps if args.steps is not None else 20
    warm = max(3, args.warmup)
    kol = synth.kolmogorov_force(n, n, 1e-5, 4)
    rnd = synth.band_limited_force(n, n, 4.0, 6.0, 1e-5, 20230804)
    force = np.stack([kol[0] + rnd[0], kol[1] + rnd[1]]).astype(np.float32)
    net = synth.regular_obs_network(n, n, 1 if dense else 4)
    ruv = L.LETKF_OBS_RHO | L.LETKF_OBS_U | L.LETKF_OBS_V
    if dense:
        loc = dict(loc_radius=1.0, loc_cutoff2=1.0, loc_kind=L.LETKF_LOC_GAUSS)
    else:
        loc = dict(loc_radius=3.0 / math.sqrt(10.0 / 3.0), loc_cutoff2=36.0,
                   loc_kind=L.LETKF_LOC_GC)
    rows = []
    for k in (4, 16, 64):
        # nature run and members spun up together (the truth is the auxiliary member)
        spin = L.Experiment(n, n, k, 0.52, net, np.ones(len(net) * 3, np.float32),
                            obs_vars=ruv, n_aux=1, force=force, device=device, **loc)
        ux0 = synth.gaussian((n, n), 1e-3, 71)
        uy0 = synth.gaussian((n, n), 1e-3, 72)
        ux = np.concatenate([ux0[None] + synth.gaussian((k, n, n), 5e-3, 73), ux0[None]])
        uy = np.concatenate([uy0[None] + synth.gaussian((k, n, n), 5e-3, 74), uy0[None]])
        spin.set_macro(np.ones((k + 1, n, n), np.float32), ux.astype(np.float32),
                       uy.astype(np.float32))
        spin.forecast(5000)
        y0 = spin.get_obs()[k]
        sig = 0.2 * np.array([np.std(y0[0::3] - 1.0), np.std(y0[1::3]), np.std(y0[2::3])])
        var = np.tile(sig ** 2, len(net)).astype(np.float32)
        yos = []
        for c in range(warm + steps):
            spin.forecast(100)
            y = spin.get_obs()[k]
            yos.append(torch.from_numpy((y + np.tile(sig, len(net)) * synth.gaussian(
                y.shape, 1.0, 9000 + c)).astype(np.float32)).to(device))
        members = torch.empty((k, 9, n, n), dtype=torch.float32, device=device)
        L.letkf_get_deviation(spin.h, members.data_ptr(), 0, k, L.LETKF_DEVICE)
        torch.cuda.synchronize(device)
        spin.close()
        row = {"M": k}
        for name, prec in (("fp32", L.LETKF_FP32), ("mixed", L.LETKF_MIXED)):
            exp = L.Experiment(n, n, k, 0.52, net, var, obs_vars=ruv, force=force,
                               precision=prec, device=device, **loc)
            L.letkf_set_deviation(exp.h, members.data_ptr(), 0, k, L.LETKF_DEVICE)
            exp.enable_timing(True)
            for c in range(warm):
                exp.cycle(100, yos[c])
            torch.cuda.synchronize(device)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            ana = []
            for c in range(steps):
                ev[c][0].record(exp.stream)
                exp.cycle(100, yos[warm + c])
                ev[c][1].record(exp.stream)
                t = exp.timings()                 # waits for this cycle's phase events
                ana.append(t["obs_ms"] + t["transpose_in_ms"] + t["gram_ms"] + t["eigen_ms"] +
                           t["transpose_out_ms"])
            torch.cuda.synchronize(device)
            cyc = [a.elapsed_time(b) for a, b in ev]
            rc = exp.sync()
            if rc:
                raise RuntimeError(f"{args.workload} M={k} {name}: {L.strerror(rc)}")
            st = exp.stats()
            row[name] = {"analyses_per_s": n * n * steps / (sum(cyc) / 1e3),
                         "ms_per_cycle": statistics.mean(cyc),
                         "analysis_ms_per_cycle": statistics.mean(ana),
                         "eig_schedule": EIG_NAMES.get(st.eig_schedule, str(st.eig_schedule))}
            exp.close()
        row["max_local_obs"] = st.max_local_obs
        rows.append(row)
        del members, yos
        torch.cuda.empty_cache()
    head = rows[-1]["fp32"]
    line = {"metric": METRIC, "value": reduce_sum(head["analyses_per_s"], device), "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": head["ms_per_cycle"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "grid": "128x128", "M": [4, 16, 64],
                       "obs": "every point, l_max = 1" if dense else
                              "every 4th point, Gaspari-Cohn cutoff 6",
                       "obs_vars": "rho,u,v", "obs_noise": "20 % of each variable's RMS",
                       "steps_per_cycle": 100, "value_at": "M = 64, FP32",
                       "parallelism": "independent replica per GPU"},
            "results": rows,
            "paper_a100_context": ({"letkf_ms_per_cycle_M64_case_A": PAPER_DENSE_LETKF_MS_M64}
                                   if dense else
                                   {"cycle_ms_M64": PAPER_SPARSE_CYCLE_MS_M64})}
    if rank == 0:
        print(json.dumps(line))
    return 0


def group_main(args, device, rank, world):
    """Uneven batching: four co-resident ensembles (k = 16, 32, 64, 128) on a 512 x 512 grid with
    a clustered observation network (every 2nd point over a quarter of the domain, every 16th
    point elsewhere, a band of rows without observations so that ~20 % of the points have no
    local observation; r = 4).  Timed: graph-captured grouped cycles (forecast of all four +
    one grouped analysis) against the same four ensembles cycled one after another with their
    own letkf_cycle.  value = grid-point analyses per second over the four ensembles."""
    import numpy as np
    import torch

    import synth
    from paper_2308_03310_gb300 import letkf as L

    nx = ny = 512
    ks = (16, 32, 64, 128)
    r = 4.0
    cut = float(np.sqrt(synth.loc_cutoff2(r)))
    band = int(0.2 * ny + 2 * cut + 1)
    net = synth.clustered_obs_network(nx, ny, 2, 16, patch=(0, 0, nx // 2, ny // 2),
                                      empty_band=(ny // 2 + 64, band))
    LV = len(net) * 2
    sigma = 0.01
    var = np.full(LV, sigma * sigma, dtype=np.float32)
    steps_cycle = 25
    steps = args.steps if args.steps is not None else 10
    warm = max(3, args.warmup)
    tx, ty = synth.band_limited_force(nx, ny, 2.0, 5.0, 0.02, 41)
    out = {}
    for name, prec in (("fp32", L.LETKF_FP32), ("mixed", L.LETKF_MIXED)):
        exps, yos = [], []
        for i, k in enumerate(ks):
            e = L.Experiment(nx, ny, k, 0.55, net, var, loc_radius=r, precision=prec,
                             device=device)
            ux = np.empty((k, ny, nx), np.float32)
            uy = np.empty((k, ny, nx), np.float32)
            for m in range(k):
                px, py = synth.band_limited_force(nx, ny, 2.0, 5.0, 0.005, 1000 * i + m)
                ux[m], uy[m] = tx + px, ty + py
            e.set_macro(np.ones((k, ny, nx), np.float32), ux, uy)
            exps.append(e)
        st = exps[0].stats()
        # observations: the truth field observed with noise, one draw per cycle
        truth_u = np.stack([tx, ty])
        xs, ys = net[:, 0], net[:, 1]
        ytrue = np.stack([truth_u[0][ys, xs], truth_u[1][ys, xs]], axis=1).reshape(-1)
        obs = [torch.from_numpy((ytrue + synth.gaussian(LV, sigma, 77 + c)).astype(np.float32))
               .to(device) for c in range(warm + steps)]
        stream = exps[0].stream

        def timed(run_cycle):
            for c in range(warm):
                run_cycle(c)
            torch.cuda.synchronize(device)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            cyc = []
            for c in range(steps):
                ev[c].record(stream)
                run_cycle(warm + c)
                ev[c + 1].record(stream)
                torch.cuda.synchronize(device)
                cyc.append(ev[c].elapsed_time(ev[c + 1]))
            return cyc

        def group_cycle(c):
            L.letkf_group_cycle(exps, steps_cycle, [obs[c]] * len(exps))

        def separate_cycles(c):
            for e in exps:
                e.cycle(steps_cycle, obs[c])
            # the timing events sit on the first handle's stream: join the others
            for e in exps[1:]:
                done = torch.cuda.Event()
                done.record(e.stream)
                stream.wait_event(done)

        g = timed(group_cycle)
        picks = [EIG_NAMES.get(e.stats().eig_schedule, "auto") for e in exps]
        sep = timed(separate_cycles)
        for e in exps:
            rc = e.sync()
            if rc:
                raise RuntimeError(f"group cycle failed: {L.strerror(rc)}")
        pts = nx * ny * len(ks)
        out[name] = {
            "value": pts * len(g) / (sum(g) / 1e3),
            "ms_per_cycle": statistics.mean(g),
            "p50_cycle_ms": float(np.percentile(g, 50)),
            "p99_cycle_ms": float(np.percentile(g, 99)),
            "separate_value": pts * len(sep) / (sum(sep) / 1e3),
            "separate_ms_per_cycle": statistics.mean(sep),
            "zero_obs_fraction": st.n_zero_obs / st.n_points,
            "max_local_obs": st.max_local_obs, "mean_local_obs": st.mean_local_obs,
            "eig_schedules": dict(zip((str(k) for k in ks), picks)),
        }
        for e in exps:
            e.close()
        del exps, obs
        torch.cuda.empty_cache()
    head = out["fp32"]
    line = {
        "metric": METRIC, "value": reduce_sum(head["value"], device), "unit": UNIT,
        "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": head["ms_per_cycle"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "group_cfg4", "grid": "512x512", "k": list(ks),
                   "network": "clustered: every 2nd point over 25 % of the domain, every 16th "
                              "elsewhere, an observation-free band", "loc_radius": r,
                   "steps_per_cycle": steps_cycle, "precision": "fp32",
                   "parallelism": "one grouped launch per column class for the fused-schedule ensembles, split kernels for the others"},
        "p50_cycle_ms": head["p50_cycle_ms"], "p99_cycle_ms": head["p99_cycle_ms"],
        "group": head, "mixed": dict(out["mixed"],
                                     speedup_vs_fp32=out["mixed"]["value"] / head["value"]),
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def group_small_main(args, device, rank, world):
    """Uneven batching where one launch has to carry the GPU: 16 co-resident ensembles on
    64 x 64 grids (4,096 points each: one ensemble alone fills a small part of the GPU), k
    cycling through 16, 24, 32, 40, 48, 56, 64 and 20, a clustered network (every 2nd point
    over a quarter of the domain, every 8th elsewhere, a band without observations, r = 2).
    Timed per form (graph-captured cycles of 25 steps):
      grouped_fused   one grouped cycle, every ensemble on the FUSED schedule: the
                      eigensolve of all 16 ensembles' points is one persistent launch per
                      column class (k <= 32, <= 64), warps taking points from a counter
      grouped_auto    one grouped cycle, each ensemble on the schedule AUTO picks for it
      separate_auto   the 16 ensembles cycled one after another on their own streams
    value = grid-point analyses per second of grouped_fused (FP32)."""
    import numpy as np
    import torch

    import synth
    from paper_2308_03310_gb300 import letkf as L

    nx = ny = 64
    ks = (16, 24, 32, 40, 48, 56, 64, 20) * 2
    r = 2.0
    net = synth.clustered_obs_network(nx, ny, 2, 8, patch=(4, 4, nx // 2, ny // 2),
                                      empty_band=(44, 12))
    LV = len(net) * 2
    sigma = 0.01
    var = np.full(LV, sigma * sigma, dtype=np.float32)
    steps_cycle = 25
    steps = args.steps if args.steps is not None else 20
    warm = max(3, args.warmup)
    tx, ty = synth.band_limited_force(nx, ny, 2.0, 5.0, 0.02, 61)
    xs, ys = net[:, 0], net[:, 1]
    ytrue = np.stack([tx[ys, xs], ty[ys, xs]], axis=1).reshape(-1)
    obs = [torch.from_numpy((ytrue + synth.gaussian(LV, sigma, 91 + c)).astype(np.float32))
           .to(device) for c in range(warm + steps)]

    def ensembles(prec, schedule):
        exps = []
        for i, k in enumerate(ks):
            e = L.Experiment(nx, ny, k, 0.55, net, var, loc_radius=r, precision=prec,
                             device=device, eig_schedule=schedule)
            px = synth.gaussian((k, ny, nx), 0.005, 3000 + 2 * i)
            py = synth.gaussian((k, ny, nx), 0.005, 3001 + 2 * i)
            e.set_macro(np.ones((k, ny, nx), np.float32), (tx[None] + px).astype(np.float32),
                        (ty[None] + py).astype(np.float32))
            exps.append(e)
        return exps

    def timed(exps, run_cycle):
        stream = exps[0].stream
        for c in range(warm):
            run_cycle(exps, c)
        torch.cuda.synchronize(device)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for c in range(steps):
            ev[c][0].record(stream)
            run_cycle(exps, warm + c)
            ev[c][1].record(stream)
        torch.cuda.synchronize(device)
        for e in exps:
            rc = e.sync()
            if rc:
                raise RuntimeError(f"group_small cycle failed: {L.strerror(rc)}")
        return [a.elapsed_time(b) for a, b in ev]

    def group_cycle(exps, c):
        L.letkf_group_cycle(exps, steps_cycle, [obs[c]] * len(exps))

    def separate_cycles(exps, c):
        for e in exps:
            e.cycle(steps_cycle, obs[c])
        stream = exps[0].stream
        for e in exps[1:]:
            done = torch.cuda.Event()
            done.record(e.stream)
            stream.wait_event(done)

    pts = nx * ny * len(ks)
    out = {}
    for name, prec in (("fp32", L.LETKF_FP32), ("mixed", L.LETKF_MIXED)):
        res = {}
        for variant, sched, runner in (("grouped_fused", L.LETKF_EIG_FUSED, group_cycle),
                                       ("grouped_auto", L.LETKF_EIG_AUTO, group_cycle),
                                       ("separate_auto", L.LETKF_EIG_AUTO, separate_cycles)):
            exps = ensembles(prec, sched)
            cyc = timed(exps, runner)
            res[variant] = {"analyses_per_s": pts * len(cyc) / (sum(cyc) / 1e3),
                            "ms_per_cycle": statistics.mean(cyc),
                            "p99_cycle_ms": float(np.percentile(cyc, 99)),
                            "schedules": sorted({EIG_NAMES.get(e.stats().eig_schedule, "auto")
                                                 for e in exps})}
            st = exps[0].stats()
            for e in exps:
                e.close()
            del exps
            torch.cuda.empty_cache()
        res["zero_obs_fraction"] = st.n_zero_obs / st.n_points
        res["max_local_obs"] = st.max_local_obs
        res["grouped_fused_vs_separate"] = (res["grouped_fused"]["analyses_per_s"] /
                                            res["separate_auto"]["analyses_per_s"])
        out[name] = res
    head = out["fp32"]["grouped_fused"]
    line = {"metric": METRIC, "value": reduce_sum(head["analyses_per_s"], device), "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": head["ms_per_cycle"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "group_small", "grid": "64x64", "ensembles": len(ks),
                       "k": list(ks), "network": "clustered: every 2nd point over a quarter, "
                       "every 8th elsewhere, a band without observations", "loc_radius": r,
                       "steps_per_cycle": steps_cycle, "precision": "fp32",
                       "parallelism": "one grouped cycle of 16 ensembles"},
            "p99_cycle_ms": head["p99_cycle_ms"], "group": out}
    if rank == 0:
        print(json.dumps(line))
    return 0


def serve_main(args, device, rank, world):
    """The serving workload: a seeded Poisson stream of independent DA experiments (arrivals
    at 20/s; grids 128^2..1024^2, k 16..128, 10..100 cycles, (u, v) every 4th or 8th point),
    served with continuous batching under an HBM budget, in the FP32 and the mixed form.
    value = grid-point analyses per second of wall time (completed cycles only); p50/p99 of
    the per-cycle device latency.  With N ranks each rank serves its own stream (weak
    scaling) and value is the sum."""
    import torch

    import synth
    from paper_2308_03310_gb300 import letkf as L
    from paper_2308_03310_gb300.serve import (GpuSlot, Request, Server, gpu_footprint,
                                              stream_priority)

    free, _ = torch.cuda.mem_get_info(device)
    budget = int(min(args.serve_budget_gb * 1e9, 0.85 * free))
    base = synth.poisson_requests(args.serve_requests, 20.0, 20230803 + 7919 * rank)
    out = {}
    forms = [("fp32", L.LETKF_FP32, True), ("mixed", L.LETKF_MIXED, True)]
    if args.serve_compare_priority:
        forms.append(("fp32_one_priority", L.LETKF_FP32, False))
    for name, prec, prio in forms:
        # the eigensolve schedule is pinned by ensemble and grid size (what the autotuner
        # picks), so that no admission pays for timing it under load
        reqs = [Request(**d, steps_per_cycle=25, precision=prec,
                        eig_schedule=(L.LETKF_EIG_CHEBYSHEV if d["k"] <= 64
                                      else L.LETKF_EIG_SPLIT if d["nx"] * d["ny"] >= 16384
                                      else L.LETKF_EIG_FUSED)) for d in base]
        srv = Server(budget, (lambda r: GpuSlot(r, device, priority=stream_priority(r)))
                     if prio else (lambda r: GpuSlot(r, device)), gpu_footprint,
                     max_active=args.serve_max_active)
        torch.cuda.synchronize(device)
        barrier()
        rep = srv.run(reqs, time_limit_s=args.serve_seconds)
        torch.cuda.synchronize(device)
        total = reduce_sum(rep["analyses"], device)
        wall = reduce_max(rep["wall_s"], device)
        out[name] = {
            "value": total / wall, "wall_s": wall, "completed_requests": rep["completed"],
            "admitted_requests": sum(1 for e in rep["timeline"] if e[1] == "admit"),
            "cycles": rep["cycles"], "p50_cycle_ms": rep["latency_ms"]["p50"],
            "p99_cycle_ms": rep["latency_ms"]["p99"],
            "cycle_ms_by_class": rep["latency_ms"]["by_class"],
            "stream_priorities": "small cycles (<= 256^2 x 64 point-members) on the most urgent "
                                 "stream priority" if prio else "one priority for every slot",
            "admission_wait_s": rep["admission_wait_s"], "max_concurrent": rep["max_concurrent"],
            "peak_footprint_gb": rep["peak_footprint_bytes"] / 1e9,
            "unfinished_requests": rep["unfinished"], "errors": rep["errors"][:3],
        }
        del srv, rep
        torch.cuda.empty_cache()
    head = out["fp32"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
        "steps": head["cycles"], "warmup": 0,
        "ms_per_step": 1e3 * head["wall_s"] / max(1, head["cycles"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "serve_cfg5", "arrivals": "Poisson, 20 per s, seeded",
                   "requests": args.serve_requests, "grids": [128, 256, 512, 1024],
                   "k": [16, 32, 64, 128], "cycles": [10, 100], "obs_stride": [4, 8],
                   "steps_per_cycle": 25, "hbm_budget_gb": budget / 1e9,
                   "time_limit_s": args.serve_seconds, "max_active": args.serve_max_active,
                   "parallelism": "continuous batching of independent experiments per GPU"},
        "p50_cycle_ms": head["p50_cycle_ms"], "p99_cycle_ms": head["p99_cycle_ms"],
        "serving": head, "mixed": dict(out["mixed"],
                                       speedup_vs_fp32=out["mixed"]["value"] / head["value"]),
        **({"fp32_one_priority": out["fp32_one_priority"]}
           if "fp32_one_priority" in out else {}),
    }
    if rank == 0:
        print(json.dumps(line))
    return 0


def measure_fp32_peak(device, iters=8192, reps=100):
    """FP32 FMA peak of this GPU, measured by the library's microbenchmark kernel (independent
    FMA chains filling every SM), timed with CUDA events on the launching stream; the median
    over reps launches, clocks sampled while they run."""
    import torch

    from paper_2308_03310_gb300 import letkf as L
    blocks, threads = L.letkf_fp32_peak_grid()
    out = torch.empty(blocks * threads, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    for _ in range(3):
        L.letkf_fp32_peak_run(iters, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    with ClockSampler(device.index) as clk:
        for a, b in ev:
            a.record(stream)
            flops = L.letkf_fp32_peak_run(iters, out.data_ptr(), stream.cuda_stream)
            b.record(stream)
        torch.cuda.synchronize(device)
    rates = sorted(flops / (a.elapsed_time(b) * 1e-3) / 1e12 for a, b in ev)
    assert torch.isfinite(out).all()
    return {"tflops": statistics.median(rates), "best_tflops": rates[-1],
            "launch": f"{blocks} x {threads} threads, 16 FMA chains x {8 * iters} rounds each",
            "clocks": clk.summary()}


def measure_error(w, setup, device, forms, eig_schedule=0, chunk_bytes=0):
    """Error of each form against the FP64 oracle at the workload's full size: the oracle
    subprocess writes a seeded synthetic ensemble of the workload's shape, observations and
    its own local analyses at sampled grid points; here each form analyses that ensemble once
    (the same handle configuration as the timed cycles) and its analysis blocks at the sampled
    points are compared with the oracle's."""
    import numpy as np
    import torch

    from paper_2308_03310_gb300 import letkf as L
    net, var, kw = setup
    out = {}
    with tempfile.TemporaryDirectory(prefix="letkf_err_") as d:
        info = _run_self(["--_oracle-error-prep", d, "--workload", w.name], timeout=1800)
        f0 = np.load(os.path.join(d, "f0.npy"), mmap_mode="r")
        yo = np.load(os.path.join(d, "yo.npy"))
        pts = np.load(os.path.join(d, "points.npy"))
        ref = np.load(os.path.join(d, "ref.npy"))
        xf = np.load(os.path.join(d, "xf.npy"))
        xs = torch.as_tensor(pts[:, 0], device=device)
        ys = torch.as_tensor(pts[:, 1], device=device)
        for prec in forms:
            exp = L.Experiment(w.nx, w.ny, w.k, w.tau, net, var, device=device, precision=prec,
                               eig_schedule=eig_schedule, chunk_bytes=chunk_bytes, **kw)
            exp.set_state(f0)
            exp.analyze(yo)
            buf = torch.empty((w.k, 9, w.ny, w.nx), dtype=torch.float32, device=device)
            torch.cuda.synchronize(device)
            L.letkf_get_deviation(exp.h, buf.data_ptr(), 0, w.k, L.LETKF_DEVICE)
            torch.cuda.synchronize(device)
            rc = exp.sync()
            if rc:
                raise RuntimeError(f"error-check analysis failed: {L.strerror(rc)}")
            got = buf[:, :, ys, xs].permute(2, 0, 1).double().cpu().numpy()   # [n, k, 9]
            out["mixed" if prec == L.LETKF_MIXED else "fp32"] = block_errors(got, ref, xf)
            exp.close()
            del buf
            torch.cuda.empty_cache()
    out.update({"points": int(len(pts)), "mean_local_obs_at_points": info["mean_local_obs"],
                "bar": 1e-5, "reference": "FP64 oracle (oracle.letkf.local_analysis)",
                "unit": "relative L2 over the sampled points' 9 x k blocks, in f - w",
                "input": ("a seeded band-limited flow (RMS 0.05) + N(0, member_sigma^2) member "
                          "perturbations, equilibria by the oracle, FP32; the workload's "
                          "network, R and localization")})
    return out


def measure(w, members, setup, yos, device, precision, steps, warm, world, eig_schedule=0,
            chunk_bytes=0, peak32=None):
    """Time `steps` cycles of one precision form (device-resident inputs), then the same
    through the public API with host buffers."""
    import numpy as np
    import torch

    from paper_2308_03310_gb300 import letkf as L

    exp = make_experiment(w, members, setup, device, precision, eig_schedule, chunk_bytes)
    st = exp.stats()
    LV = exp.L * exp.V
    stream = exp.stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)
    yo_dev = [torch.from_numpy(y).to(device) for y in yos[:warm + steps]]
    torch.cuda.synchronize(device)

    exp.enable_timing(True)
    for i in range(warm):
        exp.cycle(w.steps_per_cycle, yo_dev[i])
    rc = exp.sync()
    if rc:
        raise RuntimeError(f"warm-up cycle failed: {L.strerror(rc)}")
    counts0 = exp.work_counts()

    # ---- timed region: device-resident inputs, L2 flushed between cycles
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    phase = []
    torch.cuda.synchronize(device)
    barrier()
    torch.cuda.nvtx.range_push("timed")          # lets a profiler skip the set-up launches
    with ClockSampler(device.index) as clk:
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                starts[i].record(stream)
            exp.cycle(w.steps_per_cycle, yo_dev[warm + i])
            ends[i].record(stream)
            phase.append(exp.timings())           # waits for this cycle's events
        torch.cuda.synchronize(device)
    torch.cuda.nvtx.range_pop()
    barrier()
    clocks = clk.summary()
    rc = exp.sync()
    if rc:
        raise RuntimeError(f"timed cycles failed: {L.strerror(rc)}")
    cyc_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_s = reduce_max(sum(cyc_ms) / 1e3, device)
    counts1 = exp.work_counts()
    cheb = {n: (counts1[n] - counts0[n]) / steps for n in counts0}   # per timed cycle
    value = whole_job_rate(w.n_points * steps, total_s, world)

    # ---- per-kernel device time and roofline (the same timed cycles)
    ms = {
        "lbm_step": statistics.mean(p["forecast_ms"] for p in phase),
        "obs_operator": statistics.mean(p["obs_ms"] for p in phase),
        "transpose_in": statistics.mean(p["transpose_in_ms"] for p in phase),
        "gram": statistics.mean(p["gram_ms"] for p in phase),
        "eigen_update": statistics.mean(p["eigen_ms"] for p in phase),
        "transpose_out": statistics.mean(p["transpose_out_ms"] for p in phase),
    }
    peaks = measured_peaks()
    if peak32:
        peaks["fp32_tflops"] = peak32["tflops"]
    sm_mhz = peaks["sm_max_mhz"] or 2070.0
    work = kernel_work(w, w.k, w.n_points, st.mean_local_obs, exp.V, exp.L, st.n_chunks,
                       w.steps_per_cycle, exp.stats().eig_schedule, cheb)
    tensor_gram = precision == L.LETKF_MIXED and 17 <= w.k <= 128
    table = roofline_table(work, ms, peaks, sm_mhz, tensor_gram)
    top = max(table, key=lambda n: table[n]["ms_per_cycle"])
    t = table[top]
    unit, amount, launches = work[top]
    roofline = {"kernel": top, "bound": t["bound"], "achieved": t["achieved"], "peak": t["peak"],
                "unit": t["unit"], "frac": t["frac"],
                "traffic": traffic_for(top, w.name),
                "peak_source": (f"{peaks['source']} ({PEAK_NAMES[t['bound']]})"
                                if t["bound"] != "alu" or not peak32 else
                                "measured in this run: FP32 FMA microbenchmark "
                                "(letkf_fp32_peak_run, median of 100 launches; "
                                f"{peak32['launch']})"),
                "algorithmic_per_launch": amount / launches,
                "algorithmic_unit": "GB" if unit == "GB" else "TFLOP",
                "ms_per_launch": t["ms_per_launch"]}

    # ---- end to end through the public API with host buffers
    pinned = [torch.from_numpy(y).pin_memory() for y in yos[warm + steps:warm + 2 * steps]]
    e2e_s = []
    torch.cuda.synchronize(device)
    barrier()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        exp.cycle(w.steps_per_cycle, pinned[i])
        ya = exp.get_obs()                          # analysis in observation space -> host
        e2e_s.append(time.perf_counter() - t0)
        assert np.isfinite(ya).all()
    barrier()
    e2e_total = reduce_max(sum(e2e_s), device)
    e2e_value = whole_job_rate(w.n_points * steps, e2e_total, world)
    rc = exp.sync()
    if rc:
        raise RuntimeError(f"end-to-end cycles failed: {L.strerror(rc)}")
    st_end = exp.stats()                           # schedule resolved at the first analysis
    cycle_kernels = st_end.cycle_kernels            # kernel nodes of the cycle's graph
    exp.close()
    del flush
    return {
        "precision": "mixed" if precision == L.LETKF_MIXED else "fp32",
        "value": value, "ms_per_step": 1e3 * total_s / steps,
        "p50_cycle_ms": statistics.median(cyc_ms),
        "p99_cycle_ms": float(np.percentile(cyc_ms, 99)),
        "roofline": roofline,
        "kernels": {n: {kk: (round(vv, 6) if isinstance(vv, float) else vv)
                        for kk, vv in d.items()} for n, d in table.items()},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": LV * 4,
                "d2h_bytes_per_step": exp.nmem * LV * 4},
        "gpu_launches": cycle_kernels * steps,
        "eig_schedule": EIG_NAMES.get(st_end.eig_schedule, str(st_end.eig_schedule)),
        "gram_tile": GRAM_NAMES.get(st_end.gram_tile, str(st_end.gram_tile)),
        "chunks_per_analysis": st_end.n_chunks,
        "lbm": lbm_rates(w, ms["lbm_step"], peaks),
        "clocks": clocks,
        "local_obs": {"mean": st.mean_local_obs, "max": st.max_local_obs,
                      "zero_fraction": st.n_zero_obs / st.n_points},
        **({"chebyshev_per_cycle": {**cheb, "mean_degree": (cheb["cheb_products"]
                                                            / max(cheb["cheb_points"], 1))}}
           if st_end.eig_schedule == L.LETKF_EIG_CHEBYSHEV else {}),
    }


if __name__ == "__main__":
    sys.exit(main())
