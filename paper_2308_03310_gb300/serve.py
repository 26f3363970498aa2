"""Serving: a continuous-batching loop over independent data-assimilation experiments.

Requests (grid, ensemble size k, observation network, number of cycles, precision) arrive
over time.  Each admitted request becomes a *slot*: a libletkf handle with its own CUDA stream
and its ensemble state resident in HBM for the request's life.  A request is admitted as soon
as it has arrived and its device footprint (the handle's workspace plus the slot's buffers)
fits into the HBM budget next to the running slots; it never waits for a batch to form.  Every
running slot keeps up to two cycles enqueued on its stream, so the work of all slots overlaps
on the device, and a finished slot frees its memory for the requests that are waiting.

One cycle of a slot (Sec. II-B, cycle steps 2-3, as an OSSE): the ensemble and the slot's
nature run (an auxiliary member) advance by the cycle's LBM steps; the nature run is observed
(h(x) at the observation points) and seeded N(0, sigma^2) noise is added on the device; the
ensemble assimilates the observations.  All of it is enqueued asynchronously on the slot's
stream; the host only polls completion events.

Latency policy: a request whose cycle is small (grid points x members at most SMALL_WORK) gets
a high-priority CUDA stream, the others the default priority, so that the device schedules the
pending blocks of small cycles ahead of those of large ones: a 128^2, k = 16 cycle does not
queue behind the blocks of a 1024^2, k = 128 analysis.  Priorities change the order in which
blocks start, never the arithmetic.

Reported: throughput (grid-point analyses per second of wall time), per-cycle latency (device
time from a cycle's start to its end on its stream, which includes waiting for the other
slots' work) p50 / p99, overall and per size class, queueing delay of admissions, peak
footprint and concurrency.

A request's results depend only on its own inputs and seed: alone or in a mix, the same
arithmetic runs on its stream (the eigensolve schedule that AUTO picks is fixed per process
for a given k and chunk size).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import letkf as L

__all__ = ["Request", "Server", "GpuSlot", "percentile", "size_class", "stream_priority",
           "SMALL_WORK"]

# grid points x members of the largest "small" cycle (256^2 x 64)
SMALL_WORK = 256 * 256 * 64


@dataclasses.dataclass
class Request:
    """One DA experiment to serve."""
    rid: int
    arrival_s: float           # arrival time, seconds after the server starts
    nx: int
    ny: int
    k: int
    obs_stride: int            # (u, v) observed every obs_stride-th point in x and y
    cycles: int
    steps_per_cycle: int = 25
    loc_radius: float = 4.0
    tau: float = 0.55
    obs_sigma: float = 1e-3
    u_rms: float = 0.02        # RMS of the truth's initial velocity
    pert_rms: float = 0.005    # RMS of the members' initial perturbations
    precision: int = L.LETKF_FP32
    eig_schedule: int = L.LETKF_EIG_AUTO
    seed: int = 0

    @property
    def n_points(self) -> int:
        return self.nx * self.ny


def size_class(req) -> str:
    """'small' for a cycle of at most SMALL_WORK grid points x members, else 'large'."""
    return "small" if req.nx * req.ny * req.k <= SMALL_WORK else "large"


def stream_priority(req) -> int:
    """CUDA stream priority of a request's slot (lower is more urgent): the most urgent for
    small cycles, the default for large ones.  Out-of-range values map to the device's range."""
    return -8 if size_class(req) == "small" else 0


def percentile(values, q):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, q))


class GpuSlot:
    """A running request: handle, stream, resident state, observation buffers, events."""

    def __init__(self, req: Request, device, keep_state=False, priority=None):
        import torch
        self.torch = torch
        self.req = req
        self.device = torch.device(device)
        stream = None
        if priority is not None:
            stream = torch.cuda.Stream(device=self.device, priority=int(priority))
        nx, ny, k = req.nx, req.ny, req.k
        xs = np.arange(0, nx, req.obs_stride, dtype=np.int32)
        ys = np.arange(0, ny, req.obs_stride, dtype=np.int32)
        gy, gx = np.meshgrid(ys, xs, indexing="ij")
        net = np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.int32)
        self.LV = len(net) * 2
        var = np.full(self.LV, req.obs_sigma ** 2, dtype=np.float32)
        self.exp = L.Experiment(nx, ny, k, req.tau, net, var, n_aux=1,
                                loc_radius=req.loc_radius, precision=req.precision,
                                eig_schedule=req.eig_schedule, device=self.device,
                                stream=stream)
        self.stream = self.exp.stream
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(int(req.seed))
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            self.yf = torch.empty((k + 1, self.LV), dtype=torch.float32, device=self.device)
            self.yo = torch.empty(self.LV, dtype=torch.float32, device=self.device)
            rho, ux, uy = self._initial_fields()
            L.letkf_set_macro(self.exp.h, rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), 0,
                              k + 1, L.LETKF_DEVICE)
        self.footprint = self.exp.workspace_bytes + 4 * ((k + 2) * self.LV + 3 * (k + 1) * nx * ny)
        self.keep_state = keep_state
        self.enqueued = 0
        self.finished = 0
        self.inflight = []              # (start, end) events, oldest first
        self.latencies_ms = []
        self.state = None

    def _initial_fields(self):
        """Truth: a smooth random velocity field (a few Fourier modes); members: truth plus
        smooth random perturbations.  Drawn on the device from the request's generator."""
        torch, r = self.torch, self.req
        nx, ny, k = r.nx, r.ny, r.k
        x = torch.arange(nx, device=self.device, dtype=torch.float32)[None, :]
        y = torch.arange(ny, device=self.device, dtype=torch.float32)[:, None]

        def field(rms, n_fields):
            out = torch.zeros((n_fields, 2, ny, nx), device=self.device)
            for a in range(1, 4):
                for b in range(-3, 4):
                    ph = 2 * np.pi * torch.rand((n_fields, 1, 1), generator=self.gen,
                                                device=self.device)
                    amp = torch.randn((n_fields, 1, 1), generator=self.gen, device=self.device)
                    arg = 2 * np.pi * (a * x / nx + b * y / ny) + ph
                    s = amp * torch.sin(arg)
                    out[:, 0] += -(2 * np.pi * b / ny) * s      # divergence-free: (d psi/dy,
                    out[:, 1] += (2 * np.pi * a / nx) * s       #  -d psi/dx) of psi = cos(arg)
            norm = out.pow(2).sum(1).mean((1, 2)).sqrt().clamp_min(1e-30)
            return out * (rms / norm)[:, None, None, None]

        truth = field(r.u_rms, 1)
        members = truth + field(r.pert_rms, k)
        u = torch.cat([members, truth]).contiguous()             # [k + 1, 2, ny, nx]
        rho = torch.ones((k + 1, ny, nx), device=self.device)
        return rho, u[:, 0].contiguous(), u[:, 1].contiguous()

    def enqueue_cycle(self):
        torch, r = self.torch, self.req
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            start.record(self.stream)
            try:
                L.lbm_forecast(self.exp.h, r.steps_per_cycle)
                L.letkf_get_obs(self.exp.h, self.yf.data_ptr(), L.LETKF_DEVICE)
                noise = torch.randn(self.LV, generator=self.gen, device=self.device)
                torch.add(self.yf[r.k], noise, alpha=r.obs_sigma, out=self.yo)
                L.letkf_analyze(self.exp.h, self.yo.data_ptr(), L.LETKF_DEVICE)
            except L.LetkfError as err:
                raise RuntimeError(f"request {r.rid} cycle {self.enqueued}: {err} "
                                   f"(cudaError {self.exp.stats().cuda_error})") from err
            end.record(self.stream)
        self.inflight.append((start, end))
        self.enqueued += 1

    def poll(self) -> int:
        """Retire completed cycles; returns how many completed."""
        n = 0
        while self.inflight and self.inflight[0][1].query():
            start, end = self.inflight.pop(0)
            self.latencies_ms.append(start.elapsed_time(end))
            self.finished += 1
            n += 1
        return n

    def done(self) -> bool:
        return self.finished >= self.req.cycles

    def close(self):
        rc = self.exp.sync()
        if rc:
            raise RuntimeError(f"request {self.req.rid}: {L.strerror(rc)}")
        if self.keep_state:
            self.state = self.exp.get_deviation()
        self.exp.close()
        self.exp = None
        self.yf = self.yo = None


class Server:
    """Continuous-batching request loop under an HBM budget.

    slot_factory(req) builds a running slot (GpuSlot on a device, or a stand-in for tests of
    the scheduling logic); it must expose footprint, enqueue_cycle(), poll(), done(), close(),
    enqueued, finished and latencies_ms.  footprint_of(req) gives the admission footprint
    before a slot exists.
    """

    def __init__(self, hbm_budget_bytes, slot_factory, footprint_of, depth=2,
                 clock=time.perf_counter, sleep=time.sleep, max_active=None):
        self.budget = int(hbm_budget_bytes)
        self.slot_factory = slot_factory
        self.footprint_of = footprint_of
        self.depth = int(depth)
        self.clock = clock
        self.sleep = sleep
        self.max_active = max_active

    def run(self, requests, time_limit_s=None):
        pending = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        for r in pending:
            if self.footprint_of(r) > self.budget:
                raise ValueError(f"request {r.rid} needs {self.footprint_of(r)} bytes, more than "
                                 f"the budget of {self.budget}")
        active, done = [], []
        used = peak = 0
        max_conc = 0
        waits = []
        admitted_at, finished_at = {}, {}
        t0 = self.clock()
        analyses = 0
        timeline = []                     # (time, event, rid, used bytes) for tests
        while pending or active:
            now = self.clock() - t0
            if time_limit_s is not None and now > time_limit_s:
                break
            # admission: first come, first served, as long as memory and slots allow
            while pending and pending[0].arrival_s <= now:
                req = pending[0]
                need = self.footprint_of(req)
                if used + need > self.budget:
                    break
                if self.max_active is not None and len(active) >= self.max_active:
                    break
                pending.pop(0)
                slot = self.slot_factory(req)
                used += need
                peak = max(peak, used)
                active.append((slot, need))
                max_conc = max(max_conc, len(active))
                admitted_at[req.rid] = now
                waits.append(now - req.arrival_s)
                timeline.append((now, "admit", req.rid, used))
            # keep every running slot `depth` cycles ahead
            for slot, _ in active:
                while slot.enqueued < slot.req.cycles and slot.enqueued - slot.finished < self.depth:
                    slot.enqueue_cycle()
            progressed = 0
            still = []
            for slot, need in active:
                n = slot.poll()
                progressed += n
                analyses += n * slot.req.n_points
                if slot.done():
                    slot.close()
                    used -= need
                    t = self.clock() - t0
                    finished_at[slot.req.rid] = t
                    timeline.append((t, "finish", slot.req.rid, used))
                    done.append(slot)
                else:
                    still.append((slot, need))
            active = still
            if not progressed:
                self.sleep(2e-4)
        wall = self.clock() - t0
        errors = []
        for slot, _ in active:          # stopped by the time limit: drain, collect the status
            try:
                slot.close()
            except RuntimeError as err:
                errors.append(str(err))
        lat = [x for s in done for x in s.latencies_ms] + \
              [x for s, _ in active for x in s.latencies_ms]
        by_class = {}
        for cls in ("small", "large"):
            cl = [x for s in done if size_class(s.req) == cls for x in s.latencies_ms] + \
                 [x for s, _ in active if size_class(s.req) == cls for x in s.latencies_ms]
            by_class[cls] = {"cycles": len(cl), "p50": percentile(cl, 50),
                             "p99": percentile(cl, 99)}
        return {
            "requests": len(requests),
            "completed": len(done),
            "cycles": sum(s.finished for s in done) + sum(s.finished for s, _ in active),
            "analyses": analyses,
            "wall_s": wall,
            "analyses_per_s": analyses / wall if wall > 0 else float("nan"),
            "latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99),
                           "mean": float(np.mean(lat)) if lat else float("nan"),
                           "by_class": by_class},
            "admission_wait_s": {"p50": percentile(waits, 50), "p99": percentile(waits, 99),
                                 "max": float(max(waits)) if waits else 0.0},
            "budget_bytes": self.budget,
            "peak_footprint_bytes": peak,
            "max_concurrent": max_conc,
            "slots": done,
            "unfinished": len(active) + len(pending),
            "errors": errors,
            "timeline": timeline,
        }


def gpu_footprint(req: Request) -> int:
    """Admission footprint of a request before its slot exists: the workspace the library
    asks for plus the slot's observation and initial-field buffers."""
    xs = len(range(0, req.nx, req.obs_stride))
    ys = len(range(0, req.ny, req.obs_stride))
    LV = xs * ys * 2
    cfg = L.letkf_config()
    cfg.nx, cfg.ny, cfg.k, cfg.n_aux = req.nx, req.ny, req.k, 1
    cfg.tau = req.tau
    cfg.n_obs = xs * ys
    xy = np.zeros((xs * ys, 2), np.int32)
    var = np.ones(LV, np.float32)
    cfg.obs_xy = xy.ctypes.data_as(L.C.POINTER(L.C.c_int32))
    cfg.obs_vars = L.LETKF_OBS_U | L.LETKF_OBS_V
    cfg.obs_err_var = var.ctypes.data_as(L.C.POINTER(L.C.c_float))
    cfg.loc_kind, cfg.loc_radius = L.LETKF_LOC_GAUSS, float(req.loc_radius)
    cfg.infl = 1.0
    cfg.precision = int(req.precision)
    cfg.eig_schedule = int(req.eig_schedule)
    ws = L.letkf_workspace_size(cfg)
    return ws + 4 * ((req.k + 2) * LV + 3 * (req.k + 1) * req.nx * req.ny)
