"""Serving on the GPU: continuous batching of independent DA experiments.

Five requests of different grids, ensemble sizes and precisions arrive within 20 ms; the HBM
budget holds only some of them at once, so later arrivals wait for memory and are admitted as
earlier ones finish.  Checked:
  * every request completes all its cycles, the footprint never exceeds the budget, and at
    least two slots ran concurrently (their streams overlap);
  * each request's final ensemble is bit for bit the one it gets when served alone (the
    stated tolerance of a served result is that of the analysis; identical arithmetic makes
    the difference exactly zero);
  * every slot stays on its nature run: the analysis RMSE of its ensemble mean stays below
    the members' initial perturbation size;
  * the report carries p50 / p99 cycle latency and throughput.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_2308_03310_gb300 import _build, letkf as L
from paper_2308_03310_gb300.serve import GpuSlot, Request, Server, gpu_footprint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _requests():
    specs = [  # (arrival s, grid, k, stride, cycles, precision)
        (0.000, 48, 16, 4, 6, L.LETKF_FP32),
        (0.002, 64, 40, 4, 5, L.LETKF_MIXED),
        (0.005, 40, 8, 4, 8, L.LETKF_FP32),
        (0.010, 64, 32, 8, 4, L.LETKF_FP32),
        (0.020, 32, 24, 4, 7, L.LETKF_MIXED),
    ]
    return [Request(rid=i, arrival_s=a, nx=g, ny=g, k=k, obs_stride=s, cycles=c,
                    steps_per_cycle=20, precision=p, seed=9000 + i)
            for i, (a, g, k, s, c, p) in enumerate(specs)]


def _serve(reqs, budget):
    srv = Server(budget, lambda r: GpuSlot(r, "cuda", keep_state=True), gpu_footprint)
    return srv.run(reqs)


def _rmse(g, k):
    f = g + lbm.W[None, :, None, None].astype(np.float32)
    _, ux, uy = lbm.moments(f[:k].astype(np.float64))
    _, tx, ty = lbm.moments(f[k].astype(np.float64))
    return float(np.sqrt(np.mean((ux.mean(0) - tx) ** 2 + (uy.mean(0) - ty) ** 2)))


def test_served_results_equal_alone_and_in_the_mix():
    reqs = _requests()
    alone = {}
    for r in reqs:          # one at a time (also fixes the AUTO eigensolve choices first)
        rep = _serve([Request(**{**r.__dict__, "arrival_s": 0.0})], 1 << 40)
        assert rep["completed"] == 1
        alone[r.rid] = rep["slots"][0].state
    fps = sorted(gpu_footprint(r) for r in reqs)
    budget = fps[-1] + fps[-2] + fps[0]      # the two largest and the smallest together
    rep = _serve(reqs, budget)
    assert rep["completed"] == len(reqs)
    assert rep["cycles"] == sum(r.cycles for r in reqs)
    assert rep["peak_footprint_bytes"] <= budget
    assert rep["max_concurrent"] >= 2
    assert rep["admission_wait_s"]["max"] > 0.0            # someone waited for memory
    for slot in rep["slots"]:
        assert np.array_equal(slot.state, alone[slot.req.rid]), slot.req.rid
        assert _rmse(slot.state, slot.req.k) < slot.req.pert_rms
    lat = rep["latency_ms"]
    assert 0 < lat["p50"] <= lat["p99"]
    assert rep["analyses_per_s"] > 0
    assert rep["analyses"] == sum(r.cycles * r.nx * r.ny for r in reqs)
