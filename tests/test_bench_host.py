"""Host-side logic of bench.py, on CPU: clock parsing, roofline and D2Q9 rate arithmetic, the
multi-rank reductions (world size 2 over gloo), the all-core oracle baseline and the reference
(oracle) arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_parse_clock_csv_reads_median_max_and_reasons():
    text = ("0, 1900, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active\n"
            "0, 1950, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 2000, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.parse_clock_csv(text)
    assert c["sm_mhz"] == 1950 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert c["power_w_max"] == 1100.0


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(80.55, rel=1e-3)


def test_roofline_table_fractions_and_shares():
    work = {"a": ("GB", 6.8, 100), "b": ("TFLOP", 0.8, 2)}
    t = bench.roofline_table(work, {"a": 1.0, "b": 3.0}, {"hbm_gbs": 6800.0}, 2070.0)
    assert t["a"]["achieved"] == pytest.approx(6800.0)
    assert t["a"]["frac"] == pytest.approx(1.0)
    assert t["a"]["ms_per_launch"] == pytest.approx(0.01)
    assert t["b"]["bound"] == "alu" and t["b"]["achieved"] == pytest.approx(800 / 3)
    assert t["a"]["share"] + t["b"]["share"] == pytest.approx(1.0)


def test_whole_job_rate_is_weak_scaling_sum():
    assert bench.whole_job_rate(1000, 2.0, 4) == 2000.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_reductions_over_two_gloo_ranks():
    port = _free_port()
    code = ("import os, sys, json; sys.path.insert(0, %r); import bench; "
            "r, w = bench.dist_init('gloo'); "
            "print(json.dumps([bench.reduce_max(1.0 + r), bench.reduce_sum(10.0 * (r + 1))]))" % ROOT)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
        assert json.loads(out.strip().splitlines()[-1]) == [2.0, 30.0]


def test_reference_arm_prints_one_oracle_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tgv32_k8", "--steps", "1", "--warmup", "0",
                        "--cpu-sample-seconds", "1"], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == "tgv32_k8"


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       capture_output=True, text=True, timeout=60, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_lbm_rates_count_updates_and_single_step_bytes():
    import synth
    w = synth.WORKLOADS["turb256_k32"]
    r = bench.lbm_rates(w, 2.0, {"hbm_gbs": 6800.0})
    updates = 256 * 256 * 32 * 100
    assert r["mlups"] == pytest.approx(updates / 2e-3 / 1e6)
    assert r["mlups_per_member"] == pytest.approx(r["mlups"] / 32)
    gbs = (72.0 * updates + 8.0 * 256 * 256 * 100) / 2e-3 / 1e9
    assert r["single_step_equivalent_gbs"] == pytest.approx(gbs)
    assert r["single_step_equivalent_frac"] == pytest.approx(gbs / 6800.0)


def test_kernel_work_counts_two_step_launches():
    import synth
    w = synth.WORKLOADS["turb256_k32"]
    work = bench.kernel_work(w, 32, 65536, 42.0, 2, 1024, 1, 100)
    unit, amount, launches = work["lbm_step"]
    assert launches == 50                       # two steps per launch
    assert amount == pytest.approx((72.0 * 65536 * 32 + 8.0 * 65536) * 50 / 1e9)
    # 99 steps: 49 two-step launches and one single step, the same launch count and bytes
    assert bench.kernel_work(w, 32, 65536, 42.0, 2, 1024, 1, 99)["lbm_step"] == work["lbm_step"]


def test_all_core_oracle_baseline_sums_concurrent_samples(monkeypatch):
    calls = []

    def fake(wname, seconds):
        calls.append((wname, seconds))
        return {"value": 10.0, "unit": bench.UNIT, "cores": 1, "kind": "oracle",
                "sample": "s"}
    monkeypatch.setattr(bench, "run_oracle_subprocess", fake)
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 6)
    r = bench.run_oracle_all_cores("tgv32_k8", 1.5)
    assert r["cores"] == 6 and r["value"] == pytest.approx(60.0)
    assert calls == [("tgv32_k8", 1.5)] * 6
    assert r["sample"].startswith("6 concurrent single-threaded samples")


def test_kernel_work_counts_the_algorithm_of_each_kernel():
    # the Gram forms the upper triangle of a symmetric A (k (k+1) flops per scalar, + 2 k for
    # c); the eigen phase is an EVD with vectors (11 k^3) on the eigenvector schedules and a
    # tridiagonalization plus O(k^2) transform on the EVD-free one
    import synth
    w = synth.WORKLOADS["turb1024_k64"]
    k, npts, lv = 64, 1 << 20, 375.0
    fused = bench.kernel_work(w, k, npts, lv, 2, 65536, 16, 100, schedule=1)
    rat = bench.kernel_work(w, k, npts, lv, 2, 65536, 16, 100, schedule=4)
    assert fused["gram"][1] == pytest.approx((k * (k + 1) + 2 * k) * 2 * lv * npts / 1e12)
    assert fused["eigen_update"][1] == pytest.approx(11.0 * k ** 3 * npts / 1e12)
    assert rat["eigen_update"][1] == pytest.approx(
        (4.0 / 3.0 * k ** 3 + 40.0 * k * k + 36.0 * k * 9) * npts / 1e12)
    assert rat["eigen_update"][1] < 0.2 * fused["eigen_update"][1]
