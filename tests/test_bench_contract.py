"""bench.py's host-side contract on CPU: the reference arm's JSON line (the FP64
oracle timed on the host cores), its ``unavailable`` line on the workloads the
oracle is not run on, the roofline arithmetic against the derived FP64/FP32 pipe
peaks and the measured HBM copy bandwidth, and the clock sampler's timed-region
window."""

import json
import os
import sys
import tempfile
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _one_json_line(capsys):
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1, out
    return json.loads(out[0])


@pytest.mark.parametrize("workload", ["dense512-lanczos", "dense512-rsvd"])
def test_reference_arm_prints_the_contract_line(capsys, monkeypatch, workload):
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--workload", workload, "--steps", "2", "--warmup", "1"]) == 0
    line = _one_json_line(capsys)
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "s" and line["higher_is_better"] is False
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] == pytest.approx(line["value"] * 1e3)
    assert line["config"]["workload"] == workload and "oracle_cycles" not in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    if bench.WORKLOADS[workload]["method"] == "blanczos":
        assert str(bench.WORKLOADS[workload]["oracle_cycles"]) in cb["sample"]


def test_reference_arm_is_unavailable_where_the_oracle_is_not_run(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--workload", "powerlaw2m-lanczos-mixed", "--steps", "1",
                       "--warmup", "0"]) == 0
    line = _one_json_line(capsys)
    assert line["impl"] == "reference" and line["unavailable"]


def test_reference_arm_runs_the_whole_oracle_solve_on_the_householder_matrix(capsys, monkeypatch):
    """The dense workload's reference arm (a miniature of it here): the matrix built on
    the host with the device generator's formula, the whole oracle solve per step, and
    the same config dict as the GPU arm's line."""
    monkeypatch.delenv("RANK", raising=False)
    small = dict(bench.WORKLOADS["dense20k-lanczos"], m=700, n=500, k=8, b=16, r=4)
    monkeypatch.setitem(bench.WORKLOADS, "dense20k-lanczos", small)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    line = _one_json_line(capsys)
    assert line["impl"] == "reference" and line["value"] > 0
    assert "whole solve" in line["cpu_baseline"]["sample"]
    assert line["config"] == {"workload": "dense20k-lanczos", **{k: v for k, v in small.items()
                                                                  if k != "oracle_cycles"},
                              "parallelism": "replicas1"}


def test_every_lanczos_workload_the_oracle_runs_states_its_cycle_count():
    for name, cfg in bench.WORKLOADS.items():
        if cfg["method"] == "blanczos" and cfg["kind"] in ("csr", "dense"):
            assert int(cfg["oracle_cycles"]) >= 1, name


def _classes(dom, ms, flops, nbytes, launches):
    ms_cls, fl_cls, by_cls, ln_cls = [0.0] * 6, [0.0] * 6, [0.0] * 6, [0] * 6
    ms_cls[dom], fl_cls[dom], by_cls[dom], ln_cls[dom] = ms, flops, nbytes, launches
    return ms_cls, fl_cls, by_cls, ln_cls


def test_roofline_arithmetic(tsvd):
    from paper_2403_06218_gb300._capi import KERNEL_CLASSES
    peaks = bench._measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6790.3))
    fp64 = 152 * 4 * mhz * 1e6 / 1e12             # 2 DFMA a clock on each of the 152 SMs
    fp32 = 152 * 256 * mhz * 1e6 / 1e12           # 128 FFMA a clock
    nn, ap = KERNEL_CLASSES.index("gemm_nn"), KERNEL_CLASSES.index("a_products")
    csr = bench.WORKLOADS["sparse100k-lanczos-thick"]
    mixed = bench.WORKLOADS["sparse100k-lanczos-thick-mixed"]

    # FP64 GEMM class: 10 launches, 1e12 flops in 2 s -> 0.5 TFLOP/s against the FP64 pipe
    r = bench._roofline(csr, nn, *_classes(nn, 2000.0, 1e12, 4e9, 10))
    assert r["kernel"] == "gemm_nn" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(0.5) and r["peak"] == pytest.approx(fp64)
    assert r["frac"] == pytest.approx(0.5 / fp64)
    assert r["avg_launch_ms"] == pytest.approx(200.0) and r["flops_per_launch"] == pytest.approx(1e11)
    assert r["hbm_frac_of_measured"] == pytest.approx(2.0 / hbm)

    # the same class in the mixed form runs on the FP32 pipe
    r = bench._roofline(mixed, nn, *_classes(nn, 2000.0, 1e12, 4e9, 10))
    assert r["peak"] == pytest.approx(fp32) and r["frac"] == pytest.approx(0.5 / fp32)

    # sparse A products are bound by HBM: 6e9 algorithmic bytes in 1 ms -> 6,000 GB/s
    r = bench._roofline(csr, ap, *_classes(ap, 1.0, 1e9, 6e9, 3))
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6000.0) and r["peak"] == pytest.approx(hbm)
    assert r["frac"] == pytest.approx(6000.0 / hbm) and r["traffic"] is None

    # dense FP64 A products are sliced products on the tensor cores: 28 BF16 digit-pair
    # products per FP64 multiply-add, against the measured BF16 peak
    dense = bench.WORKLOADS["dense20k-lanczos"]
    bf16 = float(peaks.get("bf16_tflops", 1914.6))
    r = bench._roofline(dense, ap, *_classes(ap, 10.0, 1e11, 6e9, 2))
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["fp64_equiv_tflops"] == pytest.approx(10.0)
    assert r["achieved"] == pytest.approx(280.0) and r["frac"] == pytest.approx(280.0 / bf16)
    # and in the mixed form they are the split-BF16 product, bound by HBM
    r = bench._roofline(bench.WORKLOADS["dense20k-lanczos-mixed"], ap, *_classes(ap, 10.0, 1e11, 6e9, 2))
    assert r["bound"] == "hbm"


def test_default_workload_is_the_dense_20k_solve():
    src = open(bench.__file__).read()
    assert 'default="dense20k-lanczos"' in src
    cfg = bench.WORKLOADS["dense20k-lanczos"]
    assert (cfg["m"], cfg["n"], cfg["k"], cfg["b"], cfg["r"]) == (20_000, 20_000, 100, 128, 4)
    assert cfg.get("precision", "fp64") == "fp64" and cfg["tol"] == 1e-6


def test_clock_sampler_keeps_only_the_timed_window():
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    now = time.time()

    def stamp(t):
        return time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)

    rows = [(now - 5, 1000, "Active"), (now + 1, 2070, "Not Active"), (now + 2, 2060, "Not Active"),
            (now + 3, 2070, "Not Active"), (now + 9, 900, "Active")]
    with open(s.path, "w") as f:
        for t, mhz, thermal in rows:
            f.write(f"{stamp(t)}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, {thermal}, Not Active, Active\n")
    s.t0, s.t1 = now + 0.5, now + 3.5
    out = s.summary()
    assert out["window"] == "timed region" and out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    # hw_thermal_slowdown was active only outside the window; sw_power_cap is kept and noted
    assert out["reasons"] == ["sw_power_cap"]
