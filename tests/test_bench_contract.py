"""bench.py's output contract, checked on the CPU through its reference arm
(the FP64 oracle on a small sample): one JSON line with the keys the
benchmark contract names, the reference's own cpu_baseline and e2e, and
nothing printed by ranks other than 0; and the JSON assembly of the GPU
arms with their device calls replaced by fakes."""
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--n", "200000"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in r, k
    assert r["impl"] == "reference"
    assert r["steps"] == 2 and r["warmup"] == 1 and r["n_gpus"] == 1
    assert r["unit"] == "sweeps/s" and r["higher_is_better"] is True
    assert r["value"] > 0
    assert r["config"]["workload"] == "cox_l1_csc_n200000_p100"
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == r["value"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    args = types.SimpleNamespace(n=None, p=None, steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None


def test_workload_defaults():
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "ccd" and a.impl == "gb300"
    assert a.n is None and a.p is None      # the workload's own size (1e7 x 100 for ccd)


def test_gpu_arms_assemble_the_contract_line(monkeypatch):
    """The JSON assembly of the GPU arms (headline Cox and Fine-Gray), run on
    the host with the device calls replaced by fakes that return fixed fit
    records: every key of the contract is present and derived as stated
    (value = sweeps / device time, roofline fraction = achieved / peak).
    No number here is a measurement."""
    import torch
    sys.path.insert(0, ROOT)
    try:
        import bench
        import __graft_entry__
        from paper_2204_08183_gb300 import binding
    finally:
        sys.path.remove(ROOT)

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 20.0                                       # ms for the timed fits

    zeros = torch.zeros
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: zeros(*a, **{x: v for x, v in k.items() if x != "device"}))
    monkeypatch.setattr(__graft_entry__, "build", lambda: None)
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)

    def fit(sd, beta=None, **kw):
        return beta, {"sweeps": 4, "converged": 1, "loglik": -1.0, "n_groups": 100, "coordinate_passes": 40,
                      "eta_updates": 30, "ccd_kernel_ms": 0.004, "kernel_launches": 90, "row_passes": 12,
                      "nnz_beta": 3}, 0

    monkeypatch.setattr(binding, "cox_fit", fit)
    monkeypatch.setattr(binding, "fg_fit", fit)
    monkeypatch.setattr(binding, "Workspace", lambda: None)
    for argv, run in ((["--n", "20000", "--p", "10"], bench.run_gpu),
                      (["--workload", "fg", "--n", "20000", "--p", "10"], bench.run_fg)):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        a = bench.parse()
        out = run(a, 0, 1)
        for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                  "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches",
                  "e2e", "cpu_baseline"):
            assert k in out, k
        assert out["value"] == 4 * a.steps / 0.020
        assert out["gpu_launches"] == 90 * a.steps
        r = out["roofline"]
        for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
            assert k in r, k
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3, abs=1e-4) and r["frac"] > 0
        e = out["e2e"]
        assert e["unit"] == out["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
        assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
        assert out["config"]["workload"].endswith("n20000_p10")


def test_all_cores_oracle_timing(monkeypatch):
    # one spawned process per core (two here), each a one-sweep fit of its
    # own column: 3 risk-set passes each, timed from a common barrier
    sys.path.insert(0, ROOT)
    try:
        import bench
        from paper_2204_08183_gb300 import synth
    finally:
        sys.path.remove(ROOT)
    d = synth.cohort_cox_sparse(20_000, 4, seed=2, density=0.05, n_true=2, laplace_scale=0.2, censor_frac=0.5,
                                grid=365)
    monkeypatch.setattr(os, "sched_getaffinity", lambda pid: {0, 1}, raising=False)
    sps, slowest, passes, cores = bench.oracle_sample_all_cores(d, 2.0)
    assert cores == 2 and passes == 6
    assert slowest > 0 and sps == pytest.approx(passes / slowest / (d["p"] + 1))


def test_clock_record_keeps_the_samples_of_the_timed_region():
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    import time as _time
    base = _time.mktime(_time.strptime("2026/12/04 12:00:00", "%Y/%m/%d %H:%M:%S"))

    def row(sec, mhz, thermal="Not Active"):
        stamp = _time.strftime("%Y/%m/%d %H:%M:%S", _time.localtime(base + int(sec))) + ".%03d" % round(
            (sec % 1) * 1000)
        return [stamp, "0", str(mhz), "2070", "900.0", "0x0", "Not Active", thermal, "Not Active", "Not Active"]

    rows = [row(0.0, 1200), row(0.5, 1200, "Active"), row(1.00, 2070), row(1.02, 2040), row(1.04, 2070),
            row(2.0, 1000)]
    rec = bench.ClockSampler.summarize(rows, base + 0.99, base + 1.05)
    assert rec["window"] == "timed region" and rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["reasons"] == []
    # no sample inside the region: every sample, and the reasons seen anywhere
    rec = bench.ClockSampler.summarize(rows, base + 3.0, base + 3.01)
    assert rec["window"] == "whole sampler run" and rec["samples"] == len(rows)
    assert rec["reasons"] == ["hw_thermal_slowdown"]
