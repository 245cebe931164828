#!/usr/bin/env python
"""Benchmark: penalised Cox CCD at N = 10^7 subjects on GB300.

Workload (the headline configuration): N = 10,000,000 subjects, p = 100
binary covariates at 5% density in CSC form (float32 values = 1), true beta
~ Laplace(0, 0.2) on 10 coordinates, exponential event times with rate
exp(x.beta), ~50% censoring, times on a 1..3650 day grid (heavy Breslow
ties), L1 penalty lambda = 1e-4 * N, tolerance 1e-8 on the relative change
of the penalised log-likelihood.  Seeded synthetic data (no dataset exists
for this workload).

One step = one complete cox_fit through the C ABI: validation and the tie
group table (a0), then CCD sweeps until convergence (a1-a6): two kernels
per coordinate (row pass; transform + Newton step), one CUDA-graph replay
per sweep (``--schedule persistent``: one cooperative launch per fit).
value = sweeps completed / device time, summed over ranks (each rank fits
its own replica; no data-path collective).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CCD sweeps/s, Cox N=1e7 p=100 5% binary CSC, L1 lambda=1e-4*N"
SN_METRIC = METRIC + ", sparse-numerator form (not the paper's method)"
UNIT = "sweeps/s"
SEED = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--n", type=int, default=None,
                    help="subjects (default: the workload's size, 1e7 for ccd/sn, 5e6 for fg)")
    ap.add_argument("--p", type=int, default=None, help="covariates (default: 100 for ccd/sn, 50 for fg)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline run only: skip the cross-validated path, Fine-Gray and autograd lines that the "
                         "default run attaches (keys cv_path, fine_gray, autograd)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["ccd", "autograd", "cv", "sn", "fg"], default="ccd",
                    help="ccd: the headline penalised Cox fit; autograd: forward + backward of the "
                         "differentiable Cox NLL at N=2^22, p=256, 64 columns (bf16 X); cv: 10-fold "
                         "cross-validation x 20 L1 strengths (200 Cox fits) at N=1e6, p=500, 1%% binary; "
                         "sn: the headline fit in the sparse-numerator form (not the paper's method, "
                         "reported separately); fg: penalised Fine-Gray fit at N=5e6, p=50 dense float32, "
                         "L2 lambda=10")
    ap.add_argument("--ctas", type=int, default=0, help="cv: CTAs per fit (0 = the library's choice)")
    ap.add_argument("--cv-p", type=int, default=500, help="cv: covariates (500 = the benchmarked size; smaller "
                                                           "values give small cases for profiling)")
    ap.add_argument("--no-sequential", action="store_true", help="cv: skip the 200 sequential plain fits")
    ap.add_argument("--spec-b", type=int, choices=[4, 8], default=4,
                    help="coordinates per speculative batch of the default schedule (8: SURV_FLAG_SPEC_B8)")
    ap.add_argument("--schedule", choices=["graph", "one", "persistent"], default="graph",
                    help="graph: the default schedule (two kernels per row pass replayed as a CUDA graph, "
                         "speculative batches of 4 coordinates per row pass); one: one coordinate per row "
                         "pass (the paper's schedule); persistent: one cooperative launch per fit")
    return ap.parse_args()


# Steady-state DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum,
# ncu --cache-control none, means over 10 launches of each kernel) of the
# kernels as committed: per row pass of the headline batches (k_ipass<4> +
# k_itrans<4>), per coordinate of the one-coordinate Cox schedule (k_pass +
# k_btrans) and of the Fine-Gray fit (k_pass + k_btrans).
TRAFFIC_IND_ROW_PASS = 17179904
TRAFFIC_ONE_COORD = 2435456
TRAFFIC_FG_COORD = 71040486
# DRAM bytes of one autograd step's four big kernels at N = 2^20, p = 256,
# 64 columns (k_xb_tc 764.5 MB, k_nll_scan 275.1 MB, k_nll_grad 490.0 MB,
# k_xtg_tc 805.9 MB; one ncu capture each, cold caches)
TRAFFIC_AG_STEP_N20 = 2335500000


def workload(n, p):
    from paper_2204_08183_gb300 import synth
    d = synth.cohort_cox_sparse(n, p, seed=SEED, density=0.05, n_true=10, laplace_scale=0.2,
                                censor_frac=0.5, grid=3650)
    return d


def config_dict(n, p, lam):
    return {"workload": "cox_l1_csc_n%d_p%d" % (n, p), "n": n, "p": p, "density": 0.05,
            "values": "float32 ones (CSC)", "time_grid": 3650, "censoring": 0.5, "penalty": "l1",
            "lambda": lam, "tol": 1e-8, "precision": "fp32 e/scans with float-float carries, fp64 Newton",
            "l2": "inputs larger than L2 (CSC ~400 MB + eta/e 120 MB per replica)",
            "parallelism": "replicas (one independent fit per GPU)"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 20 ms, started
    before the warm-up (its start-up takes longer than a short timed region).
    begin() and end() bracket the timed region on the host clock; the record
    keeps the samples whose timestamps fall inside it (20 ms of slack), or
    every sample when none does."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        # nvidia-smi prints local time as YYYY/MM/DD HH:MM:SS.mmm
        try:
            day, clock = text.strip().split(" ")
            whole, _, frac = clock.partition(".")
            t = time.mktime(time.strptime(day + " " + whole, "%Y/%m/%d %H:%M:%S"))
            return t + (float("0." + frac) if frac else 0.0)
        except Exception:
            return None

    @classmethod
    def summarize(cls, rows, t0=None, t1=None):
        """The clock record of sample rows (lists of the FIELDS values)."""
        inside = rows
        window = "whole sampler run"
        if t0 is not None and t1 is not None:
            slack = cls.PERIOD_MS / 1e3
            sel = [r for r in rows if (lambda t: t is not None and t0 - slack <= t <= t1 + slack)(cls._stamp(r[0]))]
            if sel:
                inside, window = sel, "timed region"
        num = lambda v: v.strip().replace(".", "", 1).isdigit()  # noqa: E731
        sm = [float(r[2]) for r in inside if len(r) > 2 and num(r[2])]
        mx = [float(r[3]) for r in inside if len(r) > 3 and num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for k, name in enumerate(names):
                if len(r) > 6 + k and r[6 + k].strip() == "Active":
                    reasons.add(name)
        loaded = [v for v in sm if v > 0.5 * (max(sm) if sm else 1)]
        return {"sm_mhz": statistics.median(loaded or sm or [0.0]), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(inside), "window": window}

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        if not rows:
            return None
        return self.summarize(rows, self.t0, self.t1)


# --------------------------------------------------------------- oracle sample
def oracle_sample(d, lam, n_coords):
    """Time the FP64 oracle's CCD (as it stands) on a bounded sample of the
    workload: one sweep over the first ``n_coords`` columns at full N.  That
    runs n_coords + 2 risk-set passes (the objective before and after the
    sweep); the time per pass, times p + 1 passes per sweep, gives sweeps/s."""
    import scipy.sparse
    import oracle
    cols = slice(0, n_coords)
    cp = d["col_ptr"][: n_coords + 1]
    nnz = int(cp[-1])
    X = scipy.sparse.csc_matrix((np.ones(nnz), d["row_idx"][:nnz], cp), shape=(d["n"], n_coords))
    t0 = time.perf_counter()
    oracle.ccd_fit("cox", d["time"], d["status"], X, "l1", lam, tol=0.0, max_sweeps=1)
    dt = time.perf_counter() - t0
    passes = n_coords + 2
    per_pass = dt / passes
    return 1.0 / (per_pass * (d["p"] + 1)), dt, passes


def _oracle_core(folder, col, n, lam, barrier, results):
    """One process of the all-cores oracle timing: a one-sweep fit of column
    ``col`` alone (3 risk-set passes at full N), started with the others."""
    import scipy.sparse
    import oracle
    t = np.load(os.path.join(folder, "time.npy"))
    s = np.load(os.path.join(folder, "status.npy"))
    ri = np.load(os.path.join(folder, "ri%d.npy" % col))
    X = scipy.sparse.csc_matrix((np.ones(len(ri)), ri, np.array([0, len(ri)])), shape=(n, 1))
    m = min(n, 20000)  # warm-up on the first rows: one-time costs stay out of the timing
    oracle.ccd_fit("cox", t[:m], s[:m], X[:m], "l1", lam * m / n, tol=0.0, max_sweeps=1)
    barrier.wait()
    t0 = time.perf_counter()
    oracle.ccd_fit("cox", t, s, X, "l1", lam, tol=0.0, max_sweeps=1)
    results.put(time.perf_counter() - t0)


def oracle_sample_all_cores(d, lam):
    """The same oracle on every host core at once: one process per core, each
    a one-sweep fit of its own column (3 risk-set passes at full N), released
    together by a barrier.  Passes per second = all the processes' passes /
    the slowest process's time; sweeps/s = that / (p + 1).  Independent passes
    side by side are the most a host implementation of the same passes could
    gain from the cores (the passes of one cyclic sweep are sequential).
    Processes are spawned (this process already holds a CUDA context)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as folder:
        np.save(os.path.join(folder, "time.npy"), d["time"])
        np.save(os.path.join(folder, "status.npy"), d["status"])
        cp = d["col_ptr"]
        for c in range(cores):
            j = c % d["p"]
            np.save(os.path.join(folder, "ri%d.npy" % c), d["row_idx"][cp[j]:cp[j + 1]])
        barrier = ctx.Barrier(cores)
        results = ctx.Queue()
        procs = [ctx.Process(target=_oracle_core, args=(folder, c, d["n"], lam, barrier, results))
                 for c in range(cores)]
        # one thread per process (the children read these when numpy loads)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            for p_ in procs:
                p_.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        import queue
        times = []
        deadline = time.time() + 600
        while len(times) < cores:
            try:
                times.append(results.get(timeout=2))
            except queue.Empty:
                if any(p_.exitcode not in (None, 0) for p_ in procs) or time.time() > deadline:
                    for p_ in procs:
                        if p_.is_alive():
                            p_.kill()
                    raise RuntimeError("all-cores oracle timing: a worker process failed")
        for p_ in procs:
            p_.join(timeout=60)
    passes = 3 * cores
    per_pass = max(times) / passes
    return 1.0 / (per_pass * (d["p"] + 1)), max(times), passes, cores


# --------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import torch
    from paper_2204_08183_gb300 import binding
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n, p = args.n or 10_000_000, args.p or 100
    lam = 1e-4 * n
    d = workload(n, p)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    sd = binding.SurvData(dev(d["time"]), dev(d["status"]), col_ptr=dev(d["col_ptr"]), row_idx=dev(d["row_idx"]),
                          values=dev(d["values"]), n=n, p=p)
    ws = binding.Workspace()
    stream = torch.cuda.current_stream()
    sn = args.workload == "sn"
    flags = binding.SURV_FLAG_PERSISTENT if args.schedule == "persistent" else 0
    if sn:
        flags = binding.SURV_FLAG_SPARSE_NUMERATOR
    if args.schedule == "one":
        flags = binding.SURV_FLAG_ONE_COORDINATE
    if args.spec_b == 8 and not sn and args.schedule == "graph":
        flags |= binding.SURV_FLAG_SPEC_B8
    kw = dict(penalty="l1", lam=lam, tol=1e-8, max_sweeps=1000, workspace=ws, flags=flags)
    beta_dev = torch.zeros(p, dtype=torch.float64, device="cuda")
    # the sampler starts before the warm-up so that its start-up cannot fall
    # inside the timed region; its samples cover warm-up and timed fits
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(1.5)
    for _ in range(args.warmup):
        beta_dev.zero_()
        binding.cox_fit(sd, beta=beta_dev, **kw)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.synchronize()
    clocks.begin()
    ev0.record(stream)
    for _ in range(args.steps):
        beta_dev.zero_()
        _, info, rc = binding.cox_fit(sd, beta=beta_dev, **kw)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    sweeps = sum(i["sweeps"] for i in infos)
    launches = int(sum(i["kernel_launches"] for i in infos))
    beta_final = beta_dev.cpu().numpy()

    # max over ranks of the timed region; sum of work
    t_max, sweeps_all = ms, sweeps
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ss = torch.tensor([float(sweeps)], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(ss, op=torch.distributed.ReduceOp.SUM)
        t_max, sweeps_all = float(tt.item()), float(ss.item())
    value = sweeps_all / (t_max / 1e3)

    # Roofline of the dominant kernel.  The unit of work is one coordinate:
    # the k_pass + k_trans pair (graph schedule) that reads e over all N rows
    # and the column's CSC slice; its duration is the fit's CCD device time
    # (all graph replays, kernel gaps included) divided by the coordinate
    # passes.  Eta updates after nonzero steps are counted in the bytes.
    nnz = int(d["col_ptr"][-1])
    K = infos[-1]["n_groups"]
    passes = sum(i["coordinate_passes"] for i in infos)
    upd = sum(i["eta_updates"] for i in infos)
    # CSC values that are all 1 are indicators: the library drops them and
    # reads only the row indices of a column
    ind = d["values"] is None or bool(np.all(d["values"] == 1))
    vb = 0 if ind else 4                              # bytes of a value per nonzero
    # per coordinate: column j (row, value) + group table; e is streamed only
    # when it changed since the previous pass (after a nonzero step, and at
    # the first pass of a fit), otherwise the stored sums of e are reused
    per_pass = (4 + vb) * nnz / p + 8 * K
    per_update = (24 + vb) * nnz / p                  # row, value, eta r/w (8+8), e write
    alg_bytes = passes * per_pass + min(passes, upd + len(infos)) * 4 * n + upd * per_update
    row_passes = sum(i["row_passes"] for i in infos)
    batched = (not sn) and args.schedule == "graph" and row_passes < passes
    if batched:
        # speculative batches: a row pass reads the slices of up to B columns
        # (counted as B: an upper bound on the columns read) and the group
        # table; it streams e only when e has changed since the previous
        # pass (after a nonzero step, and at the first pass of a fit):
        # otherwise the stored sums of e are reused
        per_row_pass = args.spec_b * (4 + vb) * nnz / p + 8 * K
        dense_passes = min(row_passes, upd + len(infos))
        alg_bytes = row_passes * per_row_pass + dense_passes * 4 * n + upd * per_update
    if sn:
        # per coordinate: column j (row, value) and, per nonzero, e, its
        # group, Lambda and W (4 + 4 + 8 + 8); per rebuild of the risk sets
        # (one per nonzero step, plus the first): e over all rows and the
        # group table (Den, v1, v2, Lambda, W, d)
        per_pass = 32 * nnz / p
        alg_bytes = passes * per_pass + upd * per_update + (upd + len(infos)) * (4 * n + 44 * K)
    kern_ms = sum(i["ccd_kernel_ms"] for i in infos)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    us_per_coord = kern_ms * 1e3 / passes
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback 6800 GB/s",
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                "unit_of_work": "one coordinate (row pass + transform/Newton)",
                "algorithmic_bytes_per_coordinate": round(alg_bytes / passes),
                "us_per_coordinate": round(us_per_coord, 3),
                "passes_per_fit": passes / len(infos), "eta_updates_per_fit": upd / len(infos),
                "row_passes_per_fit": row_passes / len(infos)}
    bw4 = args.spec_b == 4
    if batched:
        roofline["unit_of_work"] = "one row pass (a speculative batch of up to %d coordinates)" % args.spec_b
        if n == 10_000_000 and p == 100 and ind and bw4 and TRAFFIC_IND_ROW_PASS:
            # dram__bytes_read.sum + dram__bytes_write.sum of k_ipass<4> +
            # k_itrans<4> per row pass, steady state (ncu --cache-control
            # none); see profiles/k_ipass_k_itrans_cox_csc_n1e7.md
            roofline["traffic"] = TRAFFIC_IND_ROW_PASS
            roofline["traffic_note"] = "bytes per row pass, ncu steady-state capture of the kernels as committed"
        roofline["algorithmic_bytes_per_row_pass"] = round(alg_bytes / row_passes)
        roofline["row_passes_streaming_e_per_fit"] = dense_passes / len(infos)
        roofline["us_per_row_pass"] = round(kern_ms * 1e3 / row_passes, 3)
    if batched:
        roofline.setdefault("traffic", None)
    elif args.schedule == "one" and n == 10_000_000 and p == 100 and not sn:
        # dram__bytes_read.sum + dram__bytes_write.sum of k_pass + k_btrans per
        # coordinate, steady state; see profiles/k_pass_k_btrans_cox_csc_n1e7.md.
        # e stays in L2 across coordinates; DRAM sees the column slice and the
        # eta / e writes.
        roofline["traffic"] = TRAFFIC_ONE_COORD
        roofline["traffic_note"] = "bytes per coordinate, ncu steady-state capture of the kernels as committed"
    else:
        roofline["traffic"] = None
    roofline["kernel"] = ("ccd_kernel<cox,csc,f32> (persistent, one launch per fit)" if args.schedule == "persistent"
                          else "k_pass + k_btrans <cox,csc,f32>, one pair per coordinate, one graph replay per sweep")
    if batched:
        bw = args.spec_b
        roofline["kernel"] = (("k_ipass<%d> + k_itrans<%d>" if ind else "k_spass<%d> + k_strans<%d>") % (bw, bw) +
                              ": one pair per speculative batch of %d coordinates, graph replays of batches" % bw)
    if sn:
        roofline["kernel"] = ("k_sn_den_a/den_b/lam (after nonzero steps only) + k_sn_col_a/col_b per coordinate, "
                              "one graph replay per sweep")
        roofline["unit_of_work"] = "one coordinate (column pass; risk-set rebuild after nonzero steps)"
    if args.schedule == "persistent":
        roofline["phase_ms_per_launch"] = {k: round(sum(i["phase_ms"][q] for i in infos) / len(infos), 4)
                                           for q, k in enumerate(["pass_cta0", "ex1_arrive", "ex1_wait",
                                                                  "ex1_after", "transform", "ex2_arrive",
                                                                  "ex2_wait", "ex2_newton", "update",
                                                                  "pass_max_cta", "pass_min_cta",
                                                                  "pass_mean_cta", "dense_max_cta",
                                                                  "sparse_max_cta", "ex1_sums", "ex1_stores"])}

    out = {"metric": SN_METRIC if sn else METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
           "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config_dict(n, p, lam), "roofline": roofline, "clocks": clk, "gpu_launches": launches,
           "fit": {"sweeps_per_fit": infos[-1]["sweeps"], "converged": infos[-1]["converged"],
                   "row_passes_per_fit": infos[-1]["row_passes"],
                   "nnz_beta": infos[-1]["nnz_beta"], "loglik": infos[-1]["loglik"], "n_groups": K,
                   "ms_per_fit": round(t_max / args.steps, 3)}}

    if sn:
        out["config"]["workload"] += "_sparse_numerator"
    # end to end: host (pinned) buffers through the same C ABI call
    if not args.no_e2e:
        host = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        ht, hs, hcp, hri, hv = host(d["time"]), host(d["status"]), host(d["col_ptr"]), host(d["row_idx"]), \
            host(d["values"])
        hd = binding.SurvData(ht, hs, col_ptr=hcp, row_idx=hri, values=hv, n=n, p=p)
        hbeta = torch.zeros(p, dtype=torch.float64).pin_memory()
        binding.cox_fit(hd, beta=hbeta, **kw)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        e_inf = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            hbeta.zero_()
            _, inf, _ = binding.cox_fit(hd, beta=hbeta, **kw)
            e_inf.append(inf)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        h2d = sum(int(a.numel() * a.element_size()) for a in (ht, hs, hcp, hri, hv)) + 8 * p
        d2h = 8 * p + 8 * p + 256 * 3
        out["e2e"] = {"value": round(sum(i["sweeps"] for i in e_inf) * world / (ems / 1e3), 2), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "note": "cox_fit with pinned host arrays: the library copies them to the device, fits, "
                              "and copies beta back inside the call"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sn:
        sps, dt, npass = oracle_sample(d, lam, 6)
        out["cpu_baseline"] = {"value": round(sps, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "oracle.ccd_fit, one sweep over the first 6 of 100 columns at "
                                         "N=1e7 (%d risk-set passes, %.1f s); sweeps/s = 1/(time per pass * "
                                         "(p+1))" % (npass, dt)}
        sps_all, dt_all, npass_all, cores = oracle_sample_all_cores(d, lam)
        out["cpu_baseline_all_cores"] = {
            "value": round(sps_all, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle.ccd_fit on every host core at once: %d processes, each a one-sweep fit of its own "
                      "column at N=1e7 (%d risk-set passes in all, slowest process %.1f s); sweeps/s = "
                      "passes / slowest time / (p+1), independent passes side by side" % (cores, npass_all, dt_all)}
    out["beta_nonzero"] = int((beta_final != 0).sum())
    return out


# ------------------------------------------------ differentiable form (f2)
AG_METRIC = "Cox NLL forward+backward/s, eta = X B, N=2^22 p=256 C=64, bf16 X (tcgen05 tensor-core products)"


def run_autograd(args, rank, world):
    """One step = cox_nll_forward + cox_nll_backward through the C ABI at
    N = 2^22, p = 256, C = 64 (X bf16 row-major, B float32), device-resident
    inputs; e2e = the autograd function with the inputs copied from pinned
    host memory each step."""
    import torch
    from paper_2204_08183_gb300 import binding, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n, p, C = args.n or (1 << 22), 256, 64
    c = synth.nll_cohort(n, p, C, seed=5, n_times=5000)
    X = torch.from_numpy(c["X"]).cuda().to(torch.bfloat16)
    B = torch.from_numpy(c["B"]).cuda()
    t = torch.from_numpy(c["time"]).cuda()
    s = torch.from_numpy(c["status"]).cuda()
    g = torch.ones(C, dtype=torch.float64, device="cuda")
    ws = binding.Workspace()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(1.5)
    for _ in range(args.warmup):
        binding.cox_nll_forward(X, t, s, B, ws)
        binding.cox_nll_backward(X, t, s, g, C, ws)
    torch.cuda.synchronize()
    # L2 (129 MB) is far smaller than X (2 GiB) and Y (2 GiB): no flush needed
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evf = torch.cuda.Event(enable_timing=True)
    fwd_ms = 0.0
    clocks.begin()
    ev0.record(stream)
    for _ in range(args.steps):
        binding.cox_nll_forward(X, t, s, B, ws)
        binding.cox_nll_backward(X, t, s, g, C, ws)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    ms = ev0.elapsed_time(ev1) / args.steps
    # forward alone, for the split
    ev0.record(stream)
    for _ in range(args.steps):
        binding.cox_nll_forward(X, t, s, B, ws)
    evf.record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(evf) / args.steps
    clk = clocks.stop()
    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    value = world * 1e3 / t_max
    # minimal bytes: X read by both products, eta written by the forward and
    # read by the backward
    alg = 2 * (2 * n * p) + 2 * (4 * n * C)
    # as implemented: X B reads X and writes eta; the forward scan reads eta;
    # the backward reads eta, writes G (bf16, 2 Cp columns) and X^T G reads
    # X and G
    Cp = max(32, (C + 15) // 16 * 16)
    moved = (2 * n * p + 4 * n * C) + 4 * n * C + (4 * n * C + 2 * n * 2 * Cp) + (2 * n * p + 2 * n * 2 * Cp)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg / (t_max / 1e3) / 1e9
    out = {"metric": AG_METRIC, "value": round(value, 2), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16 X, f32 B/eta, f64 logs", "data": "synthetic",
           "config": {"workload": "cox_nll_autograd_n%d_p256_c64" % n, "n": n, "p": p, "columns": C,
                      "time_grid": 5000, "censoring": 0.3,
                      "l2": "inputs larger than L2 (X 2 GiB, eta 1 GiB)"},
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4),
                        # DRAM bytes of k_xb_tc + k_nll_scan + k_nll_grad + k_xtg_tc
                        # in one ncu capture at N = 2^20 (the products and the
                        # scans move bytes in proportion to N), times 4; see
                        # profiles/tcgen05_products_cox_nll_p256_c64.md and
                        # profiles/k_nll_scan_k_nll_grad_n1m_c64.md
                        "traffic": (TRAFFIC_AG_STEP_N20 * n // (1 << 20)) if p == 256 and C == 64 else None,
                        "traffic_note": "bytes per step, ncu capture at N=2^20 scaled by N",
                        "algorithmic_bytes_per_step": alg, "implementation_bytes_per_step": moved,
                        "forward_ms": round(fwd_ms, 3), "backward_ms": round(t_max - fwd_ms, 3),
                        "kernel": "tcgen05 products k_xb_tc (X B) and k_xtg_tc (X^T G), TMA + TMEM, "
                                  "+ k_nll_scan/finish/lambda/grad"},
           "clocks": clk, "gpu_launches": args.steps * 14}
    if not args.no_e2e:
        # autograd function, inputs copied from pinned host memory every step
        hX = X.cpu().pin_memory()
        hB = B.cpu().pin_memory()
        ht, hs = t.cpu().pin_memory(), s.cpu().pin_memory()
        e_steps = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(e_steps):
            Xd, td, sd = hX.cuda(non_blocking=True), ht.cuda(non_blocking=True), hs.cuda(non_blocking=True)
            Bd = hB.cuda(non_blocking=True).requires_grad_(True)
            nll = binding.cox_nll(Bd, Xd, td, sd)
            (gB,) = torch.autograd.grad(nll.sum(), Bd)
            nll.detach().cpu(), gB.cpu()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / e_steps
        out["e2e"] = {"value": round(world * 1e3 / ems, 2), "unit": "steps/s",
                      "h2d_bytes_per_step": 2 * n * p + 4 * p * C + 5 * n, "d2h_bytes_per_step": 8 * C + 4 * p * C,
                      "note": "binding.cox_nll (autograd) forward + backward with X, B, time, status copied from "
                              "pinned host memory each step"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        Xo = X[:, :].float().cpu().numpy()
        t0 = time.perf_counter()
        eta = Xo.astype(np.float64) @ c["B"][:, :1].astype(np.float64)
        oracle.cox_nll(c["time"], c["status"], eta)
        ge = oracle.cox_nll_grad_eta(c["time"], c["status"], eta)
        Xo.T.astype(np.float64) @ ge
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(1.0 / (dt * C), 6), "unit": "steps/s", "cores": 1, "kind": "oracle",
                               "sample": "oracle NLL + gradient of 1 of the 64 columns at full N (%.1f s); "
                                         "steps/s = 1 / (64 x that)" % dt}
    return out


# ------------------------------------------ cross-validated path (f1)
CV_METRIC = "CV fits/s, Cox 10-fold x 20 L1 lambdas (200 fits), N=1e6 p=500 1% binary CSC"


def cv_workload(p=500):
    from paper_2204_08183_gb300 import synth
    d = synth.cohort_cox_sparse(1_000_000, p, seed=41, density=0.01, n_true=10, laplace_scale=0.2,
                                censor_frac=0.4, grid=3650)
    fold = synth.cv_folds(1_000_000, 10, seed=42)
    return d, fold


def run_cv(args, rank, world):
    """One step = one cox_cv_path call: 10 folds x 20 L1 strengths from
    lambda_max down to 1e-3 lambda_max, 200 cold-started fits in one batched
    graph schedule, then the held-out scores and the choice of lambda.
    Device-resident inputs; e2e = the same call on pinned host arrays.  The
    same 200 fits as sequential plain cox_fit calls (one per training set,
    device-resident subsets) are timed once for comparison."""
    import torch
    from paper_2204_08183_gb300 import binding, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    d, fold = cv_workload(args.cv_p)
    n, p = d["n"], d["p"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    sd = binding.SurvData(dev(d["time"]), dev(d["status"]), col_ptr=dev(d["col_ptr"]), row_idx=dev(d["row_idx"]),
                          values=dev(d["values"]), n=n, p=p)
    fold_d = dev(fold)
    lmax = binding.cox_lambda_max(sd)
    lam = synth.lambda_grid(lmax, 20)
    ws = binding.Workspace()
    stream = torch.cuda.current_stream()
    kw = dict(penalty="l1", tol=1e-8, max_sweeps=1000, workspace=ws, ctas_per_fit=args.ctas)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(1.5)
    for w in range(args.warmup):
        # the first warm-up call tunes the CTAs per fit and the row-pass form
        # (kept in the workspace)
        tune = binding.SURV_FLAG_CV_TUNE if (w == 0 and args.ctas == 0) else 0
        binding.cox_cv_path(sd, fold_d, 10, lam, flags=tune, **kw)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    clocks.begin()
    ev0.record(stream)
    for _ in range(args.steps):
        res.append(binding.cox_cv_path(sd, fold_d, 10, lam, **kw))
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    F = 200
    value = world * F * args.steps / (t_max / 1e3)
    infos = [r["info"] for r in res]
    last = res[-1]
    # roofline of the batched pass: every active fit reads its e over all N
    # rows and column j's slice per coordinate, plus the eta / e update of
    # the column's rows after a nonzero step
    nnz = int(d["col_ptr"][-1])
    K = infos[-1]["n_groups"]
    passes = sum(i["coordinate_passes"] for i in infos)
    upd = sum(i["eta_updates"] for i in infos)
    # column j's row indices (indicator data: no values) and the group table
    # per coordinate; e over all N rows only after a nonzero step and at each
    # fit's first pass (otherwise its stored sums are reused)
    per_pass = 4 * nnz / p + 8 * K
    per_update = 24 * nnz / p
    alg = passes * per_pass + min(passes, upd + F * len(infos)) * 4 * n + upd * per_update
    kern_ms = sum(i["ccd_kernel_ms"] for i in infos)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg / (kern_ms / 1e3) / 1e9
    sweeps = last["sweeps"]
    out = {"metric": CV_METRIC, "value": round(value, 2), "unit": "fits/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "cox_cv10x20_l1_csc_n1000000_p%d" % p, "n": n, "p": p, "density": 0.01,
                      "folds": 10, "fold_sizes": [int(x) for x in np.bincount(fold, minlength=10)],
                      "lambdas": 20, "lambda_max": lmax, "lambda_ratio": 1e-3, "tol": 1e-8, "censoring": 0.4,
                      "time_grid": 3650, "start": "cold (beta = 0) for every fit",
                      "ctas_per_fit": infos[-1]["ctas_per_fit"],
                      "row_pass_form": {1: "one warp reduction per group end",
                                        2: "lane scans per tile"}[infos[-1]["row_pass_form"]],
                      "tile_form": {0: "4 loads of e per lane a tile, 4 rounds of nonzeros a load",
                                    1: "2 loads of e per lane a tile, 4 rounds of nonzeros a load",
                                    2: "4 loads of e per lane a tile, 2 rounds of nonzeros a load"}[
                          infos[-1]["tile_form"]],
                      "ctas_source": "autotuned with the row-pass form and tile shape (one timed sweep per "
                                     "candidate, first warm-up call)"
                      if args.ctas == 0 else "--ctas",
                      "l2": "inputs larger than L2 (e + eta of 200 fits: 2.4 GB)"},
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "traffic_note": "not a whole-path figure: a capture of early launches (all 200 fits active, most passes streaming e) read 440-540 MB and wrote 56-78 MB a launch; see profiles/k_pass_batched_cv_n1e6.md",
                        "unit_of_work": "one coordinate of one active fit (batched row pass)",
                        "algorithmic_bytes_per_coordinate": round(alg / max(passes, 1)),
                        "coordinate_passes_per_step": passes / len(infos),
                        "eta_updates_per_step": upd / len(infos),
                        "ccd_ms_per_step": round(kern_ms / len(infos), 3),
                        "heldout_ms_per_step": round(sum(i["heldout_ms"] for i in infos) / len(infos), 3),
                        "graph_replays": infos[-1]["graph_replays"],
                        "kernel": "k_pass + k_trans <cox,csc,f32,batched>, grid (ctas_per_fit, 200)"},
           "clocks": clk, "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
           "cv": {"best_lambda": infos[-1]["best_lambda"], "sweeps_max": int(sweeps.max()),
                  "sweeps_mean": float(sweeps.mean()), "fits_converged": infos[-1]["fits_converged"],
                  "cv_mean": [round(float(x), 3) for x in last["cv_mean"]]}}
    if not args.no_e2e:
        host = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        ht, hs, hcp, hri, hv, hf = (host(d["time"]), host(d["status"]), host(d["col_ptr"]), host(d["row_idx"]),
                                    host(d["values"]), host(fold))
        hd = binding.SurvData(ht, hs, col_ptr=hcp, row_idx=hri, values=hv, n=n, p=p)
        binding.cox_cv_path(hd, hf, 10, lam, **kw)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 2))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            binding.cox_cv_path(hd, hf, 10, lam, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / e_steps
        h2d = sum(int(a.numel() * a.element_size()) for a in (ht, hs, hcp, hri, hv, hf)) + 8 * 20
        d2h = 8 * F * p + 8 * F + 8 * 20 + 4 * F
        out["e2e"] = {"value": round(world * F * 1e3 / ems, 2), "unit": "fits/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h,
                      "note": "cox_cv_path on pinned host arrays: the library copies them in and the 200 "
                              "coefficient vectors, scores and sweep counts out inside the call"}
    if not args.no_sequential and rank == 0:
        # the same fits one after another through the plain cox_fit (each
        # training set built once on the device beforehand, untimed)
        subs = []
        for k in range(10):
            m = fold != k
            rows = np.flatnonzero(m)
            newidx = np.full(n, -1, np.int64)
            newidx[rows] = np.arange(rows.shape[0])
            cp = [0]
            ri = []
            for j in range(p):
                r = d["row_idx"][d["col_ptr"][j]:d["col_ptr"][j + 1]]
                r = newidx[r]
                r = r[r >= 0].astype(np.int32)
                ri.append(r)
                cp.append(cp[-1] + r.shape[0])
            ri = np.concatenate(ri)
            subs.append(binding.SurvData(dev(d["time"][m]), dev(d["status"][m]), col_ptr=dev(np.array(cp, np.int64)),
                                         row_idx=dev(ri), values=dev(np.ones(ri.shape[0], np.float32)),
                                         n=int(m.sum()), p=p))
        ws2 = binding.Workspace()
        beta = torch.zeros(p, dtype=torch.float64, device="cuda")
        binding.cox_fit(subs[0], beta=beta, penalty="l1", lam=float(lam[10]), tol=1e-8, max_sweeps=1000,
                        workspace=ws2)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for li in range(20):
            for k in range(10):
                beta.zero_()
                binding.cox_fit(subs[k], beta=beta, penalty="l1", lam=float(lam[li]), tol=1e-8, max_sweeps=1000,
                                workspace=ws2)
        s1.record(stream)
        torch.cuda.synchronize()
        sms = s0.elapsed_time(s1)
        out["sequential_plain"] = {"value": round(F * 1e3 / sms, 3), "unit": "fits/s", "ms": round(sms, 1),
                                   "note": "the 200 fits as sequential cox_fit calls on device-resident "
                                           "training sets (same lambdas, cold start, same tolerance)"}
        out["speedup_vs_sequential_plain"] = round(value / (F * 1e3 / sms), 2)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import scipy.sparse
        import oracle
        m = fold != 0
        nc = 4
        cp = d["col_ptr"][: nc + 1]
        X = scipy.sparse.csc_matrix((np.ones(int(cp[-1])), d["row_idx"][: int(cp[-1])], cp), shape=(n, nc))
        Xt = X[np.flatnonzero(m)]
        t0 = time.perf_counter()
        oracle.ccd_fit("cox", d["time"][m], d["status"][m], Xt, "l1", float(lam[10]), tol=0.0, max_sweeps=1)
        dt = time.perf_counter() - t0
        per_pass = dt / (nc + 2)
        avg_passes = passes / len(infos) / F
        out["cpu_baseline"] = {"value": round(1.0 / (per_pass * avg_passes), 6), "unit": "fits/s", "cores": 1,
                               "kind": "oracle",
                               "sample": "oracle.ccd_fit on fold 0's training set (9e5 subjects), one sweep over "
                                         "4 columns (%d risk-set passes, %.1f s); fits/s = 1 / (time per pass x "
                                         "%.0f passes per fit, the GPU run's mean)" % (nc + 2, dt, avg_passes)}
    return out


# ------------------------------------------------ Fine-Gray, dense X
FG_METRIC = "CCD sweeps/s, Fine-Gray N=5e6 p=50 dense float32, L2 lambda=10"


def fg_config(n, p):
    return {"workload": "fg_l2_dense_n%d_p%d" % (n, p), "n": n, "p": p, "layout": "dense column-major float32",
            "outcomes": "40% censored / 35% primary / 25% competing", "time_grid": 1000, "penalty": "l2",
            "lambda": 10.0, "tol": 1e-8,
            "precision": "fp32 e/scans with float-float carries, fp64 Newton, Kaplan-Meier weights on the device",
            "l2": "inputs larger than L2 (X 1 GB + eta/e/W 80 MB per replica)",
            "parallelism": "replicas (one independent fit per GPU)"}


def run_fg(args, rank, world):
    """One step = one complete fg_fit through the C ABI on the Fine-Gray
    workload (N = 5e6, p = 50 dense float32 N(0,1) covariates, 40/35/25%
    censored/primary/competing outcomes from exponential hazards with their
    own linear predictors, times on 1..1000, L2 lambda = 10, tol 1e-8):
    Kaplan-Meier censoring weights and the tie-group table on the device
    (a0), then one coordinate per row pass (a1-a6) until convergence."""
    import torch
    from paper_2204_08183_gb300 import binding, synth
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n = args.n or 5_000_000
    p = args.p or 50
    d = synth.cohort_fg_dense(n, p, seed=3, grid=1000, n_true=10)
    Xt = torch.from_numpy(np.ascontiguousarray(d["X"].T))          # (p, n): column-major X
    t_h, s_h = torch.from_numpy(d["time"]), torch.from_numpy(d["status"])
    sd = binding.SurvData(t_h.cuda(), s_h.cuda(), X=Xt.cuda())
    ws = binding.Workspace()
    stream = torch.cuda.current_stream()
    flags = binding.SURV_FLAG_PERSISTENT if args.schedule == "persistent" else 0
    kw = dict(penalty="l2", lam=10.0, tol=1e-8, max_sweeps=1000, workspace=ws, flags=flags)
    beta_dev = torch.zeros(p, dtype=torch.float64, device="cuda")
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(1.5)
    for _ in range(args.warmup):
        beta_dev.zero_()
        binding.fg_fit(sd, beta=beta_dev, **kw)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    torch.cuda.synchronize()
    clocks.begin()
    ev0.record(stream)
    for _ in range(args.steps):
        beta_dev.zero_()
        _, info, _ = binding.fg_fit(sd, beta=beta_dev, **kw)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    sweeps = sum(i["sweeps"] for i in infos)
    t_max, sweeps_all = ms, float(sweeps)
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ss = torch.tensor([float(sweeps)], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(ss, op=torch.distributed.ReduceOp.SUM)
        t_max, sweeps_all = float(tt.item()), float(ss.item())
    value = sweeps_all / (t_max / 1e3)

    # Roofline: the unit is one coordinate (row pass + transform/Newton).  A
    # row pass reads e, x_j and the competing-event weight W over all N rows
    # (12 B/row) plus the group table (K ends: e_k, d_k, G(t_k)); after a
    # nonzero step the update reads x_j and eta (float-float) and writes eta
    # and e (24 B/row).
    K = infos[-1]["n_groups"]
    passes = sum(i["coordinate_passes"] for i in infos)
    upd = sum(i["eta_updates"] for i in infos)
    per_pass = 12 * n + 16 * K
    per_update = 24 * n
    alg_bytes = passes * per_pass + upd * per_update
    kern_ms = sum(i["ccd_kernel_ms"] for i in infos)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback 6800 GB/s",
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                "unit_of_work": "one coordinate (row pass + transform/Newton)",
                "algorithmic_bytes_per_coordinate": round(alg_bytes / passes),
                "us_per_coordinate": round(kern_ms * 1e3 / passes, 3),
                "passes_per_fit": passes / len(infos), "eta_updates_per_fit": upd / len(infos),
                "kernel": ("ccd_kernel<fg,dense,f32> (persistent, one launch per fit)"
                           if args.schedule == "persistent" else
                           "k_pass + k_btrans <fg,dense,f32>, one pair per coordinate, one graph replay per sweep")}
    if args.schedule == "graph" and n == 5_000_000 and p == 50:
        # steady-state DRAM bytes per coordinate (see
        # profiles/k_pass_k_btrans_fg_dense_n5e6.md): below the algorithmic
        # bytes because the previous coordinate's column (read again for the
        # eta update) and part of eta / e / W are still in L2
        roofline["traffic"] = TRAFFIC_FG_COORD
        roofline["traffic_note"] = "bytes per coordinate, ncu steady-state capture of the kernels as committed"
    out = {"metric": FG_METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": fg_config(n, p), "roofline": roofline, "clocks": clk,
           "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
           "fit": {"sweeps_per_fit": infos[-1]["sweeps"], "converged": infos[-1]["converged"],
                   "loglik": infos[-1]["loglik"], "n_groups": K, "ms_per_fit": round(t_max / args.steps, 3)}}
    if not args.no_e2e:
        ht, hs, hX = t_h.pin_memory(), s_h.pin_memory(), Xt.pin_memory()
        hd = binding.SurvData(ht, hs, X=hX)
        hbeta = torch.zeros(p, dtype=torch.float64).pin_memory()
        binding.fg_fit(hd, beta=hbeta, **kw)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        e_inf = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            hbeta.zero_()
            _, inf, _ = binding.fg_fit(hd, beta=hbeta, **kw)
            e_inf.append(inf)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        h2d = sum(int(a.numel() * a.element_size()) for a in (ht, hs, hX)) + 8 * p
        d2h = 8 * p + 8 * p + 256 * 3
        out["e2e"] = {"value": round(sum(i["sweeps"] for i in e_inf) * world / (ems / 1e3), 2), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "note": "fg_fit with pinned host arrays: the library copies them to the device, fits, "
                              "and copies beta back inside the call"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        nc = 10
        Xs = np.asfortranarray(d["X"][:, :nc])
        t0 = time.perf_counter()
        oracle.ccd_fit("fg", d["time"], d["status"], Xs, "l2", 10.0, tol=0.0, max_sweeps=1)
        dt = time.perf_counter() - t0
        per_pass = dt / (nc + 2)
        out["cpu_baseline"] = {"value": round(1.0 / (per_pass * (p + 1)), 5), "unit": UNIT, "cores": 1,
                               "kind": "oracle",
                               "sample": "oracle.ccd_fit('fg'), one sweep over the first %d of %d columns at "
                                         "N=%d (%d risk-set passes, %.1f s); sweeps/s = 1/(time per pass * "
                                         "(p+1))" % (nc, p, n, nc + 2, dt)}
    return out


def run_reference(args, rank, world):
    """The oracle on the host cores: each step one bounded sample."""
    if rank != 0:
        return None
    n, p = args.n or 10_000_000, args.p or 100
    lam = 1e-4 * n
    d = workload(n, p)
    vals = []
    for _ in range(args.warmup):
        oracle_sample(d, lam, 1)
    t_tot = 0.0
    for _ in range(args.steps):
        sps, dt, npass = oracle_sample(d, lam, 1)
        vals.append(sps)
        t_tot += dt
    value = float(np.mean(vals))
    sample = ("oracle.ccd_fit, one sweep over the first column at N=1e7 (3 risk-set passes); "
              "sweeps/s = 1/(time per pass * (p+1))")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_tot / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(n, p, lam),
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_extra(args):
    """The other parts of the metric, each with its own timed region and clock
    record: the batched cross-validated path against 200 sequential plain
    fits (10 folds x 20 lambdas, N = 1e6, p = 500), the Fine-Gray fit
    (N = 5e6, p = 50 dense) and the autograd step (N = 2^22, p = 256, C = 64).
    Their oracle baselines are left to their own --workload runs."""
    import copy
    import gc
    import torch
    extra = {}
    for key, fn, steps, warmup in (("cv_path", run_cv, 3, 3), ("fine_gray", run_fg, 10, 3),
                                   ("autograd", run_autograd, 20, 3)):
        a = copy.copy(args)
        a.steps, a.warmup, a.no_cpu_baseline = steps, warmup, True
        a.n = a.p = None
        a.schedule = "graph"
        try:
            extra[key] = fn(a, 0, 1)
        except Exception as e:  # report, keep the headline line
            extra[key] = {"error": "%s: %s" % (type(e).__name__, e)}
        gc.collect()
        torch.cuda.empty_cache()
    return extra


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "autograd":
        out = run_autograd(args, rank, world)
    elif args.workload == "cv":
        out = run_cv(args, rank, world)
    elif args.workload == "fg":
        out = run_fg(args, rank, world)
    elif args.workload == "sn":
        out = run_gpu(args, rank, world)
    else:
        out = run_gpu(args, rank, world)
    if (args.impl == "gb300" and args.workload == "ccd" and world == 1 and not args.no_extra and out is not None
            and args.n is None and args.p is None):
        out.update(run_extra(args))
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
