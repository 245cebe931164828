"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Integer work (sort permutation, tie-group ends, event counts) must match
bit for bit.  The Kaplan-Meier product runs in the order of its definition
for up to 4096 tie groups and must then match bit for bit too; beyond that
it runs as a fixed-order chunked product and is held to the error bound of
an FP64 product of K factors.  Floating results follow the tolerances derived
in the design notes: the FP32-compensated mode stores e = exp(eta) in FP32
(relative error ~1e-7 per term) and accumulates in float-float, so
l is within 1e-6 relative and l', l'' within 1e-6 of the scale
sum_k d_k max|x|^m; the FP64 mode is held to 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

from gpu_util import oracle_X, small_csc, survdata

pytestmark = pytest.mark.gpu


def _tol(prec):
    return 1e-6 if prec == "f32c" else 1e-10


def _check_lgh(d, model, beta, j, prec, where="device"):
    sd = survdata(d, where)
    l, g, h = binding.loglik_grad_hess(sd, model, np.asarray(beta, np.float64), j, precision=prec)
    X = oracle_X(d)
    st = d["status"] if model == "fg" else np.where(d["status"] == 2, 0, d["status"]).astype(np.int8)
    lo, go, ho = oracle.model_terms(model, d["time"], st, X, beta, j)
    D = max(1, int((st == 1).sum()))
    xm = float(np.abs(oracle.column(X, j)).max()) if len(d["time"]) else 1.0
    tol = _tol(prec)
    assert abs(l - lo) <= tol * max(abs(lo), 1.0), (l, lo)
    assert abs(g - go) <= tol * D * max(xm, 1e-300) + tol * abs(go), (g, go)
    assert abs(h - ho) <= tol * D * max(xm * xm, 1e-300) + tol * abs(ho), (h, ho)
    return (l, g, h), (lo, go, ho)


# ------------------------------------------------------------ integer parity
@pytest.mark.parametrize("n", [1, 7, 1000, 123457, 2_000_001])
def test_sort_desc_bit_exact(lib, n):
    rng = np.random.default_rng(n)
    t = rng.integers(-50, 50 if n < 1000 else 3650, size=n).astype(np.int32)
    if n > 10:
        t[:5] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0, -1, 1]
    perm = binding.surv_sort_desc(t)
    assert np.array_equal(np.asarray(perm), oracle.sort_desc(t).astype(np.int32))
    import torch
    permd = binding.surv_sort_desc(torch.from_numpy(t).cuda())
    assert np.array_equal(permd.cpu().numpy(), oracle.sort_desc(t).astype(np.int32))


@pytest.mark.parametrize("n,n_times", [(1, 1), (5, 1), (1000, 1000), (1000, 37), (3_000_017, 3650)])
def test_groups_bit_exact(lib, n, n_times):
    rng = np.random.default_rng(n + n_times)
    t = np.sort(rng.integers(1, n_times + 1, size=n))[::-1].astype(np.int32)
    st = rng.choice(np.array([0, 1, 2], np.int8), size=n, p=[0.4, 0.35, 0.25])
    gend, dk, Gk = binding.surv_groups(t, st)
    og = oracle.tie_groups(t)
    assert np.array_equal(gend, og.astype(np.int32))
    assert np.array_equal(dk, oracle.group_counts(og, st, 1).astype(np.int32))
    assert np.array_equal(Gk, oracle.km_censoring_groups(t, st, og))   # same order of FP64 products


@pytest.mark.parametrize("K", [4096, 4097, 2_000_003])
def test_groups_many_km_factors(lib, K):
    """K tie groups with censoring in most of them: up to 4096 the product is
    sequential (bit-exact); above, a chunked product whose relative error,
    like the sequential one's, stays below K u (u = 2^-53) of the exact
    value, so the two differ by at most 2 K u relative."""
    rng = np.random.default_rng(K)
    n = K + K // 3
    t = np.sort(rng.choice(np.arange(1, 4 * K + 1), size=K, replace=False))[::-1].astype(np.int32)
    t = np.sort(np.concatenate([t, rng.choice(t, size=n - K)]))[::-1].astype(np.int32)
    st = rng.choice(np.array([0, 1, 2], np.int8), size=n, p=[0.5, 0.3, 0.2])
    gend, dk, Gk = binding.surv_groups(t, st)
    og = oracle.tie_groups(t)
    assert og.shape[0] == K
    assert np.array_equal(gend, og.astype(np.int32))
    assert np.array_equal(dk, oracle.group_counts(og, st, 1).astype(np.int32))
    ref = oracle.km_censoring_groups(t, st, og)
    assert ref.min() < 0.05                          # a long product, far from 1
    if K <= 4096:
        assert np.array_equal(Gk, ref)
    else:
        np.testing.assert_allclose(Gk, ref, rtol=2 * K * 2.0 ** -53, atol=0)


def test_fg_fit_near_unique_times(lib):
    """Fine-Gray fit where almost every subject has its own time (K close to
    N): the censoring weights come from the chunked Kaplan-Meier product and
    every warp of the row pass holds many group ends."""
    n, p = 200_003, 4
    d = synth.cohort_small(n, p, seed=31, n_times=50 * n, censor_frac=0.3, competing_frac=0.25)
    st = d["status"]
    K = oracle.tie_groups(d["time"]).shape[0]
    assert K > 0.9 * n
    sd = survdata(d)
    beta, info, rc = binding.fg_fit(sd, penalty="l2", lam=2.0, tol=0.0, max_sweeps=3)
    ref = oracle.ccd_fit("fg", d["time"], st, d["X"], "l2", 2.0, tol=0.0, max_sweeps=3)
    assert info["sweeps"] == 3 and info["n_groups"] == K
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5)
    assert info["loglik"] == pytest.approx(ref["loglik"], rel=1e-6)


# ------------------------------------------------------------ one pass
@pytest.mark.parametrize("prec", ["f32c", "f64"])
@pytest.mark.parametrize("model", ["cox", "fg"])
@pytest.mark.parametrize("n,n_times", [(1, 1), (2, 2), (33, 4), (1000, 1000), (4099, 60), (20011, 365)])
def test_lgh_dense_small(lib, prec, model, n, n_times):
    d = synth.cohort_small(n, 3, seed=n, n_times=n_times, censor_frac=0.3,
                           competing_frac=0.25 if model == "fg" else 0.0)
    st = d["status"].copy()
    st[0] = 1  # at least one event
    d["status"] = st
    for j in range(3):
        _check_lgh(d, model, d["beta"], j, prec)


@pytest.mark.parametrize("prec", ["f32c", "f64"])
@pytest.mark.parametrize("model", ["cox", "fg"])
@pytest.mark.parametrize("binary", [False, True])
@pytest.mark.parametrize("n,n_times", [(517, 30), (40_003, 400), (300_007, 3650)])
def test_lgh_csc(lib, prec, model, binary, n, n_times):
    d = small_csc(n, 4, seed=n + binary, density=0.05, n_times=n_times,
                  competing=0.25 if model == "fg" else 0.0, binary=binary,
                  dtype=np.float32 if prec == "f32c" else np.float64)
    for j in range(4):
        _check_lgh(d, model, d["beta"] * 0.5, j, prec)


@pytest.mark.parametrize("model", ["cox", "fg"])
def test_lgh_many_tiles_per_warp(lib, model):
    # > 5e6 rows: every warp of the grid streams several 1024-row tiles, and
    # n is not a multiple of 4 (ragged tail).
    n = 5_300_003
    if model == "cox":
        d = synth.cohort_cox_sparse(n, 3, seed=11, density=0.05, n_true=2, grid=3650)
        d["values"] = None
        beta = np.array([0.1, -0.2, 0.05])
    else:
        d = synth.cohort_fg_dense(n, 2, seed=12, grid=1000, n_true=2)
        beta = np.array([0.2, -0.1])
    for j in range(d["p"] if "p" in d else 2):
        _check_lgh(d, model, beta, j, "f32c")


def test_lgh_edge_cases(lib):
    X = np.asfortranarray(np.array([[0.5], [-1.0], [2.0], [0.0]]))
    cases = [
        # all tied, one event
        (np.array([3, 3, 3, 3], np.int32), np.array([0, 1, 0, 0], np.int8)),
        # no ties, all events
        (np.array([9, 7, 5, 1], np.int32), np.array([1, 1, 1, 1], np.int8)),
        # all censored except the last
        (np.array([9, 7, 5, 1], np.int32), np.array([0, 0, 0, 1], np.int8)),
        # all censored except the first (risk set of one)
        (np.array([9, 7, 5, 1], np.int32), np.array([1, 0, 0, 0], np.int8)),
    ]
    for t, st in cases:
        d = {"time": t, "status": st, "X": X, "layout": "dense"}
        for prec in ["f32c", "f64"]:
            for b in [0.0, 0.7]:
                _check_lgh(d, "cox", [b], 0, prec)
                _check_lgh(d, "fg", [b], 0, prec)


def test_zero_column_has_zero_gradient(lib):
    d = synth.cohort_small(300, 2, seed=3, n_times=20)
    d["X"][:, 1] = 0.0
    sd = survdata(d)
    _, g, h = binding.loglik_grad_hess(sd, "cox", d["beta"], 1)
    assert g == 0.0 and h == 0.0


def test_host_and_device_buffers_agree(lib):
    d = small_csc(20_000, 3, seed=4, density=0.1, n_times=200)
    a = binding.loglik_grad_hess(survdata(d, "device"), "cox", d["beta"], 2)
    b = binding.loglik_grad_hess(survdata(d, "host"), "cox", d["beta"], 2)
    assert a == b


def test_deterministic(lib):
    d = small_csc(200_000, 3, seed=5, density=0.05, n_times=3000)
    sd = survdata(d)
    r = [binding.loglik_grad_hess(sd, "cox", d["beta"], 1) for _ in range(3)]
    assert r[0] == r[1] == r[2]
    f1 = binding.cox_fit(sd, penalty="l1", lam=5.0, tol=1e-10)
    f2 = binding.cox_fit(sd, penalty="l1", lam=5.0, tol=1e-10)
    assert np.array_equal(f1[0], f2[0]) and f1[1]["sweeps"] == f2[1]["sweeps"]


# ------------------------------------------------------------ full fits
# graph: the default (speculative batches for Cox CSC FP32 fits); one: one
# coordinate per row pass; persistent: one cooperative launch per fit
SCHEDULES = {"graph": 0, "one": binding.SURV_FLAG_ONE_COORDINATE, "persistent": binding.SURV_FLAG_PERSISTENT}


def _fit_check(model, d, penalty, lam, prec, beta_tol=1e-5, tol=1e-10, where="device", schedule="graph"):
    sd = survdata(d, where)
    fn = binding.cox_fit if model == "cox" else binding.fg_fit
    beta, info, rc = fn(sd, penalty=penalty, lam=lam, tol=tol, max_sweeps=500, precision=prec,
                        flags=SCHEDULES[schedule])
    X = oracle_X(d)
    st = d["status"] if model == "fg" else np.where(d["status"] == 2, 0, d["status"]).astype(np.int8)
    ref = oracle.ccd_fit(model, d["time"], st, X, penalty, lam, tol=tol, max_sweeps=500)
    assert rc == 0 and info["converged"] == 1 and ref["converged"]
    np.testing.assert_allclose(beta, ref["beta"], atol=beta_tol, rtol=0)
    assert abs(info["loglik"] - ref["loglik"]) <= 1e-6 * abs(ref["loglik"])
    # Near tol ~ 1e-10 the relative objective change reaches the FP32 rounding
    # floor of e = exp(eta) (~1e-11), so the FP32-mode stopping sweep may land
    # a little later than the FP64 oracle's; the iterates themselves must
    # agree: same number of sweeps on the oracle side, tol = 0.
    assert abs(info["sweeps"] - ref["sweeps"]) <= (1 if prec == "f64" else 3)
    same = oracle.ccd_fit(model, d["time"], st, X, penalty, lam, tol=0.0, max_sweeps=info["sweeps"])
    np.testing.assert_allclose(beta, same["beta"], atol=beta_tol, rtol=0)
    # zeros of an L1 fit are exact on both sides
    if penalty == "l1":
        assert np.array_equal(beta == 0.0, ref["beta"] == 0.0)
    return beta, info, ref


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_fit_dense_cox_l2_config1_shape(lib, prec):
    # N = 10,000 subjects, p = 10 dense N(0,1) covariates, 365-day grid,
    # ~30% censoring, L2 lambda = 1, relative-change tolerance 1e-8.
    d = synth.cohort_cox_dense(10_000, 10, seed=1, n_true=5, beta_sd=0.5, censor_frac=0.3, grid=365)
    _fit_check("cox", d, "l2", 1.0, prec, tol=1e-8)


@pytest.mark.parametrize("schedule", ["graph", "one", "persistent"])
@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_fit_csc_cox_l1(lib, prec, schedule):
    d = synth.cohort_cox_sparse(60_000, 20, seed=2, density=0.05, n_true=4, laplace_scale=0.5, grid=3650)
    if prec == "f64":
        d["values"] = d["values"].astype(np.float64)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d))
    _fit_check("cox", d, "l1", 0.2 * lmax, prec, schedule=schedule)


@pytest.mark.parametrize("schedule", ["graph", "persistent"])
@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_fit_fg_dense_l2(lib, prec, schedule):
    d = synth.cohort_fg_dense(30_000, 6, seed=3, grid=1000, n_true=4, dtype=np.float32 if prec == "f32c" else np.float64)
    _fit_check("fg", d, "l2", 10.0, prec, schedule=schedule)


@pytest.mark.parametrize("schedule", ["graph", "persistent"])
def test_fit_fg_csc_l1(lib, schedule):
    d = small_csc(40_000, 10, seed=16, density=0.08, n_times=800, competing=0.25)
    lmax = oracle.lambda_max("fg", d["time"], d["status"], oracle_X(d))
    _fit_check("fg", d, "l1", 0.25 * lmax, "f32c", schedule=schedule)


@pytest.mark.parametrize("kind", ["heavy_ties", "near_unique_times"])
def test_fit_csc_cox_staged_pass(lib, kind):
    # Millions of rows: every warp of the pass kernel owns more than one tile,
    # so e is staged in shared memory and walked lane by lane.  Near-unique
    # times put hundreds of group ends in each warp (more than 32 of them,
    # and more than two in one lane).
    if kind == "heavy_ties":
        d = synth.cohort_cox_sparse(3_000_000, 5, seed=31, density=0.05, n_true=3, laplace_scale=0.5, grid=3650)
    else:
        d = small_csc(2_000_000, 4, seed=32, density=0.05, n_times=1_500_000)
    lmax = oracle.lambda_max("cox", d["time"], np.where(d["status"] == 2, 0, d["status"]).astype(np.int8),
                             oracle_X(d))
    _fit_check("cox", d, "l1", 0.2 * lmax, "f32c", tol=1e-9)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fit_few_coordinates(lib, p):
    # p = 1 folds the finish of a coordinate and the objective evaluation
    # into the same kernel of the next sweep; p = 2, 3 cover the wrap-around
    d = synth.cohort_cox_dense(8_000, p, seed=40 + p, n_true=p, grid=150)
    _fit_check("cox", d, "l2", 2.0, "f32c", tol=1e-9)


def test_fit_graph_reuse_in_workspace(lib):
    # the second fit in a workspace replays the cached graph; a third with
    # another lambda captures a new one
    d = synth.cohort_cox_sparse(40_000, 9, seed=17, density=0.05, n_true=3, laplace_scale=0.5, grid=900)
    sd = survdata(d)
    ws = binding.Workspace()
    lmax = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d))
    runs = [binding.cox_fit(sd, penalty="l1", lam=lam * lmax, tol=1e-10, workspace=ws) for lam in (0.3, 0.3, 0.1)]
    assert np.array_equal(runs[0][0], runs[1][0]) and runs[0][1]["sweeps"] == runs[1][1]["sweeps"]
    ref = oracle.ccd_fit("cox", d["time"], d["status"], oracle_X(d), "l1", 0.1 * lmax, tol=1e-10, max_sweeps=500)
    np.testing.assert_allclose(runs[2][0], ref["beta"], atol=1e-5)


def test_fit_fg_csc_l1_host_buffers(lib):
    d = small_csc(25_000, 8, seed=6, density=0.1, n_times=500, competing=0.25)
    lmax = oracle.lambda_max("fg", d["time"], d["status"], oracle_X(d))
    _fit_check("fg", d, "l1", 0.3 * lmax, "f32c", where="host")


def test_fit_unpenalised_and_warm_start(lib):
    d = synth.cohort_cox_dense(5_000, 4, seed=7, n_true=3, grid=200)
    sd = survdata(d)
    b0 = np.array([0.1, -0.1, 0.2, 0.0])
    beta, info, rc = binding.cox_fit(sd, beta=b0.copy(), penalty="none", tol=1e-12, max_sweeps=300)
    ref = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "none", 0.0, tol=1e-12, max_sweeps=300, beta0=b0)
    np.testing.assert_allclose(beta, ref["beta"], atol=1e-6)


def test_lambda_max_gives_zero(lib):
    d = synth.cohort_cox_sparse(50_000, 12, seed=8, density=0.05, n_true=3, grid=1000)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d))
    beta, info, rc = binding.cox_fit(survdata(d), penalty="l1", lam=lmax * 1.001, tol=1e-10)
    assert np.all(beta == 0.0) and info["eta_updates"] == 0


@pytest.mark.parametrize("schedule", ["graph", "persistent"])
def test_max_sweeps_reports_not_converged(lib, schedule):
    d = synth.cohort_cox_dense(3_000, 5, seed=9, n_true=4, grid=100)
    beta, info, rc = binding.cox_fit(survdata(d), penalty="l2", lam=1.0, tol=0.0, max_sweeps=3,
                                     flags=SCHEDULES[schedule])
    assert rc == binding.SURV_W_NOT_CONVERGED and info["sweeps"] == 3 and info["converged"] == 0
    ref = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "l2", 1.0, tol=0.0, max_sweeps=3)
    np.testing.assert_allclose(beta, ref["beta"], atol=1e-7)
    assert info["coordinate_passes"] == 3 * 5 + 1
    b0 = np.full(5, 0.05)
    beta, info, rc = binding.cox_fit(survdata(d), beta=b0.copy(), penalty="l2", lam=1.0, tol=0.0, max_sweeps=0,
                                     flags=SCHEDULES[schedule])
    assert rc == binding.SURV_W_NOT_CONVERGED and info["sweeps"] == 0 and np.array_equal(beta, b0)
    ref = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "l2", 1.0, tol=0.0, max_sweeps=0, beta0=b0)
    assert abs(info["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_fit_dense_bfloat16_x(lib, prec):
    # bfloat16 dense X is widened on the device: the fit is the oracle's fit
    # of the rounded X
    import torch
    d = synth.cohort_cox_dense(6_000, 5, seed=51, n_true=3, beta_sd=0.5, grid=300)
    Xb = torch.from_numpy(np.ascontiguousarray(d["X"].T.astype(np.float32))).to(torch.bfloat16)
    sd = binding.SurvData(torch.from_numpy(d["time"]).cuda(), torch.from_numpy(d["status"]).cuda(), X=Xb.cuda())
    assert sd.c.dtype == binding.SURV_BF16
    beta, info, rc = binding.cox_fit(sd, penalty="l2", lam=1.0, tol=1e-10, precision=prec)
    Xr = Xb.float().numpy().T.astype(np.float64)
    ref = oracle.ccd_fit("cox", d["time"], d["status"], Xr, "l2", 1.0, tol=0.0, max_sweeps=info["sweeps"])
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5 if prec == "f32c" else 1e-9)


def test_bfloat16_csc_values_rejected(lib):
    import torch
    d = small_csc(500, 3, seed=52, density=0.3, n_times=40)
    sd = binding.SurvData(torch.from_numpy(d["time"]).cuda(), torch.from_numpy(d["status"]).cuda(),
                          col_ptr=torch.from_numpy(d["col_ptr"]).cuda(), row_idx=torch.from_numpy(d["row_idx"]).cuda(),
                          values=torch.from_numpy(d["values"]).cuda().to(torch.bfloat16), n=500, p=3)
    with pytest.raises(binding.SurvError) as e:
        binding.cox_fit(sd, penalty="l2", lam=1.0)
    assert e.value.code == binding.SURV_E_INVALID
