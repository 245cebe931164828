"""GPU parity of the cross-validated penalty path (cox_cv_path) and of
cox_lambda_max against the FP64 oracle (oracle/cv.py, oracle.lambda_max).

Every fit of the batched schedule is compared with the oracle's fit of the
same training subset run for the same number of sweeps: beta within 1e-5
(FP32-compensated mode; 1e-9 in FP64), held-out scores within 1e-6
relative (1e-10), and the chosen lambda identical.  At the benchmarked size
(N = 10^6, p = 500, 10 uneven folds x 20 lambdas) the check is sampled:
one fit against the oracle's fit of its training set (same sweeps), and
held-out scores recomputed by the oracle at the GPU's beta."""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

from gpu_util import oracle_X, small_csc, survdata

pytestmark = pytest.mark.gpu

TOL_B = {"f32c": 1e-5, "f64": 1e-9}
TOL_H = {"f32c": 1e-6, "f64": 1e-10}


def _compare(d, fold, nfolds, lambdas, penalty, prec, ctas=0, tol=1e-9, flags=0):
    sd = survdata(d)
    r = binding.cox_cv_path(sd, fold, nfolds, lambdas, penalty=penalty, precision=prec, tol=tol,
                            max_sweeps=200, ctas_per_fit=ctas, flags=flags)
    info = r["info"]
    assert info["nfits"] == len(lambdas) * nfolds
    assert info["fits_converged"] == info["nfits"]
    ref = oracle.cv_path(d["time"], d["status"], oracle_X(d), fold, nfolds, lambdas, penalty,
                         sweeps=r["sweeps"])
    np.testing.assert_allclose(r["beta"], ref["beta"], rtol=0, atol=TOL_B[prec])
    np.testing.assert_allclose(r["heldout"], ref["heldout"], rtol=TOL_H[prec], atol=1e-12)
    np.testing.assert_allclose(r["cv_mean"], ref["cv_mean"], rtol=TOL_H[prec], atol=1e-12)
    m = np.sort(ref["cv_mean"])
    if m.shape[0] < 2 or m[-1] - m[-2] > 1e-4 * abs(m[-1]):
        assert info["best_lambda"] == ref["best"]
    return r, ref


@pytest.mark.parametrize("prec", ["f32c", "f64"])
@pytest.mark.parametrize("ctas", [0, 1, 3])
def test_cv_path_csc_matches_oracle(lib, prec, ctas):
    d = small_csc(3001, 10, seed=21, density=0.3, n_times=300)
    d["values"] = d["values"].astype(np.float32 if prec == "f32c" else np.float64)
    fold = synth.cv_folds(3001, 3, seed=22)
    lmax = binding.cox_lambda_max(survdata(d))
    lam = synth.lambda_grid(lmax, 4, ratio=1e-2)
    _compare(d, fold, 3, lam, "l1", prec, ctas)


@pytest.mark.parametrize("tile", [1, 2])
@pytest.mark.parametrize("n_times", [20, 300])   # few ends per warp (one reduction an end) / many (lane scans)
def test_cv_path_tile_shapes_match_oracle(lib, tile, n_times):
    d = small_csc(3001, 10, seed=31, density=0.3, n_times=n_times)
    fold = synth.cv_folds(3001, 3, seed=32)
    lam = synth.lambda_grid(binding.cox_lambda_max(survdata(d)), 4, ratio=1e-2)
    flag = binding.SURV_FLAG_CV_TILE1 if tile == 1 else binding.SURV_FLAG_CV_TILE2
    r, _ = _compare(d, fold, 3, lam, "l1", "f32c", ctas=3, flags=flag)
    assert r["info"]["tile_form"] == tile
    assert r["info"]["row_pass_form"] == (2 if n_times == 300 else 1)


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_cv_path_dense_l2_matches_oracle(lib, prec):
    d = synth.cohort_small(2500, 6, seed=23, n_times=150, censor_frac=0.4,
                           dtype=np.float32 if prec == "f32c" else np.float64)
    fold = synth.cv_folds(2500, 4, seed=24)
    _compare(d, fold, 4, [10.0, 1.0, 0.1], "l2", prec, ctas=2)


def test_cv_fold_fit_equals_plain_fit_of_subset(lib):
    d = small_csc(4000, 8, seed=25, density=0.25, n_times=400)
    fold = synth.cv_folds(4000, 2, seed=26)
    r = binding.cox_cv_path(survdata(d), fold, 2, [2.0], penalty="l1", tol=1e-10, max_sweeps=200)
    for k in range(2):
        m = fold != k
        col_ptr, row_idx, values = synth.csc_from_dense(d["X_dense"][m])
        sub = {"time": d["time"][m], "status": d["status"][m], "col_ptr": col_ptr, "row_idx": row_idx,
               "values": values.astype(np.float32), "n": int(m.sum()), "p": 8, "layout": "csc"}
        b, info, _ = binding.cox_fit(survdata(sub), penalty="l1", lam=2.0, tol=0.0,
                                     max_sweeps=int(r["sweeps"][0, k]))
        np.testing.assert_allclose(r["beta"][0, k], b, rtol=0, atol=2e-6)


def test_cv_tuner_picks_a_candidate_and_is_reused(lib):
    d = small_csc(20000, 6, seed=33, density=0.2, n_times=500)
    fold = synth.cv_folds(20000, 5, seed=34)
    sd = survdata(d)
    ws = binding.Workspace()
    lam = [50.0, 5.0, 0.5]
    r = binding.cox_cv_path(sd, fold, 5, lam, penalty="l1", tol=1e-9, workspace=ws, flags=binding.SURV_FLAG_CV_TUNE)
    g, form, tile = r["info"]["ctas_per_fit"], r["info"]["row_pass_form"], r["info"]["tile_form"]
    assert g >= 1 and form in (1, 2) and tile in (0, 1, 2)
    r2 = binding.cox_cv_path(sd, fold, 5, lam, penalty="l1", tol=1e-9, workspace=ws)
    assert (r2["info"]["ctas_per_fit"], r2["info"]["row_pass_form"], r2["info"]["tile_form"]) == (g, form, tile)
    np.testing.assert_array_equal(r["beta"], r2["beta"])
    ref = oracle.cv_path(d["time"], d["status"], oracle_X(d), fold, 5, lam, "l1", sweeps=r["sweeps"])
    np.testing.assert_allclose(r["beta"], ref["beta"], rtol=0, atol=TOL_B["f32c"])


def test_cv_path_all_fits_stop_at_lambda_max(lib):
    d = small_csc(2000, 6, seed=27, density=0.3, n_times=100)
    fold = synth.cv_folds(2000, 5, seed=28)
    big = 1e6
    r = binding.cox_cv_path(survdata(d), fold, 5, [big], penalty="l1", tol=1e-8, max_sweeps=50)
    assert np.all(r["beta"] == 0.0)
    assert np.all(r["sweeps"] == 1)
    ref = oracle.cv_path(d["time"], d["status"], oracle_X(d), fold, 5, [big], "l1", sweeps=r["sweeps"])
    np.testing.assert_allclose(r["heldout"], ref["heldout"], rtol=1e-6)


@pytest.mark.parametrize("layout", ["csc", "dense"])
def test_lambda_max_matches_oracle(lib, layout):
    if layout == "csc":
        d = small_csc(5003, 9, seed=29, density=0.2, n_times=500)
    else:
        d = synth.cohort_small(4001, 7, seed=30, n_times=4001, censor_frac=0.3)
    pf = np.linspace(0.0, 2.0, oracle_X(d).shape[1])
    for f in (None, pf):
        got = binding.cox_lambda_max(survdata(d), penalty_factor=f)
        ref = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d), pf=f)
        assert got == pytest.approx(ref, rel=1e-11)


def test_cv_path_errors(lib):
    d = small_csc(500, 4, seed=31, density=0.3, n_times=50)
    sd = survdata(d)
    fold = synth.cv_folds(500, 2, seed=32)
    with pytest.raises(binding.SurvError) as e:
        binding.cox_cv_path(sd, fold, 0, [1.0])
    assert e.value.code == binding.SURV_E_INVALID
    bad = fold.copy()
    bad[7] = 5
    with pytest.raises(binding.SurvError) as e:
        binding.cox_cv_path(sd, bad, 2, [1.0])
    assert e.value.code == binding.SURV_E_INVALID
    # fold 0 holds every event: its training part has none
    ev = np.where(d["status"] == 1, 0, 1).astype(np.int8)
    with pytest.raises(binding.SurvError) as e:
        binding.cox_cv_path(sd, ev, 2, [1.0])
    assert e.value.code == binding.SURV_E_NO_EVENTS
    with pytest.raises(binding.SurvError) as e:
        binding.cox_cv_path(sd, fold, 2, [-1.0])
    assert e.value.code == binding.SURV_E_INVALID


# ------------------------------------------------------ benchmarked size
def test_cv_path_full_size_sampled(lib):
    """N = 10^6, p = 500 binary covariates at 1 %, ~40 % censoring, 10 uneven
    folds x 20 L1 strengths from lambda_max down to 1e-3 lambda_max."""
    d = synth.cohort_cox_sparse(1_000_000, 500, seed=41, density=0.01, n_true=10, laplace_scale=0.2,
                                censor_frac=0.4, grid=3650)
    fold = synth.cv_folds(1_000_000, 10, seed=42)
    sd = survdata(d)
    lmax = binding.cox_lambda_max(sd)
    lam = synth.lambda_grid(lmax, 20)
    r = binding.cox_cv_path(sd, fold, 10, lam, penalty="l1", tol=1e-8, max_sweeps=100)
    info = r["info"]
    assert info["nfits"] == 200 and info["fits_converged"] == 200
    X = oracle_X(d)
    # the strongest penalty: lambda_max of the whole data may sit a little
    # below a training set's own, so only tiny entries may appear
    assert np.abs(r["beta"][0]).max() < 1e-2
    # one fit against the oracle's fit of the same training set, sweep for sweep
    li, k = 10, 3
    m = fold != k
    Xt = X[np.flatnonzero(m)]
    ref = oracle.ccd_fit("cox", d["time"][m], d["status"][m], Xt, "l1", lam[li], tol=0.0,
                         max_sweeps=int(r["sweeps"][li, k]))
    np.testing.assert_allclose(r["beta"][li, k], ref["beta"], rtol=0, atol=1e-5)
    # held-out scores of sampled fits
    for li, k in [(0, 0), (10, 3), (19, 7)]:
        h = oracle.heldout_loglik(d["time"], d["status"], X, r["beta"][li, k], fold == k)
        assert r["heldout"][li, k] == pytest.approx(h, rel=1e-6)
