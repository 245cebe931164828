"""Pins of the cross-validation oracle (oracle/cv.py) to facts outside its
own formulas (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import synth


def _cohort(seed, n=150, p=4, n_times=25):
    return synth.cohort_small(n, p, seed, n_times=n_times, censor_frac=0.3)


def test_heldout_equals_bruteforce_risk_sets():
    d = _cohort(3)
    fold = synth.cv_folds(d["time"].shape[0], 3, seed=4)
    beta = np.array([0.3, -0.2, 0.1, 0.0])
    for k in range(3):
        m = fold == k
        eta = d["X"][m] @ beta
        ref = -oracle.cox_nll_brute(d["time"][m], d["status"][m], eta)
        assert oracle.heldout_loglik(d["time"], d["status"], d["X"], beta, m) == pytest.approx(ref, rel=1e-12)


def test_heldout_without_events_is_zero():
    d = _cohort(5, n=40)
    m = d["status"] != 1
    assert oracle.heldout_loglik(d["time"], d["status"], d["X"], np.ones(4), m) == 0.0


def test_above_lambda_max_fit_is_zero_and_score_is_null_model():
    d = _cohort(7)
    n = d["time"].shape[0]
    fold = synth.cv_folds(n, 2, seed=8)
    lmax = max(oracle.lambda_max("cox", d["time"][fold != k], d["status"][fold != k], d["X"][fold != k])
               for k in range(2))
    r = oracle.cv_path(d["time"], d["status"], d["X"], fold, 2, [1.01 * lmax], "l1", tol=1e-12)
    assert np.all(r["beta"] == 0.0)
    for k in range(2):
        m = fold == k
        t, s = d["time"][m], d["status"][m]
        # null model: each event contributes -log(number of fold subjects with time >= its time)
        ref = -sum(math.log(np.sum(t >= t[i])) for i in np.flatnonzero(s == 1))
        assert r["heldout"][0, k] == pytest.approx(ref, rel=1e-12)


def test_relabelling_folds_permutes_results():
    d = _cohort(9, n=120)
    n = d["time"].shape[0]
    fold = synth.cv_folds(n, 3, seed=10)
    perm = np.array([2, 0, 1], dtype=np.int8)  # fold k -> perm[k]
    lam = [5.0, 1.0]
    a = oracle.cv_path(d["time"], d["status"], d["X"], fold, 3, lam, "l1", tol=1e-10)
    b = oracle.cv_path(d["time"], d["status"], d["X"], perm[fold], 3, lam, "l1", tol=1e-10)
    for k in range(3):
        np.testing.assert_array_equal(a["beta"][:, k], b["beta"][:, perm[k]])
        np.testing.assert_array_equal(a["heldout"][:, k], b["heldout"][:, perm[k]])


def test_cv_mean_and_best_follow_definitions():
    d = _cohort(11, n=160)
    n = d["time"].shape[0]
    fold = synth.cv_folds(n, 4, seed=12)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], d["X"])
    lam = synth.lambda_grid(lmax, 4, ratio=1e-2)
    r = oracle.cv_path(d["time"], d["status"], d["X"], fold, 4, lam, "l1", tol=1e-9)
    np.testing.assert_allclose(r["cv_mean"], r["heldout"].sum(axis=1) / 4, rtol=1e-15)
    assert r["best"] == int(np.flatnonzero(r["cv_mean"] == r["cv_mean"].max())[0])


def test_training_fit_is_the_plain_fit_of_the_subset():
    d = _cohort(13, n=100)
    n = d["time"].shape[0]
    fold = synth.cv_folds(n, 2, seed=14)
    r = oracle.cv_path(d["time"], d["status"], d["X"], fold, 2, [0.5], "l2", tol=1e-12)
    # the same fit from an explicitly re-sorted copy of the training subjects
    m = fold != 1
    t, s, X = d["time"][m], d["status"][m], d["X"][m]
    order = synth.arrange_desc(t)
    ref = oracle.ccd_fit("cox", t[order], s[order], X[order], "l2", 0.5, tol=1e-12)
    np.testing.assert_allclose(r["beta"][0, 1], ref["beta"], rtol=0, atol=1e-12)


def test_cv_folds_sizes_are_uneven_and_cover_everyone():
    f = synth.cv_folds(1000, 10, seed=1)
    sizes = np.bincount(f, minlength=10)
    assert sizes.sum() == 1000 and sizes.min() >= 75 and sizes.max() <= 125
    assert sizes.max() - sizes.min() >= 30
