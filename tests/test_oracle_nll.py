"""Pins of the FP64 oracle for the differentiable form (oracle/nll.py):
each check compares it with something other than itself."""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import synth


def _cohort(n, p, C, seed, n_times):
    rng = np.random.default_rng(seed)
    d = synth.cohort_small(n, p, seed, n_times=n_times, censor_frac=0.3)
    B = rng.normal(0.0, 0.3, size=(p, C))
    return d["time"], d["status"], np.asarray(d["X"]), B


def test_nll_is_minus_cox_loglik_per_column():
    # independent code: oracle.cox_terms computes l from X and beta
    t, s, X, B = _cohort(400, 5, 4, seed=1, n_times=60)
    nll = oracle.cox_nll(t, s, X @ B)
    for b in range(B.shape[1]):
        l, _, _ = oracle.cox_terms(t, s, X, B[:, b], 0)
        assert nll[b] == pytest.approx(-l, rel=1e-12)


def test_grad_B_is_minus_cox_score():
    t, s, X, B = _cohort(300, 4, 3, seed=2, n_times=40)
    g = oracle.cox_nll_grad_B(X, t, s, B)
    for b in range(B.shape[1]):
        for j in range(X.shape[1]):
            _, score, _ = oracle.cox_terms(t, s, X, B[:, b], j)
            assert g[j, b] == pytest.approx(-score, rel=1e-10, abs=1e-10)


def test_grad_B_central_differences():
    t, s, X, B = _cohort(250, 3, 2, seed=3, n_times=30)
    g = oracle.cox_nll_grad_B(X, t, s, B)
    h = 1e-5
    for j in range(3):
        for b in range(2):
            Bp, Bm = B.copy(), B.copy()
            Bp[j, b] += h
            Bm[j, b] -= h
            fd = (oracle.cox_nll(t, s, X @ Bp)[b] - oracle.cox_nll(t, s, X @ Bm)[b]) / (2 * h)
            assert g[j, b] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_nll_brute_force_risk_sets():
    rng = np.random.default_rng(4)
    n = 120
    time = rng.integers(1, 15, size=n).astype(np.int32)   # heavy ties
    status = (rng.random(n) < 0.6).astype(np.int8)
    eta = rng.normal(0, 0.8, size=n)
    brute = oracle.cox_nll_brute(time, status, eta)       # any order
    perm = oracle.sort_desc(time)
    scan = oracle.cox_nll(time[perm], status[perm], eta[perm])[0]
    assert scan == pytest.approx(brute, rel=1e-12)


def test_grad_eta_sums_to_zero_and_shift_invariance():
    t, s, X, B = _cohort(500, 4, 3, seed=5, n_times=70)
    eta = X @ B
    ge = oracle.cox_nll_grad_eta(t, s, eta)
    np.testing.assert_allclose(ge.sum(axis=0), 0.0, atol=1e-10)
    np.testing.assert_allclose(oracle.cox_nll(t, s, eta + 3.7), oracle.cox_nll(t, s, eta), rtol=1e-12)
