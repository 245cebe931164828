"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties an oracle function to something it does not compute from
its own formula: a brute-force definition, a closed form derived by hand,
a textbook statistic computed by scipy, finite differences, an invariant,
or an independent optimiser.  A dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.sparse
import scipy.stats

import oracle
from paper_2204_08183_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(seed, n=60, p=4, n_times=12, competing=0.0, density=1.0):
    return synth.cohort_small(n, p, seed, n_times=n_times, censor_frac=0.3,
                              competing_frac=competing, density=density)


# ---------------------------------------------------------------- ordering
def test_sort_desc_matches_key_sort():
    rng = np.random.default_rng(0)
    for n in [0, 1, 2, 17, 300]:
        t = rng.integers(-5, 6, size=n).astype(np.int32)
        want = sorted(range(n), key=lambda i: (-int(t[i]), i))
        assert list(oracle.sort_desc(t)) == want


def test_tie_groups_hand_example():
    t = np.array([9, 7, 7, 5, 3, 3], dtype=np.int32)
    assert list(oracle.tie_groups(t)) == [0, 2, 3, 5]
    assert list(oracle.tie_groups(np.array([4], np.int32))) == [0]
    assert list(oracle.tie_groups(np.array([2, 2, 2], np.int32))) == [2]
    st = np.array([1, 0, 1, 0, 2, 0], np.int8)
    assert list(oracle.group_counts(oracle.tie_groups(t), st, 1)) == [1, 1, 0, 0]
    assert list(oracle.group_counts(oracle.tie_groups(t), st, 0)) == [0, 1, 1, 1]


# ---------------------------------------------------------------- Kaplan-Meier
def test_km_golden_six_subjects():
    g = json.load(open(os.path.join(GOLDEN, "km_censoring_6.json")))
    t = np.array(g["time"], np.int32)
    st = np.array(g["status"], np.int8)
    got = oracle.km_censoring_groups(t, st)
    np.testing.assert_allclose(got, g["G_at_group_times"], rtol=1e-15)
    for tk, gk in zip(g["group_times"], g["G_at_group_times"]):
        assert oracle.km_censoring_at(t, st, tk) == pytest.approx(gk, rel=1e-15)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_km_matches_scipy_ecdf(seed):
    d = _small(seed, n=200, n_times=25, competing=0.2)
    t, st = d["time"], d["status"]
    cens = st == 0
    sample = scipy.stats.CensoredData(uncensored=t[cens].astype(float),
                                      right=t[~cens].astype(float))
    sf = scipy.stats.ecdf(sample).sf
    gend = oracle.tie_groups(t)
    got = oracle.km_censoring_groups(t, st)
    want = sf.evaluate(t[gend].astype(float))
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_km_no_censoring_is_one():
    d = _small(4, n=50, n_times=10, competing=0.3)
    st = np.where(d["status"] == 0, 1, d["status"]).astype(np.int8)
    assert np.all(oracle.km_censoring_groups(d["time"], st) == 1.0)


# ---------------------------------------------------------------- closed forms
def test_cox_closed_form_two_subjects():
    t = np.array([2, 1], np.int32)
    st = np.array([0, 1], np.int8)
    x = np.array([[1.0], [-0.5]])
    b = 0.3
    e1, e2 = math.exp(b * 1.0), math.exp(b * -0.5)
    xbar = (e1 * 1.0 + e2 * -0.5) / (e1 + e2)
    x2bar = (e1 * 1.0 + e2 * 0.25) / (e1 + e2)
    want = (b * -0.5 - math.log(e1 + e2), -0.5 - xbar, -(x2bar - xbar ** 2))
    for f in (oracle.cox_terms, oracle.cox_terms_brute):
        got = f(t, st, x, [b], 0)
        np.testing.assert_allclose(got, want, rtol=1e-14)


def test_cox_closed_form_three_subjects_with_tie():
    # times 3, 2, 2 ; events at 3 and at the first 2; the tied censored
    # subject at 2 is in the risk set of the event at 2 (Breslow, Eq. cox_l).
    t = np.array([3, 2, 2], np.int32)
    st = np.array([1, 1, 0], np.int8)
    x = np.array([[0.2], [1.5], [-0.7]])
    b = -0.4
    e = np.exp(b * x[:, 0])
    s0, s1, s2 = e.sum(), (e * x[:, 0]).sum(), (e * x[:, 0] ** 2).sum()
    # event at 3: risk set {0}: contributes 0 to l, g', g''
    want = (b * 1.5 - math.log(s0), 1.5 - s1 / s0, -(s2 / s0 - (s1 / s0) ** 2))
    for f in (oracle.cox_terms, oracle.cox_terms_brute):
        np.testing.assert_allclose(f(t, st, x, [b], 0), want, rtol=1e-14, atol=1e-15)


def test_fg_golden_closed_form_four_subjects():
    g = json.load(open(os.path.join(GOLDEN, "fg_closed_form_4.json")))
    t = np.array(g["time"], np.int32)
    st = np.array(g["status"], np.int8)
    xv = np.array(g["x"])
    b = g["beta"]
    X = xv[:, None]
    e = np.exp(b * xv)
    den_a = e[0] + e[2] / 2
    num_a1 = e[0] * xv[0] + e[2] * xv[2] / 2
    num_a2 = e[0] * xv[0] ** 2 + e[2] * xv[2] ** 2 / 2
    den_b = e.sum()
    num_b1 = (e * xv).sum()
    num_b2 = (e * xv ** 2).sum()
    l = (b * xv[0] - math.log(den_a)) + (b * xv[3] - math.log(den_b))
    g1 = (xv[0] - num_a1 / den_a) + (xv[3] - num_b1 / den_b)
    g2 = -(num_a2 / den_a - (num_a1 / den_a) ** 2) - (num_b2 / den_b - (num_b1 / den_b) ** 2)
    for f in (oracle.fg_terms, oracle.fg_terms_brute):
        np.testing.assert_allclose(f(t, st, X, [b], 0), (l, g1, g2), rtol=1e-14)
    W, Gk, gend = oracle.fg_weights(t, st)
    np.testing.assert_allclose(Gk, [0.5, 0.5, 1.0, 1.0], rtol=0)
    np.testing.assert_allclose(W, [0, 0, 1.0, 0], rtol=0)


# ---------------------------------------------------------------- brute vs scan
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n_times", [3, 15, None])
def test_cox_scan_equals_brute(seed, n_times):
    d = _small(seed, n=80, p=3, n_times=n_times or 80)
    beta = d["beta"]
    for j in range(3):
        a = oracle.cox_terms(d["time"], d["status"], d["X"], beta, j)
        b = oracle.cox_terms_brute(d["time"], d["status"], d["X"], beta, j)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("n_times", [4, 20])
def test_fg_scan_equals_brute(seed, n_times):
    d = _small(seed, n=50, p=2, n_times=n_times, competing=0.3)
    beta = d["beta"]
    for j in range(2):
        a = oracle.fg_terms(d["time"], d["status"], d["X"], beta, j)
        b = oracle.fg_terms_brute(d["time"], d["status"], d["X"], beta, j)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_brute_is_order_free_and_scan_is_permutation_invariant():
    d = _small(11, n=70, p=2, n_times=9, competing=0.25)
    rng = np.random.default_rng(5)
    perm = rng.permutation(70)
    t, st, X = d["time"][perm], d["status"][perm], d["X"][perm]
    for model, brute, scan in [("cox", oracle.cox_terms_brute, oracle.cox_terms),
                               ("fg", oracle.fg_terms_brute, oracle.fg_terms)]:
        st_m = st if model == "fg" else np.where(st == 2, 0, st).astype(np.int8)
        s_m = d["status"] if model == "fg" else np.where(d["status"] == 2, 0, d["status"]).astype(np.int8)
        ref = scan(d["time"], s_m, d["X"], d["beta"], 1)
        np.testing.assert_allclose(brute(t, st_m, X, d["beta"], 1), ref, rtol=1e-12)
        order = oracle.sort_desc(t)
        np.testing.assert_allclose(scan(t[order], st_m[order], X[order], d["beta"], 1), ref, rtol=1e-12)


def test_sparse_and_dense_inputs_agree():
    d = _small(3, n=90, p=4, n_times=20, density=0.2)
    Xs = scipy.sparse.csc_matrix(d["X"])
    for j in range(4):
        np.testing.assert_allclose(oracle.cox_terms(d["time"], d["status"], Xs, d["beta"], j),
                                   oracle.cox_terms(d["time"], d["status"], d["X"], d["beta"], j),
                                   rtol=1e-13)


# ---------------------------------------------------------------- finite differences
@pytest.mark.parametrize("model", ["cox", "fg"])
def test_finite_differences(model):
    d = _small(21, n=120, p=3, n_times=30, competing=0.2 if model == "fg" else 0.0)
    f = oracle.cox_terms if model == "cox" else oracle.fg_terms
    beta = d["beta"]
    h = 1e-5
    for j in range(3):
        bp, bm = beta.copy(), beta.copy()
        bp[j] += h
        bm[j] -= h
        lp, gp, _ = f(d["time"], d["status"], d["X"], bp, j)
        lm, gm, _ = f(d["time"], d["status"], d["X"], bm, j)
        _, g1, g2 = f(d["time"], d["status"], d["X"], beta, j)
        assert (lp - lm) / (2 * h) == pytest.approx(g1, rel=1e-7, abs=1e-7)
        assert (gp - gm) / (2 * h) == pytest.approx(g2, rel=1e-6, abs=1e-7)


# ---------------------------------------------------------------- log-rank
def _logrank_counts(t, st, grp):
    """Textbook two-sample log-rank O - E and hypergeometric variance from
    the 2 x 2 table at each distinct event time."""
    O = E = V = 0.0
    for s in np.unique(t[st == 1]):
        at = t >= s
        n = at.sum()
        n1 = (at & grp).sum()
        d = ((t == s) & (st == 1)).sum()
        d1 = ((t == s) & (st == 1) & grp).sum()
        O += d1
        E += d * n1 / n
        if n > 1:
            V += d * (n1 / n) * (1 - n1 / n) * (n - d) / (n - 1)
    return O, E, V


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_score_at_zero_is_logrank_no_ties(seed):
    rng = np.random.default_rng(seed)
    n = 150
    t = rng.permutation(n).astype(np.int32) + 1      # distinct times
    st = (rng.random(n) > 0.3).astype(np.int8)
    grp = rng.random(n) < 0.45
    order = oracle.sort_desc(t)
    t, st, grp = t[order], st[order], grp[order]
    X = grp.astype(float)[:, None]
    _, g1, g2 = oracle.cox_terms(t, st, X, [0.0], 0)
    res = scipy.stats.logrank(
        scipy.stats.CensoredData(uncensored=t[grp & (st == 1)].astype(float),
                                 right=t[grp & (st == 0)].astype(float)),
        scipy.stats.CensoredData(uncensored=t[~grp & (st == 1)].astype(float),
                                 right=t[~grp & (st == 0)].astype(float)))
    # without ties the Breslow information equals the log-rank variance
    z = g1 / math.sqrt(-g2)
    assert abs(z) == pytest.approx(abs(res.statistic), rel=1e-10)
    O, E, V = _logrank_counts(t, st, grp)
    assert g1 == pytest.approx(O - E, rel=1e-12, abs=1e-12)
    assert -g2 == pytest.approx(V, rel=1e-12)


@pytest.mark.parametrize("seed", [3, 4])
def test_score_at_zero_is_logrank_with_ties(seed):
    rng = np.random.default_rng(seed)
    n = 200
    t = rng.integers(1, 15, size=n).astype(np.int32)
    st = (rng.random(n) > 0.3).astype(np.int8)
    grp = rng.random(n) < 0.5
    order = oracle.sort_desc(t)
    t, st, grp = t[order], st[order], grp[order]
    X = grp.astype(float)[:, None]
    _, g1, g2 = oracle.cox_terms(t, st, X, [0.0], 0)
    O, E, V = _logrank_counts(t, st, grp)
    res = scipy.stats.logrank(
        scipy.stats.CensoredData(uncensored=t[grp & (st == 1)].astype(float),
                                 right=t[grp & (st == 0)].astype(float)),
        scipy.stats.CensoredData(uncensored=t[~grp & (st == 1)].astype(float),
                                 right=t[~grp & (st == 0)].astype(float)))
    assert abs((O - E) / math.sqrt(V)) == pytest.approx(abs(res.statistic), rel=1e-10)
    # the score is O - E exactly, ties included
    assert g1 == pytest.approx(O - E, rel=1e-12, abs=1e-12)
    # Breslow information omits the hypergeometric factor (n-d)/(n-1) <= 1
    info_breslow = 0.0
    for s in np.unique(t[st == 1]):
        at = t >= s
        nn, n1 = at.sum(), (at & grp).sum()
        d = ((t == s) & (st == 1)).sum()
        info_breslow += d * (n1 / nn) * (1 - n1 / nn)
    assert -g2 == pytest.approx(info_breslow, rel=1e-12)
    assert -g2 > V


# ---------------------------------------------------------------- invariants
def test_fine_gray_without_competing_is_cox():
    d = _small(7, n=100, p=3, n_times=20, competing=0.0)
    for j in range(3):
        assert oracle.fg_terms(d["time"], d["status"], d["X"], d["beta"], j) == \
            oracle.cox_terms(d["time"], d["status"], d["X"], d["beta"], j)


def test_fine_gray_late_competing_is_cox_with_censoring():
    d = _small(8, n=100, p=2, n_times=30, competing=0.0)
    t, st = d["time"].copy(), d["status"].copy()
    # make every subject at or above the largest primary time a competing event
    last_primary = t[st == 1].max()
    st[(t >= last_primary) & (st == 0)] = 2
    assert (st == 2).any()
    st_cox = np.where(st == 2, 0, st).astype(np.int8)
    for j in range(2):
        np.testing.assert_allclose(oracle.fg_terms(t, st, d["X"], d["beta"], j),
                                   oracle.cox_terms(t, st_cox, d["X"], d["beta"], j), rtol=1e-13)


@pytest.mark.parametrize("model", ["cox", "fg"])
def test_shift_invariance(model):
    d = _small(9, n=90, p=2, n_times=12, competing=0.2 if model == "fg" else 0.0)
    f = oracle.cox_terms if model == "cox" else oracle.fg_terms
    eta = oracle.linear_predictor(d["X"], d["beta"])
    a = f(d["time"], d["status"], d["X"], d["beta"], 1, eta)
    b = f(d["time"], d["status"], d["X"], d["beta"], 1, eta + 3.7)
    np.testing.assert_allclose(a, b, rtol=1e-12)


# ---------------------------------------------------------------- CCD step
def test_newton_step_cases():
    # no penalty: -g'/g''
    assert oracle.newton_step(0.0, 3.0, -2.0, "none", 0.0) == 1.5
    # L2: (g' - lam b)/(h + lam)
    assert oracle.newton_step(0.5, 3.0, -2.0, "l2", 1.0) == pytest.approx((3.0 - 0.5) / 3.0)
    # L1 at zero: inside the dead zone -> 0, outside -> shrunk step
    assert oracle.newton_step(0.0, 0.9, -2.0, "l1", 1.0) == 0.0
    assert oracle.newton_step(0.0, -0.9, -2.0, "l1", 1.0) == 0.0
    assert oracle.newton_step(0.0, 5.0, -2.0, "l1", 1.0) == 2.0
    assert oracle.newton_step(0.0, -5.0, -2.0, "l1", 1.0) == -2.0
    # L1 nonzero: (g' - gamma sgn b)/h, stop at zero when crossing
    assert oracle.newton_step(1.0, 3.0, -2.0, "l1", 1.0) == 1.0
    assert oracle.newton_step(0.2, -3.0, -2.0, "l1", 1.0) == -0.2
    assert oracle.newton_step(-0.2, 3.0, -2.0, "l1", 1.0) == 0.2
    # no curvature: no step
    assert oracle.newton_step(0.0, 3.0, 0.0, "none", 0.0) == 0.0


def test_trust_region_cases():
    assert oracle.trust_region(2.0, 1.0) == (1.0, 2.0)
    assert oracle.trust_region(-0.1, 1.0) == (-0.1, 0.5)
    assert oracle.trust_region(0.0, 1.0) == (0.0, 0.5)
    assert oracle.trust_region(-3.0, 0.25) == (-0.25, 0.5)


# ---------------------------------------------------------------- CCD optimum
def _neg_obj(model, d, penalty, lam):
    def f(b):
        l, _, _ = oracle.model_terms(model, d["time"], d["status"], d["X"], b, 0)
        return -(l + oracle.penalty_value(b, penalty, lam))
    return f


@pytest.mark.parametrize("model", ["cox", "fg"])
def test_ccd_l2_matches_scipy_and_kkt(model):
    d = _small(13, n=150, p=4, n_times=25, competing=0.25 if model == "fg" else 0.0)
    lam = 2.0
    # tol = 0: run a fixed number of sweeps, far past convergence
    fit = oracle.ccd_fit(model, d["time"], d["status"], d["X"], "l2", lam, tol=0.0, max_sweeps=150)
    b = fit["beta"]
    for j in range(4):
        _, g1, _ = oracle.model_terms(model, d["time"], d["status"], d["X"], b, j)
        assert g1 == pytest.approx(lam * b[j], abs=1e-9)
    ref = scipy.optimize.minimize(_neg_obj(model, d, "l2", lam), np.zeros(4), method="BFGS",
                                  options={"gtol": 1e-9})
    np.testing.assert_allclose(b, ref.x, atol=1e-5)


def test_ccd_l1_kkt_and_split_variable_solution():
    d = _small(17, n=200, p=5, n_times=30)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], d["X"])
    gam = 0.8 * lmax
    fit = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "l1", gam, tol=0.0, max_sweeps=200)
    b = fit["beta"]
    assert (b == 0).any() and (b != 0).any()
    for j in range(5):
        _, g1, _ = oracle.cox_terms(d["time"], d["status"], d["X"], b, j)
        if b[j] == 0.0:
            assert abs(g1) <= gam * (1 + 1e-9)
        else:
            assert g1 == pytest.approx(gam * np.sign(b[j]), rel=1e-6)

    def obj(uv):
        bb = uv[:5] - uv[5:]
        l, _, _ = oracle.cox_terms(d["time"], d["status"], d["X"], bb, 0)
        return -l + gam * uv.sum()
    ref = scipy.optimize.minimize(obj, np.full(10, 0.01), method="L-BFGS-B",
                                  bounds=[(0, None)] * 10, options={"ftol": 1e-15, "gtol": 1e-10})
    np.testing.assert_allclose(b, ref.x[:5] - ref.x[5:], atol=2e-4)


def test_lambda_max_zeroes_the_fit():
    d = _small(19, n=120, p=4, n_times=20)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], d["X"])
    fit = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "l1", lmax * 1.0001, tol=1e-12)
    assert np.all(fit["beta"] == 0.0)
    fit = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "l1", lmax * 0.9, tol=1e-12)
    assert np.any(fit["beta"] != 0.0)


def test_ccd_recovers_truth_roughly():
    d = synth.cohort_cox_dense(4000, 4, seed=5, n_true=2, beta_sd=0.7, grid=365)
    fit = oracle.ccd_fit("cox", d["time"], d["status"], d["X"], "none", 0.0, tol=1e-10)
    np.testing.assert_allclose(fit["beta"], d["beta_true"], atol=0.12)
