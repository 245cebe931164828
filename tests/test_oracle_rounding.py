"""Rounding self-check of the oracle's O(N) scan form (not a pin of its
mathematics, which tests/test_oracle_pins.py covers): with the same inputs
e = exp(eta), x and the Fine-Gray weights, every sum of Section 2.7 taken
exactly (rational arithmetic) and rounded once agrees with the oracle's
plain left-to-right FP64 sums to a few units of N * eps.  The oracle is the
accuracy reference of the precision report, so its own rounding has to be
far below the errors that report states."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import synth


def _exact_terms(model, t, st, x, eta):
    """(l, g', g'') with every sum exact; exp, log and the Kaplan-Meier
    values are the oracle's FP64 numbers, taken as exact inputs."""
    n = t.shape[0]
    e = np.exp(eta)
    gend = oracle.tie_groups(t)
    d = oracle.group_counts(gend, st, 1)
    E = [Fraction(float(v)) for v in e]
    Xf = [Fraction(float(v)) for v in x]
    if model == "fg":
        W, Gk, _ = oracle.fg_weights(t, st)
        Wf = [Fraction(float(v)) for v in W]
        Gf = [Fraction(float(v)) for v in Gk]
    # prefix sums at group ends, exclusive suffix sums after them
    pre = [[Fraction(0)] * 3 for _ in range(len(gend))]
    run = [Fraction(0)] * 3
    k = 0
    for i in range(n):
        a = E[i]
        run = [run[0] + a, run[1] + a * Xf[i], run[2] + a * Xf[i] * Xf[i]]
        if k < len(gend) and i == gend[k]:
            pre[k] = run
            k += 1
    suf = [[Fraction(0)] * 3 for _ in range(len(gend))]
    if model == "fg":
        acc = [Fraction(0)] * 3
        k = len(gend) - 1
        for i in range(n - 1, -1, -1):
            while k >= 0 and gend[k] >= i:
                suf[k] = acc          # strictly after the end of group k
                k -= 1
            a = E[i] * Wf[i]
            acc = [acc[0] + a, acc[1] + a * Xf[i], acc[2] + a * Xf[i] * Xf[i]]
        while k >= 0:
            suf[k] = acc
            k -= 1
    g1 = sum((Xf[i] for i in range(n) if st[i] == 1), Fraction(0))
    g2 = Fraction(0)
    lin = sum((Fraction(float(eta[i])) for i in range(n) if st[i] == 1), Fraction(0))
    logs = []
    for k in range(len(gend)):
        den, n1, n2 = pre[k]
        if model == "fg":
            den, n1, n2 = den + Gf[k] * suf[k][0], n1 + Gf[k] * suf[k][1], n2 + Gf[k] * suf[k][2]
        if d[k] == 0:
            continue
        G, H = n1 / den, n2 / den
        g1 -= d[k] * G
        g2 -= d[k] * (H - G * G)
        logs.append(d[k] * math.log(float(den)))
    return float(lin) - math.fsum(logs), float(g1), float(g2)


@pytest.mark.parametrize("model", ["cox", "fg"])
def test_scan_sums_match_exact_sums(model):
    dd = synth.cohort_small(3000, 2, seed=71, n_times=60, censor_frac=0.3,
                            competing_frac=0.25 if model == "fg" else 0.0)
    t, st, X, beta = dd["time"], dd["status"], dd["X"], dd["beta"]
    eta = X @ beta
    for j in range(2):
        got = oracle.model_terms(model, t, st, X, beta, j, eta)
        ref = _exact_terms(model, t, st, X[:, j], eta)
        n = t.shape[0]
        eps = np.finfo(np.float64).eps
        assert got[0] == pytest.approx(ref[0], rel=4 * n * eps)
        # g' and g'' relative to the size of the sums they are differences of
        scale1 = abs(float(np.sum(np.abs(X[:, j])[st == 1]))) + 1.0
        assert abs(got[1] - ref[1]) <= 4 * n * eps * scale1
        assert abs(got[2] - ref[2]) <= 4 * n * eps * (abs(ref[2]) + scale1)
