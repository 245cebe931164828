"""FP64 CPU oracle: Cox (Breslow ties) and Fine-Gray partial likelihoods,
their per-coordinate gradient and Hessian, and penalised cyclic coordinate
descent, written from the paper's Sections 2.1-2.4 and 2.7.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (CPU-baseline leg and ``--impl reference``).  The CUDA path
never imports it and it never imports the CUDA path.

Conventions (the readings of the paper that the oracle fixes):

* Subjects are arranged by observed time in decreasing order (Section 2.7,
  the loading matrix M becomes lower triangular).  Ties keep input order
  (a stable sort); the paper is silent on the tie-break.
* Ties use the Breslow form: every subject with y_r >= Y_i is at risk at
  Y_i (risk set R_1 of Eq. cox_l), so a prefix sum is read at the END of a
  run of tied times ("tie group").
* Fine-Gray (Eq. fg_l): R(Y_i) = R_1(Y_i) plus the competing-event subjects
  with y_r < Y_i; the IPCW weight is w_r(t) = I(C_r >= min(T_r, t)) G(t) /
  G(min(Y_r, t)) with G the Kaplan-Meier estimate of the censoring survival
  function, right-continuous: G(t) = prod_{s <= t} (1 - c_s / n_s),
  c_s = number censored at s, n_s = #{y >= s}.
* Penalties (Section 2.3): L1 pi = -sum_j gamma_j |beta_j| with
  gamma_j = lambda * pf_j; L2 pi = -sum_j beta_j^2 / (2 tau_j) with
  1 / tau_j = lambda * pf_j.
* CCD (Section 2.4): Newton step on g = l + pi, trust-region clip to
  Delta_j, width update Delta_j <- max(2 |applied step|, Delta_j / 2),
  Delta_j^(0) = 1.  At beta_j = 0 with L1 the two directional derivatives
  decide the direction; a step that would carry a nonzero beta_j across 0
  stops at 0.  Convergence: |f_k - f_{k-1}| / |f_k| < tol after a sweep,
  f = l + pi.

Parity pins (tests/test_oracle_*.py): brute-force O(N^2) risk sets vs the
O(N) scan form, central finite differences, closed forms for N = 2, 3, 4,
scipy's log-rank statistic for the score at beta = 0, scipy's Kaplan-Meier
for G, Fine-Gray == Cox without competing events, shift and permutation
invariance, KKT conditions at the CCD optimum and an independent
scipy.optimize solution of the penalised problem.  No function here is
parity-unpinned.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "sort_desc",
    "tie_groups",
    "group_counts",
    "km_censoring_groups",
    "km_censoring_at",
    "column",
    "linear_predictor",
    "cox_terms",
    "cox_terms_brute",
    "fg_weights",
    "fg_terms",
    "fg_terms_brute",
    "model_terms",
    "penalty_value",
    "newton_step",
    "trust_region",
    "ccd_fit",
    "lambda_max",
]


# --------------------------------------------------------------------------
# Ordering and tie groups (Section 2.7: observations in decreasing time)
# --------------------------------------------------------------------------
def sort_desc(time):
    """Permutation arranging subjects by decreasing observed time.

    Section 2.7 (the loading matrix M is lower triangular once the
    observations are arranged by decreasing Y_i).  Ties keep their input
    order (stable), so perm is unique.
    """
    time = np.asarray(time)
    idx = np.arange(time.shape[0])
    # lexsort sorts by the last key first: primary key -time, then index.
    return np.lexsort((idx, -time.astype(np.int64)))


def tie_groups(time_sorted):
    """End positions e_k of the maximal runs of equal time (Breslow groups).

    With times in decreasing order, {r : y_r >= y_i} is exactly the prefix
    0..e_k of the group k that holds i (Eq. cox_l's R_1 under ties).
    """
    t = np.asarray(time_sorted)
    n = t.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    is_end = np.ones(n, dtype=bool)
    is_end[:-1] = t[:-1] != t[1:]
    return np.flatnonzero(is_end).astype(np.int64)


def group_counts(gend, status_sorted, code):
    """Number of subjects with status == code in each tie group."""
    s = (np.asarray(status_sorted) == code).astype(np.int64)
    c = np.cumsum(s)
    at_end = c[gend]
    prev = np.concatenate(([0], at_end[:-1]))
    return at_end - prev


def km_censoring_groups(time_sorted, status_sorted, gend=None):
    """Kaplan-Meier censoring survival G(t_k) at every tie-group time.

    Section 2.2: G(t) = Pr(C > t), estimated by Kaplan-Meier with the
    censored subjects (status 0) as the "events":
    G(t_k) = prod over groups k' with t_k' <= t_k of (1 - c_k' / n_k'),
    where n_k' = #{y >= t_k'} = e_k' + 1 in decreasing order.
    The product runs from the smallest time upward.
    """
    if gend is None:
        gend = tie_groups(time_sorted)
    c = group_counts(gend, status_sorted, 0).astype(np.float64)
    n_risk = (gend + 1).astype(np.float64)
    factor = 1.0 - c / n_risk
    # groups with t <= t_k are k' >= k: cumulative product from the end
    return np.cumprod(factor[::-1])[::-1]


def km_censoring_at(time, status, t):
    """G(t) from its definition, for arbitrary (unsorted) data: a loop over
    the distinct observed times s <= t (Section 2.2)."""
    time = np.asarray(time)
    status = np.asarray(status)
    g = 1.0
    for s in np.unique(time):
        if s > t:
            break
        c_s = np.count_nonzero((time == s) & (status == 0))
        n_s = np.count_nonzero(time >= s)
        g *= 1.0 - c_s / n_s
    return g


# --------------------------------------------------------------------------
# Design matrix access
# --------------------------------------------------------------------------
def column(X, j):
    """Column j of X as a dense float64 vector.  X is a 2-D ndarray
    (subjects x covariates) or a scipy.sparse matrix."""
    if hasattr(X, "tocsc"):
        return np.asarray(X[:, [j]].toarray(), dtype=np.float64).ravel()
    return np.asarray(X[:, j], dtype=np.float64)


def linear_predictor(X, beta):
    """eta = X beta in float64."""
    beta = np.asarray(beta, dtype=np.float64)
    if hasattr(X, "tocsc"):
        return np.asarray(X.astype(np.float64) @ beta, dtype=np.float64).ravel()
    return np.asarray(X, dtype=np.float64) @ beta


# --------------------------------------------------------------------------
# Cox: Eq. cox_l and its coordinate derivatives (Eqs. cox_g, cox_h)
# --------------------------------------------------------------------------
def cox_terms_brute(time, status, X, beta, j):
    """(l, g', g'') for coordinate j straight from Eq. cox_l: an explicit
    risk set R_1(Y_i) = {r : y_r >= Y_i} per event.  O(N^2); any order.

    g'  = sum_i delta_i [x_ij - sum_R e_r x_rj / sum_R e_r]
    g'' = -sum_i delta_i [sum_R e_r x_rj^2 / sum_R e_r - (sum_R e x / sum_R e)^2]
    """
    time = np.asarray(time)
    status = np.asarray(status)
    eta = linear_predictor(X, beta)
    x = column(X, j)
    e = np.exp(eta)
    l = g1 = g2 = 0.0
    for i in range(time.shape[0]):
        if status[i] != 1:
            continue
        risk = time >= time[i]
        s0 = e[risk].sum()
        s1 = (e[risk] * x[risk]).sum()
        s2 = (e[risk] * x[risk] ** 2).sum()
        l += eta[i] - math.log(s0)
        g1 += x[i] - s1 / s0
        g2 -= s2 / s0 - (s1 / s0) ** 2
    return l, g1, g2


def cox_terms(time_sorted, status_sorted, X, beta, j, eta=None):
    """(l, g', g'') for coordinate j by prefix sums (Section 2.7).

    Step 1: e = exp(X beta) and the tuple (e, e x_j, e x_j^2).
    Step 2: prefix sums S_pre of the tuple (subjects in decreasing time).
    Step 3: G = S_pre[e x] / S_pre[e], H = S_pre[e x^2] / S_pre[e], read at
            each tie-group end (Breslow).
    Step 4: g' = delta^T X_j - delta^T G (Eq. cox_g),
            g'' = -delta^T (H - G * G) (Eq. cox_h),
            l = delta^T X beta - delta^T log S_pre[e] (Eq. cox_l rewritten).
    """
    status_sorted = np.asarray(status_sorted)
    if eta is None:
        eta = linear_predictor(X, beta)
    x = column(X, j)
    delta = (status_sorted == 1).astype(np.float64)
    gend = tie_groups(time_sorted)
    d = group_counts(gend, status_sorted, 1).astype(np.float64)
    e = np.exp(eta)
    s0 = np.cumsum(e)[gend]
    s1 = np.cumsum(e * x)[gend]
    s2 = np.cumsum(e * x * x)[gend]
    G = s1 / s0
    H = s2 / s0
    g1 = delta @ x - d @ G
    g2 = -(d @ (H - G * G))
    l = delta @ eta - d @ np.log(s0)
    return float(l), float(g1), float(g2)


# --------------------------------------------------------------------------
# Fine-Gray: Eq. fg_l and Eqs. fg_g, fg_h
# --------------------------------------------------------------------------
def fg_terms_brute(time, status, X, beta, j):
    """(l, g', g'') for coordinate j straight from Eq. fg_l.

    For each primary event i (status 1) at t = Y_i the risk set is
    R(t) = {r : y_r >= t} U {r : y_r < t, status_r != 1}, and the weight is
    w_r(t) = I(C_r >= min(T_r, t)) G(t) / G(min(Y_r, t)).  On observed data
    the indicator is I(y_r >= t) for a censored r (C_r = y_r < T_r) and 1
    for an event r (T_r = y_r <= C_r).  G is the Kaplan-Meier censoring
    survival (km_censoring_at).  O(N^2) with a G evaluation per pair; tiny N.
    """
    time = np.asarray(time)
    status = np.asarray(status)
    eta = linear_predictor(X, beta)
    x = column(X, j)
    e = np.exp(eta)
    G_at = {}

    def G(t):
        if t not in G_at:
            G_at[t] = km_censoring_at(time, status, t)
        return G_at[t]

    l = g1 = g2 = 0.0
    n = time.shape[0]
    for i in range(n):
        if status[i] != 1:
            continue
        t = time[i]
        s0 = s1 = s2 = 0.0
        for r in range(n):
            in_R = time[r] >= t or (time[r] < t and status[r] != 1)
            if not in_R:
                continue
            indicator = (time[r] >= t) if status[r] == 0 else True
            if not indicator:
                continue
            w = G(t) / G(min(time[r], t))
            s0 += w * e[r]
            s1 += w * e[r] * x[r]
            s2 += w * e[r] * x[r] ** 2
        l += eta[i] - math.log(s0)
        g1 += x[i] - s1 / s0
        g2 -= s2 / s0 - (s1 / s0) ** 2
    return l, g1, g2


def fg_weights(time_sorted, status_sorted):
    """Per-subject competing-risk weight W_r = I(status_r = 2) / G(y_r) and
    the group values G(t_k) (Section 2.7, the vector W; the factor G(t) of
    w_r(t) is applied per tie group)."""
    status_sorted = np.asarray(status_sorted)
    gend = tie_groups(time_sorted)
    Gk = km_censoring_groups(time_sorted, status_sorted, gend)
    # group index of every position: number of group ends strictly before it
    n = len(status_sorted)
    gid = np.searchsorted(gend, np.arange(n), side="left")
    with np.errstate(divide="ignore"):   # G = 0 only in a group with no competing event
        W = np.where(status_sorted == 2, 1.0 / Gk[gid], 0.0)
    return W, Gk, gend


def fg_terms(time_sorted, status_sorted, X, beta, j, eta=None):
    """(l, g', g'') for coordinate j by a forward and a backward scan
    (Section 2.7, Eqs. fg_g, fg_h).

    Numerators and denominators are S_pre[.] (risk set R_1, read at each
    group end) plus G(t_k) times S_suf[. * W] taken strictly after the
    group end (R_2: competing events with y_r < t_k).  delta = I(status=1).
    """
    status_sorted = np.asarray(status_sorted)
    if eta is None:
        eta = linear_predictor(X, beta)
    x = column(X, j)
    W, Gk, gend = fg_weights(time_sorted, status_sorted)
    delta = (status_sorted == 1).astype(np.float64)
    d = group_counts(gend, status_sorted, 1).astype(np.float64)
    e = np.exp(eta)

    def S_pre(v):
        return np.cumsum(v)[gend]

    def S_suf_after(v):
        suf = np.cumsum(v[::-1])[::-1]
        suf = np.append(suf, 0.0)
        return suf[gend + 1]

    den = S_pre(e) + Gk * S_suf_after(e * W)
    num1 = S_pre(e * x) + Gk * S_suf_after(e * x * W)
    num2 = S_pre(e * x * x) + Gk * S_suf_after(e * x * x * W)
    G = num1 / den
    H = num2 / den
    g1 = delta @ x - d @ G
    g2 = -(d @ (H - G * G))
    l = delta @ eta - d @ np.log(den)
    return float(l), float(g1), float(g2)


def model_terms(model, time_sorted, status_sorted, X, beta, j, eta=None):
    """Dispatch to cox_terms ("cox") or fg_terms ("fg")."""
    if model == "cox":
        return cox_terms(time_sorted, status_sorted, X, beta, j, eta)
    if model == "fg":
        return fg_terms(time_sorted, status_sorted, X, beta, j, eta)
    raise ValueError(model)


# --------------------------------------------------------------------------
# Penalties and the CCD step (Sections 2.3, 2.4)
# --------------------------------------------------------------------------
def _pf(pf, p):
    return np.ones(p) if pf is None else np.asarray(pf, dtype=np.float64)


def penalty_value(beta, penalty, lam, pf=None):
    """pi(beta) of Section 2.3 (a non-positive number)."""
    beta = np.asarray(beta, dtype=np.float64)
    w = lam * _pf(pf, beta.shape[0])
    if penalty == "none":
        return 0.0
    if penalty == "l1":
        return float(-(w * np.abs(beta)).sum())
    if penalty == "l2":
        return float(-(w * beta * beta).sum() / 2.0)
    raise ValueError(penalty)


def newton_step(beta_j, grad, hess, penalty, lam_j):
    """Newton step Delta beta_j = -g'(beta_j) / g''(beta_j) on the penalised
    g = l + pi (Section 2.4), before the trust-region clip.

    grad, hess are the log-likelihood derivatives l', l''.  With L1 at
    beta_j = 0 the forward (+) and backward (-) directional derivatives
    l' - gamma and -l' - gamma decide: move only along an ascent direction
    of g.  With L1 at beta_j != 0 a step that crosses zero stops at zero.
    A non-negative l'' (no curvature) gives no step.
    """
    h = -hess
    if not h > 0.0:
        return 0.0
    if penalty == "none":
        return grad / h
    if penalty == "l2":
        return (grad - lam_j * beta_j) / (h + lam_j)
    if penalty == "l1":
        if beta_j == 0.0:
            if grad > lam_j:
                return (grad - lam_j) / h
            if grad < -lam_j:
                return (grad + lam_j) / h
            return 0.0
        s = 1.0 if beta_j > 0.0 else -1.0
        step = (grad - lam_j * s) / h
        new = beta_j + step
        if not ((new > 0.0) if s > 0.0 else (new < 0.0)):
            step = -beta_j
        return step
    raise ValueError(penalty)


def trust_region(step, width):
    """Clip to the half-width Delta_j and update it (Section 2.4):
    applied = sgn(step) min(|step|, Delta_j);
    Delta_j <- max(2 |applied|, Delta_j / 2)."""
    applied = math.copysign(min(abs(step), width), step) if step != 0.0 else 0.0
    return applied, max(2.0 * abs(applied), width / 2.0)


def ccd_fit(model, time_sorted, status_sorted, X, penalty="none", lam=0.0,
            pf=None, tol=1e-8, max_sweeps=100, beta0=None, width0=None):
    """Penalised cyclic coordinate descent (Section 2.4), one Newton step per
    coordinate j = 0..p-1 per sweep, eta kept up to date after every
    nonzero step (Section 2.7, step 1).  Stops when the relative change of
    f = l + pi over a sweep is below tol, or after max_sweeps sweeps.

    Returns a dict with beta, sweeps, loglik, objective, converged, width.
    """
    p = X.shape[1]
    w = lam * _pf(pf, p)
    beta = np.zeros(p) if beta0 is None else np.array(beta0, dtype=np.float64)
    width = np.ones(p) if width0 is None else np.array(width0, dtype=np.float64)
    eta = linear_predictor(X, beta)

    def objective():
        l, _, _ = model_terms(model, time_sorted, status_sorted, X, beta, 0, eta)
        return l, l + penalty_value(beta, penalty, lam, pf)

    l, f_prev = objective()
    history = [f_prev]
    converged = False
    sweeps = 0
    while sweeps < max_sweeps:
        for j in range(p):
            _, g1, g2 = model_terms(model, time_sorted, status_sorted, X, beta, j, eta)
            step = newton_step(beta[j], g1, g2, penalty, w[j])
            applied, width[j] = trust_region(step, width[j])
            if applied != 0.0:
                beta[j] += applied
                eta = eta + applied * column(X, j)
        sweeps += 1
        l, f = objective()
        history.append(f)
        if abs(f - f_prev) / abs(f) < tol:
            converged = True
            break
        f_prev = f
    return {"beta": beta, "sweeps": sweeps, "loglik": l, "objective": history[-1],
            "converged": converged, "width": width, "history": history}


def lambda_max(model, time_sorted, status_sorted, X, pf=None):
    """Smallest L1 gamma whose penalised optimum is beta = 0:
    max_j |l'_j(0)| / pf_j over penalised j (the KKT condition at 0)."""
    p = X.shape[1]
    pf = _pf(pf, p)
    beta = np.zeros(p)
    eta = np.zeros(X.shape[0])
    best = 0.0
    for j in range(p):
        if pf[j] == 0.0:
            continue
        _, g1, _ = model_terms(model, time_sorted, status_sorted, X, beta, j, eta)
        best = max(best, abs(g1) / pf[j])
    return best
