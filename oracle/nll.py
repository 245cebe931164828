"""FP64 CPU oracle for the differentiable form: the Cox negative log partial
likelihood (Breslow ties) of several linear predictors at once, eta = X B,
and its gradient (Section 2.9: the likelihood and its derivatives through
the same risk-set sums of Section 2.7, so the gradient is O(N) per column).

TEST INFRASTRUCTURE ONLY, like oracle/survival.py.

For column b of eta (subjects in decreasing time, tie groups k = 1..K with
last index e_k and d_k events):

    NLL_b = - sum_i delta_i eta_ib + sum_k d_k log den_kb,
    den_kb = sum_{r <= e_k} exp(eta_rb)                     (risk set at t_k)

    dNLL_b / d eta_ib = - delta_i + exp(eta_ib) Lambda_b(i),
    Lambda_b(i) = sum_{k : e_k >= i} d_k / den_kb            (groups whose
                                                              risk set holds i)

    dNLL / dB = X^T (dNLL / d eta)      (column b: X^T of column b).

Pins (tests/test_oracle_nll.py): NLL_b equals minus the Cox log-likelihood of
oracle/survival.py at beta = B[:, b]; the gradient equals minus its score;
central finite differences; a brute-force O(N^2) risk-set sum; and the
gradient with respect to eta sums to zero over subjects (a shift of eta by a
constant leaves NLL unchanged).
"""
from __future__ import annotations

import numpy as np

from .survival import tie_groups

__all__ = ["cox_nll", "cox_nll_grad_eta", "cox_nll_grad_B", "cox_nll_brute"]


def _groups(time_sorted, status_sorted):
    gend = tie_groups(time_sorted)
    delta = (np.asarray(status_sorted) == 1)
    cs = np.concatenate([[0], np.cumsum(delta)])
    dk = cs[gend + 1] - cs[np.concatenate([[-1], gend[:-1]]) + 1]
    return gend, dk.astype(np.float64), delta


def cox_nll(time_sorted, status_sorted, eta):
    """NLL per column of eta (n, C) in float64; returns (C,)."""
    eta = np.asarray(eta, dtype=np.float64)
    if eta.ndim == 1:
        eta = eta[:, None]
    gend, dk, delta = _groups(time_sorted, status_sorted)
    e = np.exp(eta)
    den = np.cumsum(e, axis=0)[gend]          # (K, C) prefix sums at the group ends
    return -(delta[:, None] * eta).sum(axis=0) + (dk[:, None] * np.log(den)).sum(axis=0)


def cox_nll_grad_eta(time_sorted, status_sorted, eta):
    """dNLL_b / d eta_ib, shape (n, C)."""
    eta = np.asarray(eta, dtype=np.float64)
    if eta.ndim == 1:
        eta = eta[:, None]
    gend, dk, delta = _groups(time_sorted, status_sorted)
    e = np.exp(eta)
    den = np.cumsum(e, axis=0)[gend]
    # Lambda at group k: sum over groups k' >= k of d_k' / den_k'
    lam_k = np.cumsum((dk[:, None] / den)[::-1], axis=0)[::-1]
    n = eta.shape[0]
    grp = np.searchsorted(gend, np.arange(n))  # group of each subject
    return -delta[:, None].astype(np.float64) + e * lam_k[grp]


def cox_nll_grad_B(X, time_sorted, status_sorted, B):
    """dNLL / dB = X^T dNLL/deta at eta = X B, shape (p, C)."""
    X = np.asarray(X, dtype=np.float64)
    eta = X @ np.asarray(B, dtype=np.float64)
    return X.T @ cox_nll_grad_eta(time_sorted, status_sorted, eta)


def cox_nll_brute(time, status, eta):
    """NLL of one column from explicit risk sets {r : y_r >= Y_i} per event
    (any subject order).  O(N^2)."""
    time = np.asarray(time)
    eta = np.asarray(eta, dtype=np.float64)
    total = 0.0
    for i in np.flatnonzero(np.asarray(status) == 1):
        risk = time >= time[i]
        total += -eta[i] + np.log(np.exp(eta[risk]).sum())
    return total
