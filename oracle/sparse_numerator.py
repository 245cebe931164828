"""FP64 restatement of the Cox coordinate derivatives in sparse-numerator
form: the same l'_j and l''_j as Eqs. cox_g / cox_h (Section 2.7), with the
sums over tie groups moved onto the nonzeros of column j.  This is not in
the paper; it is the algebra behind the library's sparse-numerator fit
(cox_fit with SURV_FLAG_SPARSE_NUMERATOR), written out plainly so that it
can be checked against the definition.

TEST INFRASTRUCTURE ONLY, like oracle/survival.py.

Subjects in decreasing time, tie groups k = 0..K-1 with last subject e_k,
events d_k, Den_k = sum_{r <= e_k} exp(eta_r).  Subject i belongs to group
g(i) (the first k with e_k >= i) and is at risk at every t_k with k >= g(i).
With a_t = x_{i_t j} exp(eta_{i_t}) over the nonzeros t = 1..m of column j
(rows increasing):

    sum_k d_k N1_k / Den_k = sum_t a_t Lam(g_t),
    sum_k d_k N2_k / Den_k = sum_t x_t a_t Lam(g_t),
    Lam(g) = sum_{k >= g} d_k / Den_k;

    sum_k d_k (N1_k / Den_k)^2 = sum_t C_t^2 [W(g_{t+1}) - W(g_t)],
    C_t = a_1 + ... + a_t,  W(g) = sum_{k < g} d_k / Den_k^2,  g_{m+1} = K,

because N1_k = C_t for k in [g_t, g_{t+1}).  Then
    l'_j = delta^T X_j - sum_k d_k N1_k / Den_k,
    l''_j = -(sum_k d_k N2_k / Den_k - sum_k d_k (N1_k / Den_k)^2),
    l = delta^T eta - sum_k d_k log Den_k.

Pin (tests/test_oracle_sparse_numerator.py): equal to oracle.cox_terms (the
definition, itself pinned to brute-force risk sets) on tied and untied,
binary and valued columns, including empty columns and nonzeros in the last
group.
"""
from __future__ import annotations

import numpy as np

from .survival import column, linear_predictor, tie_groups

__all__ = ["cox_terms_sparse_numerator"]


def cox_terms_sparse_numerator(time_sorted, status_sorted, X, beta, j, eta=None):
    """(l, l'_j, l''_j) from the sparse-numerator sums above."""
    time_sorted = np.asarray(time_sorted)
    delta = (np.asarray(status_sorted) == 1).astype(np.float64)
    if eta is None:
        eta = linear_predictor(X, beta)
    e = np.exp(eta)
    gend = tie_groups(time_sorted)
    K = gend.shape[0]
    cs = np.concatenate([[0.0], np.cumsum(delta)])
    dk = cs[gend + 1] - cs[np.concatenate([[-1], gend[:-1]]) + 1]
    den = np.cumsum(e)[gend]
    lam = np.cumsum((dk / den)[::-1])[::-1]                       # Lam(g), g = 0..K-1
    W = np.concatenate([[0.0], np.cumsum(dk / den ** 2)])          # W(g), g = 0..K
    x = column(X, j)
    rows = np.flatnonzero(x)
    g = np.searchsorted(gend, rows)                                # group of each nonzero row
    a = x[rows] * e[rows]
    C = np.cumsum(a)
    g_next = np.concatenate([g[1:], [K]])
    s1 = float(np.sum(a * lam[g]))
    s2 = float(np.sum(x[rows] * a * lam[g]))
    q = float(np.sum(C ** 2 * (W[g_next] - W[g])))
    grad = float(delta @ x) - s1
    hess = -(s2 - q)
    l = float(delta @ eta) - float(np.sum(dk * np.log(den)))
    return l, grad, hess
