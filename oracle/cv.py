"""FP64 CPU oracle for the cross-validated penalty path (Section 2.8): k-fold
cross-validation over a grid of penalty strengths, one penalised Cox CCD fit
per (lambda, fold) pair on the subjects outside the fold, each scored by the
log partial likelihood of the fold's own subjects on their own risk sets.

TEST INFRASTRUCTURE ONLY, like oracle/survival.py.

Written as the plain definition: each training set is cut out of the data
(subjects keep their decreasing-time order, so tie groups stay runs) and
fitted with ``ccd_fit``; each held-out set is cut out the same way and
scored with ``cox_terms``.  Nothing is batched or masked here.

Readings fixed here (Section 2.8 names cross-validation and its
out-of-sample likelihood but not these details):
* every fit starts from beta = 0 (cold start), width 1;
* the held-out score of fit (l, k) is the Breslow log partial likelihood of
  the subjects of fold k alone, at the fit's beta (their risk sets contain
  only fold-k subjects);
* the path's score at lambda l is the mean over folds of the held-out
  scores, and the chosen lambda is the first index with the largest mean.

Pins (tests/test_oracle_cv.py): the held-out score equals an O(N^2)
brute-force risk-set sum on the fold; a fold without events scores 0; above
the training set's lambda_max a fit is exactly zero and its score has the
closed form -sum_g dh_g log n_g (null model on the fold); relabelling the
folds permutes the results; cv_mean / best follow their definitions.
"""
from __future__ import annotations

import numpy as np

from .survival import ccd_fit, cox_terms

__all__ = ["heldout_loglik", "cv_path"]


def _rows(X, mask):
    return X[np.flatnonzero(mask)] if hasattr(X, "tocsc") else np.asarray(X)[mask]


def heldout_loglik(time_sorted, status_sorted, X, beta, mask):
    """Breslow log partial likelihood of the subjects in ``mask`` on their
    own risk sets at ``beta`` (0 when the subset has no event)."""
    mask = np.asarray(mask, dtype=bool)
    st = np.asarray(status_sorted)[mask]
    if not np.any(st == 1):
        return 0.0
    l, _, _ = cox_terms(np.asarray(time_sorted)[mask], st, _rows(X, mask), beta, 0)
    return float(l)


def cv_path(time_sorted, status_sorted, X, fold_id, nfolds, lambdas, penalty="l1", pf=None, tol=1e-8,
            max_sweeps=100, sweeps=None):
    """Fit f = l * nfolds + k for every lambda l and fold k.  ``sweeps``
    (optional [nlambda][nfolds]) runs exactly that many sweeps per fit
    (tol = 0), to compare with another implementation sweep for sweep.

    Returns dict(beta [L, K, p], heldout [L, K], cv_mean [L], best,
    sweeps [L, K], converged [L, K])."""
    fold_id = np.asarray(fold_id)
    lambdas = np.asarray(lambdas, dtype=np.float64)
    L, K = lambdas.shape[0], int(nfolds)
    p = X.shape[1]
    time_sorted = np.asarray(time_sorted)
    status_sorted = np.asarray(status_sorted)
    beta = np.zeros((L, K, p))
    held = np.zeros((L, K))
    sw = np.zeros((L, K), np.int64)
    conv = np.zeros((L, K), bool)
    for li, lam in enumerate(lambdas):
        for k in range(K):
            train = fold_id != k
            kw = dict(tol=tol, max_sweeps=max_sweeps) if sweeps is None else \
                dict(tol=0.0, max_sweeps=int(sweeps[li][k]))
            r = ccd_fit("cox", time_sorted[train], status_sorted[train], _rows(X, train), penalty, lam, pf=pf, **kw)
            beta[li, k] = r["beta"]
            sw[li, k] = r["sweeps"]
            conv[li, k] = r["converged"]
            held[li, k] = heldout_loglik(time_sorted, status_sorted, X, r["beta"], fold_id == k)
    mean = held.mean(axis=1)
    return {"beta": beta, "heldout": held, "cv_mean": mean, "best": int(np.argmax(mean)), "sweeps": sw,
            "converged": conv}
