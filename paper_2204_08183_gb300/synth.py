"""Seeded synthetic survival cohorts (data simulation only).

These generators produce inputs in the layout the library expects:
subjects already arranged by decreasing integer time (ties in draw order),
``status`` codes 0 = censored, 1 = event (Cox) / primary event (Fine-Gray),
2 = competing event, and X either dense column-major or column-compressed
(CSC) with row indices in the sorted subject order.  They hold none of the
likelihood, scan or coordinate-descent arithmetic; the tests and the bench
feed the same arrays to the CUDA path and to the CPU oracle.

Cohort recipes (shapes follow the paper's synthetic design, Section 3.2,
with the sizes of the workloads benchmarked here):

* ``cohort_cox_dense``   N(0,1) covariates, beta ~ N(0, sd^2) on the first
  ``n_true`` coordinates, T ~ Exponential(rate exp(x.beta)),
  C ~ Uniform(0, c) with c bisected on the draw to hit ``censor_frac``.
* ``cohort_cox_sparse``  binary covariates, each entry 1 with probability
  ``density``, beta ~ Laplace(0, scale) on ``n_true`` random coordinates,
  same event and censoring model.
* ``cohort_fg_dense``    N(0,1) covariates, latent T1 ~ Exp(l1 exp(x.b1)),
  T2 ~ Exp(l2 exp(x.b2)), C ~ Exp(lc); (l1, l2, lc) calibrated on a
  100,000-subject pilot to the requested censored/primary/competing mix.

Observed times are mapped to an integer grid 1..G by
clip(ceil(G * y / q_0.99(y)), 1, G), which creates heavy Breslow ties.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "to_grid",
    "arrange_desc",
    "cohort_cox_dense",
    "cohort_cox_sparse",
    "cohort_fg_dense",
    "cohort_small",
    "csc_from_dense",
    "nll_cohort",
]


def to_grid(y, grid):
    """Map positive observed times to integers 1..grid (quantile scaled)."""
    q = np.quantile(y, 0.99)
    t = np.ceil(grid * y / q)
    return np.clip(t, 1, grid).astype(np.int32)


def arrange_desc(time):
    """Stable order of decreasing time (ties keep draw order)."""
    idx = np.arange(time.shape[0])
    return np.lexsort((idx, -time.astype(np.int64)))


def _bisect_uniform_censoring(T, u, frac, iters=60):
    """Scale c of C = c * u such that mean(C < T) is ``frac``."""
    lo, hi = 0.0, float(np.max(T) / max(np.min(u), 1e-12)) + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.mean(mid * u < T) > frac:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def csc_from_dense(X):
    """(col_ptr int64, row_idx int32, values float32) of a dense matrix."""
    X = np.asarray(X)
    cols, rows, vals = [], [], []
    col_ptr = np.zeros(X.shape[1] + 1, dtype=np.int64)
    for j in range(X.shape[1]):
        nz = np.flatnonzero(X[:, j])
        rows.append(nz.astype(np.int32))
        vals.append(X[nz, j].astype(np.float32))
        col_ptr[j + 1] = col_ptr[j] + nz.shape[0]
    row_idx = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    values = np.concatenate(vals) if vals else np.zeros(0, np.float32)
    return col_ptr, row_idx, values


def cohort_cox_dense(n, p, seed, n_true=5, beta_sd=0.5, censor_frac=0.30,
                     grid=365, dtype=np.float64):
    """Dense Cox cohort; X returned column-major (Fortran order)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p)).astype(dtype)
    beta = np.zeros(p)
    k = min(n_true, p)
    beta[:k] = rng.normal(0.0, beta_sd, size=k)
    eta = X.astype(np.float64) @ beta
    T = rng.exponential(1.0, size=n) / np.exp(eta)
    u = rng.random(n)
    c = _bisect_uniform_censoring(T, u, censor_frac)
    C = c * u
    y = np.minimum(T, C)
    status = (T <= C).astype(np.int8)
    time = to_grid(y, grid)
    perm = arrange_desc(time)
    return {
        "time": np.ascontiguousarray(time[perm]),
        "status": np.ascontiguousarray(status[perm]),
        "X": np.asfortranarray(X[perm]),
        "beta_true": beta,
        "layout": "dense",
    }


def cohort_cox_sparse(n, p, seed, density=0.05, n_true=10, laplace_scale=0.2,
                      censor_frac=0.50, grid=3650, binary_values=True):
    """Sparse binary Cox cohort in CSC form (rows in sorted subject order).

    Returns col_ptr (int64, p+1), row_idx (int32), values (float32 ones, or
    None when ``binary_values`` is False) plus time/status.
    """
    rng = np.random.default_rng(seed)
    true_cols = np.sort(rng.choice(p, size=min(n_true, p), replace=False))
    beta = np.zeros(p)
    beta[true_cols] = rng.laplace(0.0, laplace_scale, size=true_cols.shape[0])
    cols = []
    eta = np.zeros(n)
    for j in range(p):
        r = np.flatnonzero(rng.random(n, dtype=np.float32) < density)
        cols.append(r)
        if beta[j] != 0.0:
            eta[r] += beta[j]
    T = rng.exponential(1.0, size=n) / np.exp(eta)
    u = rng.random(n)
    c = _bisect_uniform_censoring(T, u, censor_frac)
    C = c * u
    y = np.minimum(T, C)
    status = (T <= C).astype(np.int8)
    time = to_grid(y, grid)
    perm = arrange_desc(time)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    row_parts = []
    for j, r in enumerate(cols):
        nr = inv[r].astype(np.int32)
        nr.sort()
        row_parts.append(nr)
        col_ptr[j + 1] = col_ptr[j] + nr.shape[0]
    row_idx = np.concatenate(row_parts) if row_parts else np.zeros(0, np.int32)
    values = np.ones(row_idx.shape[0], dtype=np.float32) if binary_values else None
    return {
        "time": np.ascontiguousarray(time[perm]),
        "status": np.ascontiguousarray(status[perm]),
        "col_ptr": col_ptr,
        "row_idx": row_idx,
        "values": values,
        "n": n,
        "p": p,
        "beta_true": beta,
        "layout": "csc",
    }


def _fg_rates(eta1, eta2, fracs, iters=200):
    """Calibrate (l1, l2, lc) so that the expected shares of primary,
    competing and censored outcomes match ``fracs`` = (cens, prim, comp)."""
    cens, prim, comp = fracs
    e1, e2 = np.exp(eta1), np.exp(eta2)
    l1, l2, lc = 1.0, 1.0, 1.0
    for _ in range(iters):
        tot = l1 * e1 + l2 * e2 + lc
        p1 = np.mean(l1 * e1 / tot)
        p2 = np.mean(l2 * e2 / tot)
        pc = np.mean(lc / tot)
        l1 *= (prim / p1) ** 0.5
        l2 *= (comp / p2) ** 0.5
        lc *= (cens / pc) ** 0.5
    return l1, l2, lc


def cohort_fg_dense(n, p, seed, fracs=(0.40, 0.35, 0.25), grid=1000,
                    dtype=np.float32, n_true=10, beta_sd=0.3):
    """Dense competing-risks cohort; status 0/1/2; X column-major."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p), dtype=np.float32).astype(dtype, copy=False)
    k = min(n_true, p)
    b1 = np.zeros(p)
    b2 = np.zeros(p)
    b1[:k] = rng.normal(0.0, beta_sd, size=k)
    lo2 = min(k // 2, p)
    hi2 = min(lo2 + k, p)
    b2[lo2:hi2] = rng.normal(0.0, beta_sd, size=hi2 - lo2)
    pilot = min(n, 100_000)
    Xp = X[:pilot].astype(np.float64)
    l1, l2, lc = _fg_rates(Xp @ b1, Xp @ b2, fracs)
    Xd = X.astype(np.float64) if dtype != np.float64 else X
    eta1 = Xd @ b1
    eta2 = Xd @ b2
    del Xd
    T1 = rng.exponential(1.0, size=n) / (l1 * np.exp(eta1))
    T2 = rng.exponential(1.0, size=n) / (l2 * np.exp(eta2))
    C = rng.exponential(1.0, size=n) / lc
    y = np.minimum(np.minimum(T1, T2), C)
    status = np.where(C <= np.minimum(T1, T2), 0, np.where(T1 <= T2, 1, 2)).astype(np.int8)
    time = to_grid(y, grid)
    perm = arrange_desc(time)
    return {
        "time": np.ascontiguousarray(time[perm]),
        "status": np.ascontiguousarray(status[perm]),
        "X": np.asfortranarray(X[perm]),
        "beta_true": b1,
        "beta2_true": b2,
        "layout": "dense",
    }


def cohort_small(n, p, seed, n_times=None, censor_frac=0.3, competing_frac=0.0,
                 density=1.0, dtype=np.float64, scale=0.5):
    """Small mixed cohort for parity tests: arbitrary tie structure
    (``n_times`` distinct integer times, default n), optional competing
    events (status 2) and optional sparsity.  Already in decreasing order."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    if density < 1.0:
        X *= rng.random((n, p)) < density
    X = X.astype(dtype)
    n_times = n if n_times is None else n_times
    time = rng.integers(1, n_times + 1, size=n).astype(np.int32)
    u = rng.random(n)
    status = np.where(u < censor_frac, 0,
                      np.where(u < censor_frac + competing_frac, 2, 1)).astype(np.int8)
    perm = arrange_desc(time)
    beta = rng.normal(0.0, scale, size=p)
    return {
        "time": np.ascontiguousarray(time[perm]),
        "status": np.ascontiguousarray(status[perm]),
        "X": np.asfortranarray(X[perm]),
        "beta": beta,
        "layout": "dense",
    }


def nll_cohort(n, p, C, seed, n_times=5000, censor_frac=0.3, b_sd=0.05):
    """Inputs of the differentiable form: X ~ N(0, 1) float32 (n, p)
    row-major (the caller rounds it to bfloat16), B ~ N(0, b_sd^2) float32
    (p, C), integer times uniform on 1..n_times in decreasing order, status
    1 (event) with probability 1 - censor_frac, else 0."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p), dtype=np.float32)
    B = rng.normal(0.0, b_sd, size=(p, C)).astype(np.float32)
    time = np.sort(rng.integers(1, n_times + 1, size=n).astype(np.int32))[::-1].copy()
    status = (rng.random(n) >= censor_frac).astype(np.int8)
    return {"X": X, "B": B, "time": time, "status": status}


def cv_folds(n, nfolds, seed, lo=0.8, hi=1.2):
    """Uneven random fold assignment (int8 [n]): fold sizes spaced evenly
    from lo to hi times n / nfolds (rescaled to sum to n), subjects assigned
    to folds by a random permutation."""
    rng = np.random.default_rng(seed)
    w = np.linspace(lo, hi, nfolds) if nfolds > 1 else np.ones(1)
    sizes = np.floor(w / w.sum() * n).astype(np.int64)
    sizes[: n - sizes.sum()] += 1
    fold = np.repeat(np.arange(nfolds, dtype=np.int8), sizes)
    return np.ascontiguousarray(fold[rng.permutation(n)])


def lambda_grid(lambda_max, nlambda, ratio=1e-3):
    """nlambda log-spaced strengths from lambda_max down to ratio * lambda_max."""
    return lambda_max * np.logspace(0.0, np.log10(ratio), nlambda)
