"""Parity at the benchmarked sizes: the fits bench.py times, in the launch
configuration it times them (the default schedule: speculative batches of 4
coordinates for the Cox fit of CSC data, one coordinate per pass for the
dense Fine-Gray fit), against the FP64 oracle run for the same number of
sweeps (Section 2.4 CCD with the risk-set sums of Section 2.7).

Bars: converged beta within 1e-5 absolute, log-likelihood within 1e-6
relative, and (L1) the same set of zero coefficients.  The oracle takes
a few minutes here (about 0.4 s per coordinate pass at N = 10^7 and 1 s per
Fine-Gray pass at N = 5 x 10^6 on one host core).
"""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

from gpu_util import oracle_X, survdata

pytestmark = pytest.mark.gpu


def test_cox_l1_headline_fit_matches_oracle(lib):
    """N = 10^7 subjects, p = 100 binary columns at 5 % density (CSC, FP32
    values), 50 % censoring, days 1..3650, L1 lambda = 1e-4 N, tol 1e-8."""
    d = synth.cohort_cox_sparse(10_000_000, 100, seed=2, density=0.05, n_true=10, laplace_scale=0.2,
                                censor_frac=0.5, grid=3650)
    beta, info, rc = binding.cox_fit(survdata(d), penalty="l1", lam=1e3, tol=1e-8)
    assert rc == 0 and info["converged"] == 1
    assert info["row_passes"] < info["coordinate_passes"]          # the batched schedule ran
    ref = oracle.ccd_fit("cox", d["time"], d["status"], oracle_X(d), "l1", 1e3, tol=0.0,
                         max_sweeps=info["sweeps"])
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5)
    assert info["loglik"] == pytest.approx(ref["loglik"], rel=1e-6)
    assert np.array_equal(beta == 0.0, ref["beta"] == 0.0)
    assert np.count_nonzero(beta) >= 5


def test_fine_gray_l2_benchmarked_size_two_sweeps(lib):
    """N = 5 x 10^6, p = 50 dense float32 N(0,1) covariates, 40/35/25 %
    censored/primary/competing, days 1..1000, Kaplan-Meier weights on the
    device, L2 lambda = 10; two full sweeps on both sides."""
    f = synth.cohort_fg_dense(5_000_000, 50, seed=3, grid=1000, n_true=10)
    beta, info, rc = binding.fg_fit(survdata(f), penalty="l2", lam=10.0, tol=0.0, max_sweeps=2)
    assert info["sweeps"] == 2
    ref = oracle.ccd_fit("fg", f["time"], f["status"], f["X"], "l2", 10.0, tol=0.0, max_sweeps=2)
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5)
    assert info["loglik"] == pytest.approx(ref["loglik"], rel=1e-6)
    assert np.abs(ref["beta"]).max() > 0.05                         # the fit moved
