"""GPU parity of the speculative coordinate batches (the default for Cox
fits of CSC data in the FP32 mode): every committed step is the one cyclic
CCD takes, so the fit must match the oracle run for the same number of
sweeps (beta within 1e-5) and the one-coordinate-per-pass fit
(SURV_FLAG_ONE_COORDINATE: same sweeps, beta within 1e-6), with fewer
passes over the subjects.  The stopping tolerance of the
comparisons is 1e-7: the FP32 mode's objective carries rounding noise near
1e-11 relative, which decides the sweep count at tighter tolerances."""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

from gpu_util import oracle_X, small_csc, survdata

pytestmark = pytest.mark.gpu
SPEC = 0                                   # the default
ONE = binding.SURV_FLAG_ONE_COORDINATE


@pytest.fixture(params=[0, binding.SURV_FLAG_SPEC_B8], ids=["B4", "B8"])
def batch(request):
    """Extra flags selecting 4 (default) or 8 coordinates per batch."""
    return request.param


@pytest.mark.parametrize("binary", [True, False])
@pytest.mark.parametrize("n,p,n_times", [(3001, 10, 40), (20000, 13, 300), (7, 3, 4)])
def test_spec_fit_matches_oracle_l1(lib, batch, binary, n, p, n_times):
    d = small_csc(n, p, seed=n + p, density=0.3 if n < 100 else 0.15, n_times=n_times, binary=binary)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d))
    lam = 0.3 * lmax
    sd = survdata(d)
    beta, info, rc = binding.cox_fit(sd, penalty="l1", lam=lam, tol=1e-7, max_sweeps=200, flags=SPEC | batch)
    ref = oracle.ccd_fit("cox", d["time"], d["status"], oracle_X(d), "l1", lam, tol=0.0,
                         max_sweeps=info["sweeps"])
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5)
    assert info["loglik"] == pytest.approx(ref["loglik"], rel=1e-6)
    b0, i0, _ = binding.cox_fit(sd, penalty="l1", lam=lam, tol=1e-7, max_sweeps=200, flags=ONE)
    assert i0["sweeps"] == info["sweeps"]
    np.testing.assert_allclose(beta, b0, rtol=0, atol=1e-6)
    assert info["row_passes"] <= i0["row_passes"]


def test_spec_l2_all_nonzero_steps(lib, batch):
    # L2 with small lambda: nearly every step is nonzero (batches of one)
    d = small_csc(5000, 9, seed=5, density=0.3, n_times=500)
    sd = survdata(d)
    b1, i1, _ = binding.cox_fit(sd, penalty="l2", lam=0.5, tol=1e-7, flags=SPEC | batch)
    ref = oracle.ccd_fit("cox", d["time"], d["status"], oracle_X(d), "l2", 0.5, tol=0.0, max_sweeps=i1["sweeps"])
    np.testing.assert_allclose(b1, ref["beta"], rtol=0, atol=1e-5)


def test_spec_max_sweeps_zero_and_one(lib):
    d = small_csc(2000, 6, seed=6, density=0.3, n_times=100)
    sd = survdata(d)
    for ms in (0, 1, 2):
        b1, i1, rc1 = binding.cox_fit(sd, penalty="l1", lam=5.0, tol=0.0, max_sweeps=ms, flags=SPEC)
        b0, i0, rc0 = binding.cox_fit(sd, penalty="l1", lam=5.0, tol=0.0, max_sweeps=ms, flags=ONE)
        assert i1["sweeps"] == i0["sweeps"] == ms and rc1 == rc0
        np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-7)
        assert i1["loglik"] == pytest.approx(i0["loglik"], rel=1e-10)


def test_spec_headline_size(lib):
    """N = 10^7, p = 100 binary at 5 %, L1 lambda = 1e-4 N: the batched and
    the one-coordinate schedules agree (a check of the schedule, GPU against
    GPU; the oracle parity of this fit is tests/test_gpu_fullsize.py)."""
    d = synth.cohort_cox_sparse(10_000_000, 100, seed=2, density=0.05, n_true=10, laplace_scale=0.2,
                                censor_frac=0.5, grid=3650)
    sd = survdata(d)
    b0, i0, _ = binding.cox_fit(sd, penalty="l1", lam=1e3, tol=1e-8, flags=ONE)
    b1, i1, _ = binding.cox_fit(sd, penalty="l1", lam=1e3, tol=1e-8, flags=SPEC)
    assert i1["converged"] == 1 and i1["sweeps"] == i0["sweeps"]
    np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-5)
    assert i1["loglik"] == pytest.approx(i0["loglik"], rel=1e-7)
    assert i1["row_passes"] < i0["row_passes"] / 2
