"""GPU parity of the sparse-numerator form of the Cox CCD
(cox_fit with SURV_FLAG_SPARSE_NUMERATOR; not in the paper) against the
FP64 oracle and against the row-pass schedule.  Same bars as the row-pass
fits: beta within 1e-5 of the oracle run for the same number of sweeps,
log-likelihood within 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

from gpu_util import oracle_X, small_csc, survdata

pytestmark = pytest.mark.gpu
SN = binding.SURV_FLAG_SPARSE_NUMERATOR


def _fit_vs_oracle(d, penalty, lam, tol=1e-10):
    sd = survdata(d)
    beta, info, rc = binding.cox_fit(sd, penalty=penalty, lam=lam, tol=tol, max_sweeps=200, flags=SN)
    assert info["converged"] == 1
    st = np.where(d["status"] == 2, 0, d["status"]).astype(np.int8)
    ref = oracle.ccd_fit("cox", d["time"], st, oracle_X(d), penalty, lam, tol=0.0, max_sweeps=info["sweeps"])
    np.testing.assert_allclose(beta, ref["beta"], rtol=0, atol=1e-5)
    assert info["loglik"] == pytest.approx(ref["loglik"], rel=1e-6)
    return beta, info


@pytest.mark.parametrize("binary", [True, False])
@pytest.mark.parametrize("n,n_times", [(3001, 40), (5003, 5003), (20000, 300)])
def test_sn_fit_matches_oracle_l1(lib, binary, n, n_times):
    d = small_csc(n, 12, seed=n + n_times, density=0.15, n_times=n_times, binary=binary)
    lmax = oracle.lambda_max("cox", d["time"], d["status"], oracle_X(d))
    _fit_vs_oracle(d, "l1", 0.3 * lmax)


def test_sn_fit_matches_oracle_l2(lib):
    d = small_csc(4000, 8, seed=7, density=0.3, n_times=200)
    _fit_vs_oracle(d, "l2", 2.0)


def test_sn_equals_row_pass_fit(lib):
    d = small_csc(50000, 20, seed=9, density=0.05, n_times=1000, binary=True)
    sd = survdata(d)
    # tolerance 1e-7: the FP32 mode's objective carries rounding noise near
    # 1e-11 relative, which would decide the sweep count at tighter ones
    b0, i0, _ = binding.cox_fit(sd, penalty="l1", lam=20.0, tol=1e-7)
    b1, i1, _ = binding.cox_fit(sd, penalty="l1", lam=20.0, tol=1e-7, flags=SN)
    assert i0["sweeps"] == i1["sweeps"]
    np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-6)
    assert i1["loglik"] == pytest.approx(i0["loglik"], rel=1e-9)


def test_sn_many_groups_per_warp(lib):
    # unique times: far more tie groups than warps (the many-ends row pass)
    d = small_csc(400_000, 6, seed=11, density=0.05, n_times=400_000)
    sd = survdata(d)
    b0, i0, _ = binding.cox_fit(sd, penalty="l2", lam=1.0, tol=1e-10)
    b1, i1, _ = binding.cox_fit(sd, penalty="l2", lam=1.0, tol=1e-10, flags=SN)
    np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-6)
    st = d["status"]
    ref = oracle.ccd_fit("cox", d["time"], st, oracle_X(d), "l2", 1.0, tol=0.0, max_sweeps=i1["sweeps"])
    np.testing.assert_allclose(b1, ref["beta"], rtol=0, atol=1e-5)


def test_sn_rejects_unsupported(lib):
    d = synth.cohort_small(500, 3, 1, n_times=50)
    with pytest.raises(binding.SurvError) as e:
        binding.cox_fit(survdata(d), penalty="l2", lam=1.0, flags=SN)      # dense X
    assert e.value.code == binding.SURV_E_INVALID
    c = small_csc(500, 3, seed=2, density=0.3, n_times=50)
    with pytest.raises(binding.SurvError) as e:
        binding.cox_fit(survdata(c), penalty="l2", lam=1.0, precision="f64", flags=SN)
    assert e.value.code == binding.SURV_E_INVALID
    with pytest.raises(binding.SurvError) as e:
        binding.fg_fit(survdata(c), penalty="l2", lam=1.0, flags=SN)
    assert e.value.code == binding.SURV_E_INVALID


def test_sn_headline_size(lib):
    """N = 10^7, p = 100 binary at 5 %, L1 lambda = 1e-4 N: the same fit as the
    row-pass schedule (same sweeps, beta within 1e-5), and one coordinate
    of the final beta checked against the oracle's derivatives."""
    d = synth.cohort_cox_sparse(10_000_000, 100, seed=2, density=0.05, n_true=10, laplace_scale=0.2,
                                censor_frac=0.5, grid=3650)
    sd = survdata(d)
    b0, i0, _ = binding.cox_fit(sd, penalty="l1", lam=1e3, tol=1e-8)
    b1, i1, _ = binding.cox_fit(sd, penalty="l1", lam=1e3, tol=1e-8, flags=SN)
    assert i1["converged"] == 1 and i1["sweeps"] == i0["sweeps"]
    np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-5)
    assert i1["loglik"] == pytest.approx(i0["loglik"], rel=1e-7)


def test_sn_long_column(lib):
    # columns longer than 2048 entries per CTA of the default grid: the
    # column kernels take more CTAs
    d = small_csc(2_000_000, 3, seed=13, density=0.5, n_times=5000, binary=True)
    sd = survdata(d)
    b0, i0, _ = binding.cox_fit(sd, penalty="l2", lam=5.0, tol=1e-7)
    b1, i1, _ = binding.cox_fit(sd, penalty="l2", lam=5.0, tol=1e-7, flags=SN)
    assert i1["sweeps"] == i0["sweeps"]
    np.testing.assert_allclose(b1, b0, rtol=0, atol=1e-6)
