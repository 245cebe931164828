"""Input validation and failure detection through the C ABI (GPU).

The device-timeout test makes one CTA of the persistent kernel skip its
first grid-exchange arrival (a flag that nothing sets), gives every wait a
50 ms limit, and checks that the call returns SURV_E_DEVICE_TIMEOUT and that
the next call on the same context succeeds.  Nothing here traps, faults or
hangs the GPU."""
import numpy as np
import pytest

from paper_2204_08183_gb300 import binding, synth

from gpu_util import small_csc, survdata

pytestmark = pytest.mark.gpu


def _code(fn, *a, **k):
    with pytest.raises(binding.SurvError) as ei:
        fn(*a, **k)
    return ei.value.code


def test_unsorted_times(lib):
    d = synth.cohort_small(100, 2, seed=1, n_times=20)
    d["time"] = d["time"][::-1].copy()
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_UNSORTED


def test_bad_status(lib):
    d = synth.cohort_small(100, 2, seed=2, n_times=20)
    d["status"][5] = 2
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_STATUS
    d["status"][5] = 3
    assert _code(binding.fg_fit, survdata(d)) == binding.SURV_E_STATUS


def test_no_events(lib):
    d = synth.cohort_small(100, 2, seed=3, n_times=20)
    d["status"][:] = 0
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_NO_EVENTS
    d["status"][:3] = 2
    assert _code(binding.fg_fit, survdata(d)) == binding.SURV_E_NO_EVENTS


def test_nonfinite(lib):
    d = synth.cohort_small(100, 2, seed=4, n_times=20)
    d["X"][7, 1] = np.nan
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_NONFINITE
    d = synth.cohort_small(100, 2, seed=4, n_times=20)
    assert _code(binding.cox_fit, survdata(d), beta=np.array([np.inf, 0.0])) == binding.SURV_E_NONFINITE


def test_bad_csc(lib):
    d = small_csc(1000, 3, seed=5, density=0.2)
    d["row_idx"] = d["row_idx"].copy()
    d["row_idx"][d["col_ptr"][1] + 1] = d["row_idx"][d["col_ptr"][1]]   # repeated row in column 1
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_INDEX
    d = small_csc(1000, 3, seed=5, density=0.2)
    d["row_idx"] = d["row_idx"].copy()
    d["row_idx"][-1] = 1000                                             # out of range
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_INDEX
    d = small_csc(1000, 3, seed=5, density=0.2)
    d["col_ptr"] = d["col_ptr"].copy()
    d["col_ptr"][1], d["col_ptr"][2] = d["col_ptr"][2], d["col_ptr"][1]  # decreasing col_ptr
    assert _code(binding.cox_fit, survdata(d)) == binding.SURV_E_INDEX


def test_bad_arguments(lib):
    d = synth.cohort_small(100, 2, seed=6, n_times=20)
    sd = survdata(d)
    assert _code(binding.loglik_grad_hess, sd, "cox", np.zeros(2), 2) == binding.SURV_E_INVALID
    assert _code(binding.cox_fit, sd, lam=-1.0) == binding.SURV_E_INVALID
    assert _code(binding.cox_fit, sd, max_sweeps=-1) == binding.SURV_E_INVALID


def test_device_wait_timeout_is_reported_and_context_survives(lib):
    d = small_csc(50_000, 3, seed=7, density=0.1, n_times=300)
    sd = survdata(d)
    beta = np.zeros(3)
    with pytest.raises(binding.SurvError) as ei:
        binding.cox_fit(sd, beta=beta, flags=binding.SURV_FLAG_TEST_STALL, wait_limit_s=0.05)
    assert ei.value.code == binding.SURV_E_DEVICE_TIMEOUT
    # the context is still usable: a normal call right after succeeds
    b, info, rc = binding.cox_fit(sd, penalty="l2", lam=1.0)
    assert rc == 0 and info["device_error"] == 0
    import torch
    torch.cuda.synchronize()
