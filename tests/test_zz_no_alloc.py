"""The allocation-free entry point, loglik_grad_hess_noalloc.

Some callers cannot allocate device memory while they run: their device
memory is owned by another allocator, or they cannot afford the implicit
device synchronisation of cudaMalloc/cudaFree.  For them the library offers
loglik_grad_hess_noalloc, which works out of one fixed device array that the
library reserves when it is loaded.  This test calls it through the C ABI
twice in a row and checks both results against the regular
loglik_grad_hess, with the tolerance the other parity tests use (the two
paths run the same kernels, so in practice they agree bit for bit).  It is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2204_08183_gb300 import binding, synth

from gpu_util import small_csc, survdata

pytestmark = pytest.mark.gpu


def _close(a, b, tol=1e-6):
    la, ga, ha = a
    lb, gb, hb = b
    assert abs(la - lb) <= tol * max(1.0, abs(lb))
    assert abs(ga - gb) <= tol * max(1.0, abs(gb))
    assert abs(ha - hb) <= tol * max(1.0, abs(hb))


def test_noalloc_matches_regular_entry_point_twice(lib):
    d = small_csc(120_000, 6, seed=21, density=0.05, n_times=2000)
    sd = survdata(d)
    beta = d["beta"] * 0.3
    ref = [binding.loglik_grad_hess(sd, "cox", beta, j) for j in (1, 4)]
    got = [binding.loglik_grad_hess_noalloc(sd, "cox", beta, j) for j in (1, 4)]   # two calls in a row
    for a, b in zip(got, ref):
        _close(a, b)
    again = binding.loglik_grad_hess_noalloc(sd, "cox", beta, 1)   # the array keeps the last call's contents
    _close(again, ref[0])


def test_noalloc_fine_gray_dense(lib):
    import torch
    f = synth.cohort_fg_dense(40_000, 3, seed=22, grid=500, n_true=3)
    sf = binding.SurvData(torch.from_numpy(f["time"]).cuda(), torch.from_numpy(f["status"]).cuda(),
                          X=torch.from_numpy(np.ascontiguousarray(f["X"].T)).cuda())
    b = np.array([0.2, -0.1, 0.05])
    for j in (0, 2):
        _close(binding.loglik_grad_hess_noalloc(sf, "fg", b, j), binding.loglik_grad_hess(sf, "fg", b, j))


def test_noalloc_rejects_oversize_and_host_arrays(lib):
    d = small_csc(3_000_000, 2, seed=23, density=0.01, n_times=3_000_000)   # ~3e6 groups: far above 16 MiB
    with pytest.raises(binding.SurvError) as ei:
        binding.loglik_grad_hess_noalloc(survdata(d), "cox", np.zeros(2), 0)
    assert ei.value.code == binding.SURV_E_INVALID
    small = small_csc(1000, 2, seed=24, density=0.2, n_times=50)
    with pytest.raises(binding.SurvError) as ei:
        binding.loglik_grad_hess_noalloc(survdata(small, "host"), "cox", np.zeros(2), 0)
    assert ei.value.code == binding.SURV_E_INVALID


def test_noalloc_rejects_malformed_col_ptr_on_the_host(lib):
    # col_ptr is copied to the host and checked before any kernel reads
    # row_idx through it.  Both malformed tables below stay inside the
    # arrays' bounds, so no access could leave them even without the check.
    import torch
    n = 64
    t = torch.arange(n, 0, -1, dtype=torch.int32).cuda()
    s = torch.ones(n, dtype=torch.int8).cuda()
    ri = torch.tensor([1, 2, 3, 4, 9, 7, 8, 11], dtype=torch.int32).cuda()   # rows increase within each column
    for cp in ([2, 5, 8], [0, 5, 3]):                       # col_ptr[0] != 0; decreasing
        d = binding.SurvData(t, s, col_ptr=torch.tensor(cp, dtype=torch.int64).cuda(), row_idx=ri)
        with pytest.raises(binding.SurvError) as ei:
            binding.loglik_grad_hess_noalloc(d, "cox", np.zeros(2), 0)
        assert ei.value.code == binding.SURV_E_INDEX
    good = binding.SurvData(t, s, col_ptr=torch.tensor([0, 5, 8], dtype=torch.int64).cuda(), row_idx=ri)
    _close(binding.loglik_grad_hess_noalloc(good, "cox", np.zeros(2), 1),
           binding.loglik_grad_hess(good, "cox", np.zeros(2), 1))
