"""Differentiable form: the Cox NLL of eta = X B and its gradient through
the C ABI (cox_nll_forward / cox_nll_backward) and the autograd function,
against the FP64 oracle (oracle/nll.py).

Tolerances.  X B runs on the tensor cores with bf16 inputs and FP32
accumulation, B split into bf16 high + low parts.  Against the oracle
evaluated at the split B (B_eff = hi + lo, the B the GPU actually uses) the
error is the FP32 GEMM accumulation and the FP32 scans: NLL within 1e-6
relative, gradient within 2e-3 of its largest entry.  Against the exact B
the split adds ~2^-16 relative per entry of B."""
import numpy as np
import pytest

import oracle
from paper_2204_08183_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _to_gpu(c):
    import torch
    X = torch.from_numpy(c["X"]).cuda().to(torch.bfloat16)
    return (X, torch.from_numpy(c["B"]).cuda(), torch.from_numpy(c["time"]).cuda(),
            torch.from_numpy(c["status"]).cuda())


def _split(B):
    import torch
    Bt = torch.from_numpy(B)
    hi = Bt.to(torch.bfloat16).float()
    lo = (Bt - hi).to(torch.bfloat16).float()
    return (hi.double() + lo.double()).numpy()


def _case(n, p, C, seed, n_times=500):
    c = synth.nll_cohort(n, p, C, seed, n_times=n_times)
    X, B, t, s = _to_gpu(c)
    Xo = X.float().cpu().numpy().astype(np.float64)   # the bf16 values the GPU uses
    return c, X, B, t, s, Xo


@pytest.mark.parametrize("C", [1, 8, 64])
def test_forward_and_gradient_match_oracle(lib, C):
    import torch
    c, X, B, t, s, Xo = _case(30_000, 16, C, seed=40 + C)
    Beff = _split(c["B"])
    Bt = B.clone().requires_grad_(True)
    nll = binding.cox_nll(Bt, X, t, s)
    ref = oracle.cox_nll(c["time"], c["status"], Xo @ Beff)
    np.testing.assert_allclose(nll.detach().cpu().numpy(), ref, rtol=1e-6, atol=0)
    w = torch.linspace(0.5, 1.5, C, dtype=torch.float64, device="cuda")
    (g,) = torch.autograd.grad((nll * w).sum(), Bt)
    gref = oracle.cox_nll_grad_B(Xo, c["time"], c["status"], Beff) * w.cpu().numpy()[None, :]
    scale = np.abs(gref).max()
    assert np.abs(g.cpu().numpy() - gref).max() <= 2e-3 * scale
    # against the exact float32 B: the split's error only
    exact = oracle.cox_nll(c["time"], c["status"], Xo @ c["B"].astype(np.float64))
    np.testing.assert_allclose(nll.detach().cpu().numpy(), exact, rtol=1e-5, atol=0)


def test_gradient_central_differences(lib):
    import torch
    c, X, B, t, s, Xo = _case(20_000, 12, 4, seed=51)
    Bt = B.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(binding.cox_nll(Bt, X, t, s).sum(), Bt)
    g = g.cpu().numpy()
    Beff = _split(c["B"])
    h = 1e-3
    rng = np.random.default_rng(0)
    for _ in range(8):
        j, b = int(rng.integers(12)), int(rng.integers(4))
        Bp, Bm = Beff.copy(), Beff.copy()
        Bp[j, b] += h
        Bm[j, b] -= h
        fd = (oracle.cox_nll(c["time"], c["status"], Xo @ Bp)[b]
              - oracle.cox_nll(c["time"], c["status"], Xo @ Bm)[b]) / (2 * h)
        assert g[j, b] == pytest.approx(fd, rel=5e-3, abs=5e-3 * np.abs(g).max())


def test_heavy_ties_and_no_events_columns(lib):
    import torch
    c, X, B, t, s, Xo = _case(5_000, 8, 3, seed=52, n_times=7)      # 7 distinct times
    nll = binding.cox_nll(B, X, t, s)
    ref = oracle.cox_nll(c["time"], c["status"], Xo @ _split(c["B"]))
    np.testing.assert_allclose(nll.cpu().numpy(), ref, rtol=1e-6)
    s0 = torch.zeros_like(s)                                         # no events: NLL = 0, gradient 0
    Bt = B.clone().requires_grad_(True)
    out = binding.cox_nll(Bt, X, t, s0)
    assert np.all(out.detach().cpu().numpy() == 0.0)
    (g,) = torch.autograd.grad(out.sum(), Bt)
    assert float(g.abs().max()) == 0.0


def test_errors(lib):
    import torch
    c, X, B, t, s, Xo = _case(2_000, 8, 2, seed=53)
    ws = binding.Workspace()
    with pytest.raises(binding.SurvError) as ei:     # backward before any forward
        binding.cox_nll_backward(X, t, s, torch.ones(2, dtype=torch.float64, device="cuda"), 2, ws)
    assert ei.value.code == binding.SURV_E_INVALID
    with pytest.raises(binding.SurvError) as ei:     # more than 64 columns
        binding.cox_nll_forward(X, t, s, torch.zeros((8, 65), device="cuda"), ws)
    assert ei.value.code == binding.SURV_E_INVALID
    with pytest.raises(binding.SurvError) as ei:     # unsorted times
        binding.cox_nll_forward(X, t.flip(0).contiguous(), s, B, ws)
    assert ei.value.code == binding.SURV_E_UNSORTED
    with pytest.raises(binding.SurvError) as ei:     # host arrays
        binding.cox_nll_forward(X.cpu(), t, s, B, ws)
    assert ei.value.code == binding.SURV_E_INVALID


def test_full_size_sampled(lib):
    """N = 2^22, p = 256, C = 64: NLL of 4 columns and 16 gradient entries
    against the oracle."""
    import torch
    n, p, C = 1 << 22, 256, 64
    c = synth.nll_cohort(n, p, C, seed=5, n_times=5000)
    X, B, t, s = _to_gpu(c)
    Bt = B.clone().requires_grad_(True)
    nll = binding.cox_nll(Bt, X, t, s)
    (g,) = torch.autograd.grad(nll.sum(), Bt)
    Xo = X.float().cpu().numpy()
    Beff = _split(c["B"])
    cols = [0, 17, 42, 63]
    eta = (Xo.astype(np.float64) @ Beff[:, cols])
    ref = oracle.cox_nll(c["time"], c["status"], eta)
    np.testing.assert_allclose(nll.detach().cpu().numpy()[cols], ref, rtol=1e-6)
    ge = oracle.cox_nll_grad_eta(c["time"], c["status"], eta)
    gref = Xo.T.astype(np.float64) @ ge                     # (p, 4)
    gg = g.cpu().numpy()[:, cols]
    assert np.abs(gg - gref).max() <= 2e-3 * np.abs(gref).max()
