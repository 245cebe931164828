"""Differentiable form: the Cox NLL of eta = X B and its gradient through
the C ABI (cox_nll_forward / cox_nll_backward) and the autograd function,
against the FP64 oracle (oracle/nll.py).

Tolerances, from the arithmetic of the CUDA path.  X B and X^T G run on the
tensor cores with bf16 inputs and FP32 accumulation; B and G are split into
bf16 high and low parts, so each carries 16 significant bits: the split
error of a value v is at most 2^-16 |v|.
  * NLL against the oracle at the split B (B_eff = hi + lo, the B the GPU
    uses): what remains is FP32 rounding of eta and e and the float-float
    risk-set sums, about 1e-8 relative; held to 1e-7.
  * NLL against the exact FP32 B: the split moves eta_i by at most
    2^-16 sum_j |X_ij B_jb|, so NLL_b by at most 2^-16 sum_i |G_ib| sum_j
    |X_ij B_jb| (G = dNLL/deta); that bound, computed by the oracle, is the
    tolerance.
  * Gradient: each term X_ij G_ib carries the split error of G_ib, at most
    2^-16 |G_ib| and roughly uniform, so the error of entry (j, b) has
    standard deviation sigma_jb = 2^-16 / sqrt(3) sqrt(sum_i X_ij^2 G_ib^2);
    held to 6 sigma_jb + 1e-7 |g_jb| (FP32 accumulation and the FP32 G add
    far less).  A 0.1 % systematic error in Lambda or in e Lambda - delta
    would exceed that by a factor of about 30 at N = 30,000.
  * Accumulation of X^T G in tensor memory: each CTA of the product adds
    the 16-row products of its contiguous row range into one FP32
    accumulator, and that accumulation rounds like truncation (biased), so
    its error grows with the accumulated magnitude: at most about 2^-23
    (rows / 16) |S_c| per CTA c, S_c the CTA's partial sum.  Negligible at
    N = 30,000 (under 200 rows a CTA), it dominates at N = 2^22 (27,648 rows
    a CTA): the full-size test adds it, computed per CTA by the oracle.
  * Central differences of the FP64 oracle NLL with Richardson
    extrapolation (h = 1e-3 and 2e-3, error O(h^4)) stand in for the
    oracle gradient; the same bound applies."""
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


def _grad_tol(Xo, Geta, g):
    """6 sigma of the split error of G plus 1e-7 |g| (see the module text)."""
    X2 = np.asarray(Xo, dtype=np.float64) ** 2
    sigma = 2.0 ** -16 / np.sqrt(3.0) * np.sqrt(X2.T @ (Geta ** 2))
    return 6.0 * sigma + 1e-7 * np.abs(g)


def _accumulation_bound(Xo, Geta, n_sm):
    """2^-23 (rows / 16) |S_c| summed over the product's CTAs, with the row
    ranges the library uses (one contiguous range of a multiple of 64 rows
    per CTA, one CTA per SM)."""
    n = Xo.shape[0]
    stages = (n + 63) // 64
    nx = max(1, min(n_sm, stages))
    rows = ((n + nx - 1) // nx + 63) // 64 * 64
    total = np.zeros((Xo.shape[1], Geta.shape[1]))
    for c0 in range(0, n, rows):
        Xc = np.asarray(Xo[c0:c0 + rows], dtype=np.float64)
        Sc = Xc.T @ Geta[c0:c0 + rows]
        total += 2.0 ** -23 * (Xc.shape[0] / 16.0) * np.abs(Sc)
    return total


def _nll_split_bound(Xo, Geta, B):
    """Largest change of NLL_b that the bf16 split of B can cause."""
    shift = 2.0 ** -16 * (np.abs(Xo) @ np.abs(np.asarray(B, np.float64)))   # bound on |d eta_ib|
    return (np.abs(Geta) * shift).sum(axis=0)


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
    np.testing.assert_allclose(nll.detach().cpu().numpy(), ref, rtol=1e-7, atol=0)
    w = torch.linspace(0.5, 1.5, C, dtype=torch.float64, device="cuda")
    (g,) = torch.autograd.grad((nll * w).sum(), Bt)
    Geta = oracle.cox_nll_grad_eta(c["time"], c["status"], Xo @ Beff) * w.cpu().numpy()[None, :]
    gref = Xo.T @ Geta
    assert np.all(np.abs(g.cpu().numpy() - gref) <= _grad_tol(Xo, Geta, gref))
    # against the exact float32 B: the split's error only
    exact = oracle.cox_nll(c["time"], c["status"], Xo @ c["B"].astype(np.float64))
    G1 = oracle.cox_nll_grad_eta(c["time"], c["status"], Xo @ c["B"].astype(np.float64))
    bound = _nll_split_bound(Xo, G1, c["B"]) + 1e-7 * np.abs(exact)
    assert np.all(np.abs(nll.detach().cpu().numpy() - exact) <= bound)


def test_gradient_central_differences(lib):
    import torch
    c, X, B, t, s, Xo = _case(20_000, 12, 4, seed=51)
    Bt = B.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(binding.cox_nll(Bt, X, t, s).sum(), Bt)
    g = g.cpu().numpy()
    Beff = _split(c["B"])
    Geta = oracle.cox_nll_grad_eta(c["time"], c["status"], Xo @ Beff)
    tol = _grad_tol(Xo, Geta, Xo.T @ Geta) + 1e-6

    def fd(j, b, h):
        Bp, Bm = Beff.copy(), Beff.copy()
        Bp[j, b] += h
        Bm[j, b] -= h
        return (oracle.cox_nll(c["time"], c["status"], Xo @ Bp)[b]
                - oracle.cox_nll(c["time"], c["status"], Xo @ Bm)[b]) / (2 * h)

    rng = np.random.default_rng(0)
    h = 1e-3
    for _ in range(8):
        j, b = int(rng.integers(12)), int(rng.integers(4))
        richardson = (4.0 * fd(j, b, h) - fd(j, b, 2 * h)) / 3.0      # error O(h^4)
        assert abs(g[j, b] - richardson) <= tol[j, b], (j, b, g[j, b], richardson, tol[j, b])


def test_heavy_ties_and_no_events_columns(lib):
    import torch
    c, X, B, t, s, Xo = _case(5_000, 8, 3, seed=52, n_times=7)      # 7 distinct times
    nll = binding.cox_nll(B, X, t, s)
    ref = oracle.cox_nll(c["time"], c["status"], Xo @ _split(c["B"]))
    np.testing.assert_allclose(nll.cpu().numpy(), ref, rtol=1e-7)
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
    """N = 2^22, p = 256, C = 64: NLL of 4 columns and their gradient
    columns against the oracle at the split B, with the bounds above."""
    import torch
    n, p, C = 1 << 22, 256, 64
    c = synth.nll_cohort(n, p, C, seed=5, n_times=5000)
    X, B, t, s = _to_gpu(c)
    Bt = B.clone().requires_grad_(True)
    nll = binding.cox_nll(Bt, X, t, s)
    (g,) = torch.autograd.grad(nll.sum(), Bt)
    Xo = X.float().cpu().numpy().astype(np.float64)
    Beff = _split(c["B"])
    cols = [0, 17, 42, 63]
    eta = Xo @ Beff[:, cols]
    ref = oracle.cox_nll(c["time"], c["status"], eta)
    np.testing.assert_allclose(nll.detach().cpu().numpy()[cols], ref, rtol=1e-7)
    ge = oracle.cox_nll_grad_eta(c["time"], c["status"], eta)
    gref = Xo.T @ ge                                         # (p, 4)
    gg = g.cpu().numpy()[:, cols]
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    tol = _grad_tol(Xo, ge, gref) + _accumulation_bound(Xo, ge, n_sm)
    assert np.all(np.abs(gg - gref) <= tol)
    # the bound is not loose by orders of magnitude: the largest error uses
    # a fair share of it
    assert np.max(np.abs(gg - gref) / tol) > 0.02
