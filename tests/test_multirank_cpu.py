"""Multi-rank algebra on CPU ranks (gloo, world size 2).

The risk-set pass shards over contiguous ranges of time-sorted subjects with
one small exchange per coordinate: an exclusive scan of the ranks' tuple
totals (an all-gather of 3 or 6 numbers) seeds each rank's prefix, the
Fine-Gray suffix uses the grand total from the same all-gather, and an
all-reduce of (g', g'', l) finishes the coordinate.  A tie group belongs to
the rank that holds its last subject.  This file checks that algebra,
emulated with numpy on gloo ranks, against the single-process oracle, and
checks the bench's cross-rank aggregation (max of times, sum of work).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2204_08183_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_terms(model, t, st, X, beta, j, rank, world):
    """(l, g', g'') for coordinate j with subjects split across ranks."""
    n = t.shape[0]
    bounds = np.linspace(0, n, world + 1).astype(int)
    lo, hi = bounds[rank], bounds[rank + 1]
    eta = X @ beta
    e = np.exp(eta[lo:hi])
    x = X[lo:hi, j]
    gend = oracle.tie_groups(t)
    d = oracle.group_counts(gend, st, 1).astype(float)
    if model == "fg":
        W, Gk, _ = oracle.fg_weights(t, st)
        w = W[lo:hi]
    else:
        w = np.zeros(hi - lo)
    comps = np.stack([e, e * x, e * x * x, w * e, w * e * x, w * e * x * x])
    local_total = comps.sum(axis=1)
    allt = [torch.zeros(6, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allt, torch.from_numpy(local_total))
    allt = torch.stack(allt).numpy()
    T = allt[:rank].sum(axis=0)             # exclusive prefix over ranks
    grand = allt.sum(axis=0)
    pre = np.cumsum(comps, axis=1)
    mine = (gend >= lo) & (gend < hi)
    g1 = g2 = l = 0.0
    for k in np.flatnonzero(mine):
        P = T + pre[:, gend[k] - lo]
        den, n1, n2 = P[0], P[1], P[2]
        if model == "fg":
            Q = grand[3:] - P[3:]            # competing suffix strictly after the group end
            den, n1, n2 = den + Gk[k] * Q[0], n1 + Gk[k] * Q[1], n2 + Gk[k] * Q[2]
        G, H = n1 / den, n2 / den
        g1 += d[k] * G
        g2 += d[k] * (H - G * G)
        l += d[k] * np.log(den)
    lin_local = (st[lo:hi] == 1) @ eta[lo:hi]
    dtx_local = (st[lo:hi] == 1) @ x
    part = torch.tensor([g1, g2, l, lin_local, dtx_local], dtype=torch.float64)
    dist.all_reduce(part)
    g1, g2, l, lin, dtx = part.tolist()
    return lin - l, dtx - g1, -g2


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for model, comp in [("cox", 0.0), ("fg", 0.25)]:
            dd = synth.cohort_small(4001, 3, seed=7, n_times=150, censor_frac=0.3, competing_frac=comp)
            got = [_shard_terms(model, dd["time"], dd["status"], dd["X"], dd["beta"], j, rank, world)
                   for j in range(3)]
            out[model] = got
        # a sharded CCD sweep: every rank takes the same Newton step
        dd = synth.cohort_small(3001, 3, seed=8, n_times=100, censor_frac=0.3)
        beta = np.zeros(3)
        width = np.ones(3)
        for _ in range(3):
            for j in range(3):
                _, g1, g2 = _shard_terms("cox", dd["time"], dd["status"], dd["X"], beta, j, rank, world)
                step = oracle.newton_step(beta[j], g1, g2, "l2", 1.0)
                applied, width[j] = oracle.trust_region(step, width[j])
                beta[j] += applied
        out["beta"] = beta
        # the bench's aggregation: max over ranks of the timed region, sum of work
        ms = torch.tensor([10.0 + rank], dtype=torch.float64)
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        work = torch.tensor([5.0 * (rank + 1)], dtype=torch.float64)
        dist.all_reduce(work, op=dist.ReduceOp.SUM)
        out["agg"] = (ms.item(), work.item())
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_sharded_exchange_matches_single_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for model, comp in [("cox", 0.0), ("fg", 0.25)]:
        dd = synth.cohort_small(4001, 3, seed=7, n_times=150, censor_frac=0.3, competing_frac=comp)
        # the rank boundary falls inside a tie group (owned by rank 1, which
        # holds its last subject): the case the exchange must get right
        cut = np.linspace(0, 4001, world + 1).astype(int)[1]
        assert dd["time"][cut - 1] == dd["time"][cut]
        for j in range(3):
            ref = oracle.model_terms(model, dd["time"], dd["status"], dd["X"], dd["beta"], j)
            for r in range(world):
                np.testing.assert_allclose(res[r][model][j], ref, rtol=1e-11)
    dd = synth.cohort_small(3001, 3, seed=8, n_times=100, censor_frac=0.3)
    ref = oracle.ccd_fit("cox", dd["time"], dd["status"], dd["X"], "l2", 1.0, tol=0.0, max_sweeps=3)
    for r in range(world):
        np.testing.assert_allclose(res[r]["beta"], ref["beta"], rtol=1e-10)
        assert res[r]["agg"] == (11.0, 15.0)
