"""One sequence split over ranks (paper, Section 3.3: consecutive batches depend on each
other only through one carried state).

CPU: world_size 2 and 3 gloo process groups run the exchange of
paper_2604_01342_gb300.sharded with the FP64 oracle as the per-slice backend (test
infrastructure), and must reproduce the whole-sequence oracle.
GPU: the CUDA slice entry points (aggregate, slice log-likelihood with a carried state)
on emulated ranks (slices run one after another on one GPU, exchange on the host) must
match the oracle and the single-call result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2604_01342_gb300 import sharded, synth


class OracleSlices:
    """Per-slice backend on the FP64 oracle (test infrastructure only)."""

    def aggregate(self, t, c, M, beta, shared, t_next):
        b = beta.double().reshape(-1).numpy()
        b = np.full(M, b[0]) if shared else b
        return oracle.slice_aggregate(t.numpy(), c.numpy(), M, b, t_next)

    def loglik_grad(self, t, c, T, mu, alpha, beta, shared, cS, cG, base):
        M = mu.shape[0]
        b = beta.double().reshape(-1).numpy()
        b = np.full(M, b[0]) if shared else b
        r = oracle.loglik_grad_carry(t.numpy(), c.numpy(), T, mu.double().numpy(),
                                     alpha.double().numpy(), b, cS, cG, base)
        db = np.array([r["dbeta"].sum()]) if shared else r["dbeta"]
        return (torch.tensor(r["ll"], dtype=torch.float64), torch.from_numpy(r["dmu"]),
                torch.from_numpy(r["dalpha"]), torch.from_numpy(db))


def _problem(shared):
    return synth.random_problem(5, 900, 77 if shared else 78, shared)


def _cuts(n, world, seed):
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.choice(np.arange(1, n), size=world - 1, replace=False))
    return [0, *inner.tolist(), n]


def _worker(rank, world, port, shared, cuts, empty_rank, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem(shared)
        a, b = cuts[rank], cuts[rank + 1]
        if rank == empty_rank:
            a = b = cuts[rank]
        t = torch.from_numpy(p.t[a:b].copy())
        c = torch.from_numpy(p.c[a:b].copy())
        beta = torch.tensor(p.beta[:1] if shared else p.beta)
        out = sharded.loglik_grad_sharded(t, c, p.T, torch.from_numpy(p.mu),
                                          torch.from_numpy(p.alpha), beta, beta_shared=shared,
                                          backend=OracleSlices())
        q.put((rank, [x.numpy().copy() for x in out]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,shared,empty", [(2, False, -1), (3, True, -1), (3, False, 1)])
def test_gloo_exchange_matches_whole_sequence(world, shared, empty):
    p = _problem(shared)
    cuts = _cuts(p.N, world, world * 10 + shared)
    if empty >= 0:
        # rank `empty` gets no events: its slice is merged into the next one
        cuts = cuts.copy()
        cuts[empty + 1] = cuts[empty]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shared, cuts, -1, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ref = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    ref_db = np.array([ref["dbeta"].sum()]) if shared else ref["dbeta"]
    for r in range(world):
        ll, dmu, dal, dbe = results[r]
        assert float(ll) == pytest.approx(ref["ll"], rel=1e-12)
        np.testing.assert_allclose(dmu, ref["dmu"], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(dal, ref["dalpha"], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(dbe, ref_db, rtol=1e-9, atol=1e-9)


def test_exchange_carries_is_the_state_recurrence():
    # carries built from slice aggregates equal the state the oracle's recurrence reaches
    p = synth.random_problem(4, 400, 5, False)
    cuts = [0, 120, 121, 300, 400]
    firsts = [float(p.t[a]) for a in cuts[:-1]]
    aS, aG = [], []
    for r in range(len(cuts) - 1):
        a, b = cuts[r], cuts[r + 1]
        nxt = sharded.next_first(firsts, r)
        s, g = oracle.slice_aggregate(p.t[a:b], p.c[a:b], 4, p.beta, nxt if nxt else p.t[b - 1])
        aS.append(s); aG.append(g)
    cS, cG = sharded.exchange_carries(firsts, aS, aG, p.beta)
    # brute force: S at the first event of each slice from all earlier events
    for r, a in enumerate(cuts[:-1]):
        S = np.zeros(4); G = np.zeros(4)
        for l in range(a):
            x = p.t[a] - p.t[l]
            S[p.c[l]] += np.exp(-p.beta[p.c[l]] * x)
            G[p.c[l]] += x * np.exp(-p.beta[p.c[l]] * x)
        np.testing.assert_allclose(cS[r], S, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(cG[r], G, rtol=1e-12, atol=1e-14)


@pytest.mark.gpu
@pytest.mark.parametrize("m,shared,path,nslices", [(8, False, 1, 3), (48, True, 2, 4),
                                                   (64, True, 1, 2)])
def test_gpu_slices_match_oracle(m, shared, path, nslices):
    from helpers import assert_close, f32, gpu_run, maxnorm_rel, oracle_ref, rel_err
    p = synth.random_problem(m, 6000, 90 + m, shared)
    dev = torch.device("cuda")
    cuts = _cuts(p.N, nslices, m)
    firsts = [float(p.t[a]) for a in cuts[:-1]]
    be = torch.tensor(p.beta[:1] if shared else p.beta, dtype=torch.float32, device=dev)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    al = torch.tensor(p.alpha, dtype=torch.float32, device=dev)
    back = sharded.CudaSlices()
    aS, aG, parts = [], [], []
    for r in range(nslices):
        a, b = cuts[r], cuts[r + 1]
        t = torch.from_numpy(p.t[a:b].copy()).to(dev)
        c = torch.from_numpy(p.c[a:b].copy()).to(dev)
        nxt = sharded.next_first(firsts, r)
        s, g = back.aggregate(t, c, m, be, shared, nxt) if nxt else (np.zeros(m), np.zeros(m))
        aS.append(s); aG.append(g)
    cS, cG = sharded.exchange_carries(firsts, aS, aG, f32(p.beta[:1] if shared else p.beta)
                                      if not shared else np.full(m, f32(p.beta[:1])[0]))
    tot = None
    for r in range(nslices):
        a, b = cuts[r], cuts[r + 1]
        t = torch.from_numpy(p.t[a:b].copy()).to(dev)
        c = torch.from_numpy(p.c[a:b].copy()).to(dev)
        carry = (cS[r], cG[r]) if r > 0 else (None, None)
        out = back.loglik_grad(t, c, p.T, mu, al, be, shared, carry[0], carry[1], r == 0)
        out = [x.cpu().numpy() for x in out]
        tot = out if tot is None else [x + y for x, y in zip(tot, out)]
    got = {"ll": float(tot[0]), "dmu": tot[1], "dalpha": tot[2], "dbeta": tot[3]}
    assert_close(got, oracle_ref(p), what=f"{nslices} slices")
    whole = gpu_run(p, path=path)
    assert rel_err(got["ll"], whole["ll"]) < 1e-6
    assert maxnorm_rel(got["dalpha"], whole["dalpha"]) < 1e-4
