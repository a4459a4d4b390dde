"""One long event sequence split over several ranks (one GPU each).

The paper notes that a batch of events depends on the events before it only through one
carried state (Section 3.3), and that batches could therefore be spread over GPUs.  Here
rank r holds the contiguous slice r of the events (in time order).  The exchange is:

1. every rank computes its slice aggregate at the first event time of the next non-empty
   slice: ``agg_S[j] = sum_{l in slice, c_l = j} exp(-beta_j (t_next - t_l))`` and ``agg_G``
   (the same times ``t_next - t_l``) -- ``hawkes_slice_aggregate``;
2. one all-gather of the aggregates and first event times; every rank then scans them in
   order (``exchange_carries``):
       S_{r+1} = d_r S_r + agg_S_r,   G_{r+1} = d_r (G_r + D_r S_r) + agg_G_r,
       D_r = t_first[r+1] - t_first[r],  d_r = exp(-beta D_r);
3. every rank computes its slice's log-likelihood and gradient starting from its carried
   state (``hawkes_loglik_grad_slice``; rank 0 alone adds the ``-T sum(mu)`` term);
4. one all-reduce sums L and the gradients.

The slice computations go through a backend object; ``CudaSlices`` (the default) runs the
library's kernels on the rank's GPU.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.distributed as dist

from . import binding as _b
from . import torch_api as _t


def exchange_carries(firsts, aggs_S, aggs_G, beta):
    """Carried states (S, G) at the first event of every slice, in FP64.

    firsts[r] is the first event time of slice r (None if the slice is empty); aggs_*[r]
    its aggregate at the first event time of the next non-empty slice (ignored for empty
    slices and for the last non-empty one).  Returns lists of arrays (None for empty
    slices); the first non-empty slice gets zeros."""
    beta = np.asarray(beta, dtype=np.float64)
    M = beta.shape[0]
    S, G = np.zeros(M), np.zeros(M)
    out_S, out_G = [None] * len(firsts), [None] * len(firsts)
    prev = None
    for r, tf in enumerate(firsts):
        if tf is None:
            continue
        if prev is not None:
            D = tf - firsts[prev]
            d = np.exp(-beta * D)
            G = d * (G + D * S) + np.asarray(aggs_G[prev], dtype=np.float64)
            S = d * S + np.asarray(aggs_S[prev], dtype=np.float64)
        out_S[r], out_G[r] = S.copy(), G.copy()
        prev = r
    return out_S, out_G


def next_first(firsts, r):
    """First event time of the next non-empty slice after r, or None."""
    for q in range(r + 1, len(firsts)):
        if firsts[q] is not None:
            return firsts[q]
    return None


class CudaSlices:
    """Slice computations on the current GPU through the C ABI."""

    def aggregate(self, t, c, M, beta, shared, t_next):
        dev = t.device
        opts = _b.make_opts(shared)
        ws = _t._workspace(256, dev)
        aS = torch.empty(M, dtype=torch.float32, device=dev)
        aG = torch.empty(M, dtype=torch.float32, device=dev)
        be = beta.detach().contiguous().to(torch.float32).reshape(-1)
        _b.hawkes_slice_aggregate(t.data_ptr(), c.data_ptr(), t.shape[0], M, be.data_ptr(), opts,
                                  float(t_next), ws.data_ptr(), ws.numel(), aS.data_ptr(),
                                  aG.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
        return aS.double().cpu().numpy(), aG.double().cpu().numpy()

    def loglik_grad(self, t, c, T, mu, alpha, beta, shared, carry_S, carry_G, base_term):
        dev = t.device
        t, c, mu, alpha, beta = _t._prep(t, c, mu, alpha, beta)
        N, M = t.shape[0], mu.shape[0]
        opts = _b.make_opts(shared)
        nbytes = _b.hawkes_workspace_size(N, M, 1, True, opts)
        ws = _t._workspace(nbytes, dev)
        ll = torch.empty((), dtype=torch.float64, device=dev)
        dmu = torch.empty(M, dtype=torch.float32, device=dev)
        dal = torch.empty(M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(1 if shared else M, dtype=torch.float32, device=dev)
        cS = cG = None
        if carry_S is not None:
            cS = torch.as_tensor(carry_S, dtype=torch.float32, device=dev).contiguous()
            cG = torch.as_tensor(carry_G, dtype=torch.float32, device=dev).contiguous()
        s = torch.cuda.current_stream(dev).cuda_stream
        _b.hawkes_loglik_grad_slice(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                                    alpha.data_ptr(), beta.data_ptr(), opts,
                                    cS.data_ptr() if cS is not None else None,
                                    cG.data_ptr() if cG is not None else None, base_term,
                                    ws.data_ptr(), ws.numel(), ll.data_ptr(), dmu.data_ptr(),
                                    dal.data_ptr(), dbe.data_ptr(), s)
        rc = _b.hawkes_last_device_status(ws.data_ptr(), s)
        if rc:
            raise _b.HawkesError(rc, "device check")
        return ll.double(), dmu.double(), dal.double(), dbe.double()


def _beta_vector(beta, M, shared):
    b = beta.detach().double().reshape(-1).cpu().numpy()
    return np.full(M, b[0]) if shared else b


def loglik_grad_sharded(t_local, c_local, T, mu, alpha, beta, beta_shared=None, group=None,
                        backend=None):
    """L and gradients of a sequence whose events are split over the ranks of ``group``
    (rank r holds the r-th contiguous slice).  Every rank returns the same totals
    (float64 tensors on the device of ``t_local``)."""
    backend = backend or CudaSlices()
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    dev = t_local.device
    M = mu.shape[0]
    shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == 1 and M != 1)
    bvec = _beta_vector(beta, M, shared)
    n = t_local.shape[0]
    first = float(t_local[0].item()) if n > 0 else math.nan
    # 1 + 2: first event times, then aggregates at the next slice's first time
    ft = torch.tensor([first], dtype=torch.float64, device=dev)
    fts = [torch.empty_like(ft) for _ in range(world)]
    dist.all_gather(fts, ft, group=group)
    firsts = [None if math.isnan(float(x.item())) else float(x.item()) for x in fts]
    t_next = next_first(firsts, rank)
    if n > 0 and t_next is not None:
        aS, aG = backend.aggregate(t_local, c_local, M, beta, shared, t_next)
    else:
        aS, aG = np.zeros(M), np.zeros(M)
    agg = torch.tensor(np.concatenate([aS, aG]), dtype=torch.float64, device=dev)
    aggs = [torch.empty_like(agg) for _ in range(world)]
    dist.all_gather(aggs, agg, group=group)
    aggs = [a.cpu().numpy() for a in aggs]
    carries_S, carries_G = exchange_carries(firsts, [a[:M] for a in aggs], [a[M:] for a in aggs],
                                            bvec)
    # 3: this slice from its carried state (the first non-empty slice starts from zero)
    cS, cG = carries_S[rank], carries_G[rank]
    if cS is not None and not np.any(cS) and not np.any(cG):
        cS = cG = None
    base = rank == 0
    ll, dmu, dal, dbe = backend.loglik_grad(t_local, c_local, T, mu, alpha, beta, shared, cS, cG,
                                            base)
    # 4: sum over ranks
    flat = torch.cat([ll.reshape(1).to(dev), dmu.reshape(-1).to(dev), dal.reshape(-1).to(dev),
                      dbe.reshape(-1).to(dev)]).to(torch.float64)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    nb = dbe.numel()
    return (flat[0], flat[1:1 + M], flat[1 + M:1 + M + M * M].reshape(M, M),
            flat[1 + M + M * M:1 + M + M * M + nb])
