"""Chunk-size (and path) autotuner.

The chunk length C trades the inter-chunk work (checkpoints and, on the chunk-GEMM path,
GEMMs that shrink as 1/C) against the work inside chunks (state walk or pair kernels that
grow with C).  The best C depends on M, the decay mode, the sequence lengths and the GPU,
so it is measured: every candidate runs the caller's own call (log-likelihood + gradient)
a few times, timed with CUDA events on the current stream, and the fastest is kept per
problem shape.  Where both the state walk and the chunk-GEMM path apply (one shared decay,
small M), the path is tuned too.

    best = tune(t, c, T, mu, alpha, beta)                 # {"chunk": C, "path": p, "ms": ...}
    ll, dmu, dal, dbe = torch_api.loglik_grad(t, c, T, mu, alpha, beta, chunk=best["chunk"],
                                              path=best["path"])
"""
from __future__ import annotations

import torch

from . import binding as _b
from . import torch_api as _t

WALK_CHUNKS = (32, 64, 96, 128, 192, 256)
GEMM_CHUNKS = (128, 160, 192, 224, 256)
WALK_MAX_M_GRAD = 64            # largest M the state walk takes with the gradient

_cache: dict = {}


def _candidates(M: int, shared: bool):
    out = []
    if M <= WALK_MAX_M_GRAD:
        out += [(1, c) for c in WALK_CHUNKS]
    if shared and M > 1:
        out += [(2, c) for c in GEMM_CHUNKS]
    return out


def _time(fn, reps: int, device) -> float:
    fn()                                               # warm-up (also sets kernel attributes)
    s = torch.cuda.current_stream(device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune(t, c, T, mu, alpha, beta, beta_shared=None, offsets=None, reps: int = 3,
         candidates=None) -> dict:
    """Fastest (path, chunk) for this problem shape; cached by (N, B, M, decay mode)."""
    M = mu.shape[-1]
    B = 1 if offsets is None else offsets.shape[0] - 1
    if offsets is None:
        shared = _t._shared(beta.reshape(-1), M, beta_shared)
    else:
        shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == B and M != 1)
    key = (t.device.index, int(t.shape[0]), B, M, shared)
    if key in _cache:
        return _cache[key]
    cands = list(candidates) if candidates is not None else _candidates(M, shared)
    if not cands:
        raise ValueError("no candidate configuration for this problem")
    timings = {}
    for path, chunk in cands:
        if offsets is None:
            fn = lambda: _t.loglik_grad(t, c, T, mu, alpha, beta, beta_shared=shared,  # noqa: E731
                                        chunk=chunk, path=path, check=False)
        else:
            fn = lambda: _t.loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta,  # noqa: E731
                                               beta_shared=shared, chunk=chunk, path=path,
                                               check=False)
        try:
            timings[(path, chunk)] = _time(fn, reps, t.device)
        except _b.HawkesError:
            continue                                   # e.g. a path that rejects this shape
    if not timings:
        raise ValueError("no candidate configuration ran")
    (path, chunk), ms = min(timings.items(), key=lambda kv: kv[1])
    best = {"path": path, "chunk": chunk, "ms": ms,
            "timings": {f"path{p}_chunk{c}": round(v, 4) for (p, c), v in timings.items()}}
    _cache[key] = best
    return best
