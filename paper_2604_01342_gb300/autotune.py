"""Launch-shape autotuner: chunk length, walker lanes, path.

The chunk length C trades the inter-chunk work (checkpoints and, on the chunk-GEMM path,
GEMMs that shrink as 1/C) against the work inside chunks (state walk or pair kernels that
grow with C).  On the state walk the lanes of one walker (the threads per group of marks:
8 or 16 lanes with one mark each, or 32) decide how many chunks a warp walks at once; on
the mark-major path the segment length decides how many (segment, mark) work items there
are.  The best choice depends on M, the decay mode, the sequence lengths and the GPU, so it
is measured: every candidate runs the caller's own call (log-likelihood + gradient) a few
times, timed with CUDA events on the current stream, and the fastest is kept per problem
shape and GPU, in memory and in a JSON file (``$HAWKES_GB300_TUNE_CACHE``, else
``~/.cache/hawkes_gb300/autotune.json``; ``cache_path=None`` or an empty variable turns the
file off), so that a later process reuses it.

    best = tune(t, c, T, mu, alpha, beta)        # {"path": p, "chunk": C, "walk_lanes": W, ...}
    ll, dmu, dal, dbe = torch_api.loglik_grad(t, c, T, mu, alpha, beta, chunk=best["chunk"],
                                              path=best["path"], walk_lanes=best["walk_lanes"])
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import binding as _b
from . import torch_api as _t

WALK_CHUNKS = (32, 64, 96, 128, 192, 256)
GEMM_CHUNKS = (128, 160, 192, 224, 256)
MARK_SEGMENTS = (0, 1 << 18, 1 << 19, 1 << 20)   # 0 = the library's choice
WALK_MAX_M_GRAD = 64            # largest M the state walk takes with the gradient

_cache: dict = {}
_lock = threading.Lock()
_DEFAULT = object()


def default_cache_path():
    env = os.environ.get("HAWKES_GB300_TUNE_CACHE")
    if env is not None:
        return env or None
    return os.path.join(os.path.expanduser("~"), ".cache", "hawkes_gb300", "autotune.json")


def _walk_lanes(M: int):
    return [w for w in (8, 16, 32) if w == 32 or M <= w]


def _candidates(M: int, shared: bool, B: int):
    """(path, chunk, walk_lanes) triples that apply to the shape."""
    out = []
    if M <= WALK_MAX_M_GRAD:
        out += [(1, c, w) for c in WALK_CHUNKS for w in _walk_lanes(M)]
    if shared and M > 1 and B == 1:
        out += [(2, c, 0) for c in GEMM_CHUNKS]
    if not shared and B == 1 and M > WALK_MAX_M_GRAD:
        out += [(3, c, 0) for c in MARK_SEGMENTS]
    return out


def _key(device, N: int, B: int, M: int, shared: bool) -> str:
    prop = torch.cuda.get_device_properties(device)
    return f"{prop.name}|sms={prop.multi_processor_count}|N={N}|B={B}|M={M}|shared={int(shared)}"


def _load_file(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_file(path, key, value):
    """Adds one entry to the JSON cache (read-merge-replace, so concurrent writers lose at
    most their own entry)."""
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        data = _load_file(path)
        data[key] = value
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass                                            # a read-only home: memory cache only


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
         candidates=None, cache_path=_DEFAULT, support: bool = False) -> dict:
    """Fastest (path, chunk, walk lanes) for this problem shape on this GPU; cached in memory
    and in the JSON file.  ``candidates``: (path, chunk, walk_lanes) triples to try instead
    of the default set (results with explicit candidates are not written to the file)."""
    M = mu.shape[-1]
    B = 1 if offsets is None else offsets.shape[0] - 1
    if offsets is None:
        shared = _t._shared(beta.reshape(-1), M, beta_shared)
    else:
        shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == B and M != 1)
    key = _key(t.device, int(t.shape[0]), B, M, shared)
    path_file = default_cache_path() if cache_path is _DEFAULT else cache_path
    with _lock:
        if candidates is None and key in _cache:
            return _cache[key]
    if candidates is None and path_file:
        hit = _load_file(path_file).get(key)
        if hit is not None:
            with _lock:
                _cache[key] = hit
            return hit
    cands = [tuple(x) + (0,) * (3 - len(x)) for x in candidates] if candidates is not None \
        else _candidates(M, shared, B)
    if not cands:
        raise ValueError("no candidate configuration for this problem")
    timings = {}
    for path, chunk, lanes in cands:
        if offsets is None:
            fn = lambda: _t.loglik_grad(t, c, T, mu, alpha, beta, beta_shared=shared,  # noqa: E731
                                        chunk=chunk, path=path, check=False, walk_lanes=lanes,
                                        support=support)
        else:
            fn = lambda: _t.loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta,  # noqa: E731
                                               beta_shared=shared, chunk=chunk, path=path,
                                               check=False, walk_lanes=lanes)
        try:
            timings[(path, chunk, lanes)] = _time(fn, reps, t.device)
        except _b.HawkesError:
            continue                                   # e.g. a path that rejects this shape
    if not timings:
        raise ValueError("no candidate configuration ran")
    (path, chunk, lanes), ms = min(timings.items(), key=lambda kv: kv[1])
    best = {"path": path, "chunk": chunk, "walk_lanes": lanes, "ms": ms,
            "timings": {f"path{p}_chunk{c}_lanes{w}": round(v, 4)
                        for (p, c, w), v in timings.items()}}
    if candidates is None:
        with _lock:
            _cache[key] = best
        if path_file:
            _store_file(path_file, key, best)
    return best
