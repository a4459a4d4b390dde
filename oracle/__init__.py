"""FP64 CPU oracle for the Hawkes log-likelihood and its gradient.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library
(``paper_2604_01342_gb300``) never does.  The arithmetic lives in plain C
(``hawkes_oracle.c``, FP64, sequential, one loop over events); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.

Conventions: marks are 0-based; ``alpha[i, j]`` is the influence of source
mark ``j`` on target mark ``i`` (paper, Section 2, Eq. hawkes_excitation);
``beta`` is a per-source decay vector, a shared decay being the all-equal
vector.  Gradients are of L itself (not of -L/N).

What pins each function (see ``tests/test_oracle_pins.py``):
  * ``loglik_grad``: brute-force O(N^2 M) double sum of Eq. hawkes_excitation,
    quadrature of the compensator integral, the Poisson closed form at
    alpha = 0, hand-derived one- and two-event closed forms, central finite
    differences, the Euler identity for the 1-homogeneous (mu, alpha), time
    shift / rescale / relabelling invariances.
  * ``grad_adjoint``: equals ``loglik_grad`` (two derivations) and FD.
  * ``paper_grad_shared``: the paper's R/K/L form, equal to the others at
    small T.
  * ``loglik_grad_multi`` (several decay kernels): equals ``loglik_grad`` at K = 1; its
    intensity against the brute-force double sum over kernels and pairs; two kernels
    with one decay equal one kernel with the summed matrix; central finite differences;
    quadrature of the compensator.
  * ``loglik_grad_support`` (lazy per-component form, gradient on alpha's support): equals
    ``loglik_grad`` on L, dmu, dbeta and the support entries of dalpha for sparse alpha,
    and in every entry for a fully supported alpha; L against the brute-force intensity
    and the closed-form compensator; ties and times near 1e7.
  * ``chunk_table``, ``bucket_order`` (integer passes): numpy counting and stable sorting.
  * ``condition``: a brute-force double sum with distinct per-source decays, and planted
    source/target slips that it rejects.
  * ``condition_multi``: equals ``condition`` at K = 1; a brute-force double sum over
    kernels and event pairs; bounds every term it sums (|dbeta| <= its scale).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hawkes_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "unsorted times", 3: "mark out of range",
          4: "time outside [0, T]", 5: "parameter outside its domain", 6: "intensity <= 0"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle: {STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math: IEEE FP64 throughout)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
            p = ctypes.c_void_p
            lib.oracle_loglik_grad.argtypes = [i64, p, p, d, i32, p, p, p, p, p, p, p, p]
            lib.oracle_grad_adjoint.argtypes = [i64, p, p, d, i32, p, p, p, p, p, p, p]
            lib.oracle_paper_grad_shared.argtypes = [i64, p, p, d, i32, p, p, d, p, p, p, p]
            lib.oracle_loglik_grad_varlen.argtypes = [p, p, p, i32, p, i32, p, p, p, p, p, p, p]
            lib.oracle_mark_counts.argtypes = [i64, p, i32, p]
            lib.oracle_condition.argtypes = [i64, p, p, d, i32, p, p, p, p, p]
            lib.oracle_loglik_grad_support.argtypes = [i64, p, p, d, i32, p, p, p, p, p, p, p]
            lib.oracle_loglik_grad_support.restype = ctypes.c_int
            lib.oracle_chunk_table.argtypes = [i32, p, i32, p, p]
            lib.oracle_support_rows.argtypes = [i32, p, i32, p, p]
            lib.oracle_support_rows.restype = ctypes.c_int
            lib.oracle_mark_sort.argtypes = [i64, p, i32, i64, p, p]
            lib.oracle_mark_sort.restype = ctypes.c_int
            lib.oracle_chunk_table.restype = ctypes.c_int
            lib.oracle_bucket_order.argtypes = [i64, p, i32, i32, i32, p, p]
            lib.oracle_bucket_order.restype = ctypes.c_int
            lib.oracle_loglik_grad_carry.argtypes = [i64, p, p, d, i32, p, p, p, p, p,
                                                     ctypes.c_int, p, p, p, p, p]
            lib.oracle_loglik_grad_carry.restype = ctypes.c_int
            lib.oracle_slice_aggregate.argtypes = [i64, p, p, i32, p, d, p, p]
            lib.oracle_loglik_grad_multi.argtypes = [i64, p, p, d, i32, i32, p, p, p, p, p, p, p, p]
            lib.oracle_loglik_grad_multi.restype = ctypes.c_int
            lib.oracle_condition_multi.argtypes = [i64, p, p, d, i32, i32, p, p, p, p, p]
            lib.oracle_condition_multi.restype = ctypes.c_int
            lib.oracle_slice_aggregate.restype = ctypes.c_int
            lib.oracle_condition.restype = ctypes.c_int
            for f in (lib.oracle_loglik_grad, lib.oracle_grad_adjoint, lib.oracle_paper_grad_shared,
                      lib.oracle_loglik_grad_varlen, lib.oracle_mark_counts):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(t, c, mu, alpha, beta):
    t = np.ascontiguousarray(t, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    M = mu.shape[-1]
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    if beta.ndim == 0 or beta.shape[-1] != M:
        beta = np.broadcast_to(beta.reshape(beta.shape + (1,) if beta.ndim else (1,)),
                               mu.shape)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    return t, c, mu, alpha, beta, M


def loglik_grad(t, c, T, mu, alpha, beta, want_grad=True, want_lam=False):
    """L and (dmu, dalpha, dbeta per source) in one FP64 forward pass."""
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    N = t.shape[0]
    ll = np.zeros(1)
    lam = np.zeros(N) if want_lam else None
    dmu = np.zeros(M) if want_grad else None
    dal = np.zeros((M, M)) if want_grad else None
    dbe = np.zeros(M) if want_grad else None
    rc = _load().oracle_loglik_grad(N, _ptr(t), _ptr(c), float(T), M, _ptr(mu), _ptr(alpha),
                                    _ptr(beta), _ptr(ll), _ptr(lam), _ptr(dmu), _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    out = {"ll": float(ll[0])}
    if want_grad:
        out.update(dmu=dmu, dalpha=dal, dbeta=dbe)
    if want_lam:
        out["lam"] = lam
    return out


def loglik(t, c, T, mu, alpha, beta) -> float:
    return loglik_grad(t, c, T, mu, alpha, beta, want_grad=False)["ll"]


def grad_adjoint(t, c, T, mu, alpha, beta):
    """Reverse-adjoint gradient (stores all N states: small N only)."""
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    N = t.shape[0]
    ll, dmu, dal, dbe = np.zeros(1), np.zeros(M), np.zeros((M, M)), np.zeros(M)
    rc = _load().oracle_grad_adjoint(N, _ptr(t), _ptr(c), float(T), M, _ptr(mu), _ptr(alpha),
                                     _ptr(beta), _ptr(ll), _ptr(dmu), _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    return {"ll": float(ll[0]), "dmu": dmu, "dalpha": dal, "dbeta": dbe}


def paper_grad_shared(t, c, T, mu, alpha, gamma):
    """The paper's R/K/L gradient formulas for one shared decay (small T only)."""
    t, c, mu, alpha, _, M = _prep(t, c, mu, alpha, np.ones(np.shape(mu)))
    N = t.shape[0]
    ll, dmu, dal, dg = np.zeros(1), np.zeros(M), np.zeros((M, M)), np.zeros(1)
    rc = _load().oracle_paper_grad_shared(N, _ptr(t), _ptr(c), float(T), M, _ptr(mu),
                                          _ptr(alpha), float(gamma), _ptr(ll), _ptr(dmu),
                                          _ptr(dal), _ptr(dg))
    if rc:
        raise OracleError(rc)
    return {"ll": float(ll[0]), "dmu": dmu, "dalpha": dal, "dbeta": float(dg[0])}


def loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta, want_grad=True):
    """Per-sequence L and gradients for B independent sequences."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = offsets.shape[0] - 1
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(B)
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    ll = np.zeros(B)
    dmu = np.zeros((B, M)) if want_grad else None
    dal = np.zeros((B, M, M)) if want_grad else None
    dbe = np.zeros((B, M)) if want_grad else None
    rc = _load().oracle_loglik_grad_varlen(_ptr(t), _ptr(c), _ptr(offsets), B, _ptr(T), M,
                                           _ptr(mu), _ptr(alpha), _ptr(beta), _ptr(ll),
                                           _ptr(dmu), _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    out = {"ll": ll}
    if want_grad:
        out.update(dmu=dmu, dalpha=dal, dbeta=dbe)
    return out


def mark_counts(c, M):
    c = np.ascontiguousarray(c, dtype=np.int32)
    out = np.zeros(M, dtype=np.int64)
    rc = _load().oracle_mark_counts(c.shape[0], _ptr(c), M, _ptr(out))
    if rc:
        raise OracleError(rc)
    return out


def loglik_grad_support(t, c, T, mu, alpha, beta):
    """L and gradients by the lazy per-component form (cost per event: the nonzeros of its
    row of alpha).  dalpha is the gradient on alpha's support (alpha != 0), 0 elsewhere;
    L, dmu and dbeta are exact for any alpha."""
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    ll, dmu, dal, dbe = np.zeros(1), np.zeros(M), np.zeros((M, M)), np.zeros(M)
    rc = _load().oracle_loglik_grad_support(t.shape[0], _ptr(t), _ptr(c), float(T), M, _ptr(mu),
                                            _ptr(alpha), _ptr(beta), _ptr(ll), _ptr(dmu),
                                            _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    return {"ll": float(ll[0]), "dmu": dmu, "dalpha": dal, "dbeta": dbe}


def chunk_table(offsets, C):
    """(chunk_base [B+1] int64, chunk_seq [chunks] int32) of sequences cut into chunks of C."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = offsets.shape[0] - 1
    lens = np.diff(offsets)
    nb = int(sum((int(x) + C - 1) // C for x in lens))
    base = np.zeros(B + 1, dtype=np.int64)
    seq = np.zeros(max(nb, 1), dtype=np.int32)
    rc = _load().oracle_chunk_table(B, _ptr(offsets), int(C), _ptr(base), _ptr(seq))
    if rc:
        raise OracleError(rc)
    return base, seq[:nb]


def bucket_order(c, M, C, P):
    """(bucket_start [chunks, P+1] int32, order [N] int32): per chunk of C events, the
    events ordered by (mark mod P, mark // P, index), and each block's first slot."""
    c = np.ascontiguousarray(c, dtype=np.int32)
    N = c.shape[0]
    nb = (N + C - 1) // C
    bs = np.zeros((max(nb, 1), P + 1), dtype=np.int32)
    order = np.zeros(max(N, 1), dtype=np.int32)
    rc = _load().oracle_bucket_order(N, _ptr(c), int(M), int(C), int(P), _ptr(bs), _ptr(order))
    if rc:
        raise OracleError(rc)
    return bs[:nb], order[:N]


def support_rows(alpha, all_entries=False):
    """(row_ptr [M+1], col [entries]) of alpha's support (alpha != 0, or every entry)."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    M = alpha.shape[0]
    row_ptr = np.zeros(M + 1, dtype=np.int32)
    col = np.zeros(max(M * M, 1), dtype=np.int32)
    rc = _load().oracle_support_rows(M, _ptr(alpha), int(bool(all_entries)), _ptr(row_ptr),
                                     _ptr(col))
    if rc:
        raise OracleError(rc)
    return row_ptr, col[:row_ptr[M]]


def mark_sort(c, M, L):
    """(start [nseg*M + 1], order [N]) of the events ordered by (segment of L events, mark,
    index)."""
    c = np.ascontiguousarray(c, dtype=np.int32)
    N = c.shape[0]
    nseg = (N + L - 1) // L
    start = np.zeros(nseg * M + 1, dtype=np.int32)
    order = np.zeros(max(N, 1), dtype=np.int32)
    rc = _load().oracle_mark_sort(N, _ptr(c), int(M), int(L), _ptr(start), _ptr(order))
    if rc:
        raise OracleError(rc)
    return start, order[:N]


def condition(t, c, T, mu, alpha, beta):
    """Sums of magnitudes of the terms of L and of each dL/dbeta_j (their conditioning
    scales): {"ll": float, "dbeta": array[M]}."""
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    sl, sb = np.zeros(1), np.zeros(M)
    rc = _load().oracle_condition(t.shape[0], _ptr(t), _ptr(c), float(T), M, _ptr(mu),
                                  _ptr(alpha), _ptr(beta), _ptr(sl), _ptr(sb))
    if rc:
        raise OracleError(rc)
    return {"ll": float(sl[0]), "dbeta": sb}


def loglik_grad_carry(t, c, T, mu, alpha, beta, S0=None, G0=None, base_term=True):
    """L and gradients of a slice whose first event sees the carried state (S0, G0)."""
    t, c, mu, alpha, beta, M = _prep(t, c, mu, alpha, beta)
    S0 = None if S0 is None else np.ascontiguousarray(S0, dtype=np.float64)
    G0 = None if G0 is None else np.ascontiguousarray(G0, dtype=np.float64)
    ll, dmu, dal, dbe = np.zeros(1), np.zeros(M), np.zeros((M, M)), np.zeros(M)
    rc = _load().oracle_loglik_grad_carry(t.shape[0], _ptr(t), _ptr(c), float(T), M, _ptr(mu),
                                          _ptr(alpha), _ptr(beta), _ptr(S0), _ptr(G0),
                                          int(bool(base_term)), _ptr(ll), None, _ptr(dmu),
                                          _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    return {"ll": float(ll[0]), "dmu": dmu, "dalpha": dal, "dbeta": dbe}


def slice_aggregate(t, c, M, beta, t_next):
    """(aggS, aggG): the slice's state contributions at time t_next."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.int32)
    beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, np.float64), (M,)))
    aS, aG = np.zeros(M), np.zeros(M)
    rc = _load().oracle_slice_aggregate(t.shape[0], _ptr(t), _ptr(c), M, _ptr(beta),
                                        float(t_next), _ptr(aS), _ptr(aG))
    if rc:
        raise OracleError(rc)
    return aS, aG


def _prep_multi(t, c, mu, alphas, betas):
    t = np.ascontiguousarray(t, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    M = mu.shape[0]
    alphas = np.ascontiguousarray(alphas, dtype=np.float64)
    betas = np.asarray(betas, dtype=np.float64)
    if betas.ndim == 1:
        betas = np.repeat(betas[:, None], M, axis=1)
    return t, c, mu, alphas, np.ascontiguousarray(betas, dtype=np.float64), M, alphas.shape[0]


def loglik_grad_multi(t, c, T, mu, alphas, betas, want_grad=True, want_lam=False):
    """K decay kernels: alphas [K, M, M] (row = target), betas [K] (one decay per kernel)
    or [K, M] (per source).  Returns L and (dmu [M], dalpha [K, M, M], dbeta [K, M])."""
    t, c, mu, alphas, betas, M, K = _prep_multi(t, c, mu, alphas, betas)
    N = t.shape[0]
    ll = np.zeros(1)
    lam = np.zeros(N) if want_lam else None
    dmu = np.zeros(M) if want_grad else None
    dal = np.zeros((K, M, M)) if want_grad else None
    dbe = np.zeros((K, M)) if want_grad else None
    rc = _load().oracle_loglik_grad_multi(N, _ptr(t), _ptr(c), float(T), M, K, _ptr(mu),
                                          _ptr(alphas), _ptr(betas), _ptr(ll), _ptr(lam),
                                          _ptr(dmu), _ptr(dal), _ptr(dbe))
    if rc:
        raise OracleError(rc)
    out = {"ll": float(ll[0])}
    if want_grad:
        out.update(dmu=dmu, dalpha=dal, dbeta=dbe)
    if want_lam:
        out["lam"] = lam
    return out


def condition_multi(t, c, T, mu, alphas, betas):
    """Conditioning scales with K decay kernels (sums of magnitudes of the terms of L and
    of each dL/dbeta^(q)_j): {"ll": float, "dbeta": array[K, M]}."""
    t, c, mu, alphas, betas, M, K = _prep_multi(t, c, mu, alphas, betas)
    sl, sb = np.zeros(1), np.zeros((K, M))
    rc = _load().oracle_condition_multi(t.shape[0], _ptr(t), _ptr(c), float(T), M, K, _ptr(mu),
                                        _ptr(alphas), _ptr(betas), _ptr(sl), _ptr(sb))
    if rc:
        raise OracleError(rc)
    return {"ll": float(sl[0]), "dbeta": sb}
