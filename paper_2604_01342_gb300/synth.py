"""Seeded synthetic event streams and parameters.

This module only draws inputs: it holds none of the likelihood arithmetic, and
it imports neither the CUDA library nor the oracle, so both can be fed the
same arrays.  Events are drawn from the cluster (branching) representation of
the linear exponential Hawkes process (paper, Section 2, Eq.
hawkes_excitation): immigrants of mark i arrive as a Poisson process of rate
mu_i; an event of mark j has Poisson(sum_i alpha[i, j]) children, each child's
mark is i with probability alpha[i, j] / sum_i alpha[i, j] and its delay is
Exp(beta_j).  This realises the same process that Ogata's thinning
(paper, Section 4.3) simulates.  A stream "of N events" is the first N events
of a realisation on a long enough horizon, and T is the time of the N-th
event; restricted to [0, T] this is an exact realisation.

The five workloads (``workload(n)``):
  1. M=4, shared beta=1, mu=(0.2, 0.3, 0.4, 0.5), alpha U[0,1] at spectral
     radius 0.5, N=10,000, seed 0.
  2. M=64, beta_j ~ U[0.5, 2], mu_i ~ U[0.01, 0.1], alpha 10% Bernoulli mask x
     U[0,1] at spectral radius 0.8, N=1,000,000, seed 1.
  3. 4,096 sequences, each M=8 with its own beta_j ~ U[0.5, 3],
     mu_i ~ U[0.05, 0.5], dense alpha at spectral radius ~U[0.3, 0.9]; lengths
     lognormal(median 2,000, sigma 1) clipped to [50, 200,000]; seed 2.
  4. M=1,024, shared beta=1, mu_i proportional to (i+1)^-1.1 with sum 50,
     dense alpha U[0,1] at spectral radius 0.7, N=10,000,000, seed 3.
  5. M=4,096, beta_j ~ U[0.2, 5], alpha 1% at spectral radius 0.85,
     mu_i ~ U[0.001, 0.01] rescaled so that about N events arrive by T=1e7,
     N=50,000,000, seed 4.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One event stream and its parameters (float64 master copies)."""
    t: np.ndarray            # float64 [N], non-decreasing
    c: np.ndarray            # int32 [N], marks in [0, M)
    T: float
    mu: np.ndarray           # float64 [M]
    alpha: np.ndarray        # float64 [M, M], row = target, column = source
    beta: np.ndarray         # float64 [M] (all equal when the decay is shared)
    shared_beta: bool
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.t.shape[0])

    @property
    def M(self) -> int:
        return int(self.mu.shape[0])


@dataclass
class VarlenProblem:
    """B independent sequences, concatenated; params are per sequence."""
    t: np.ndarray            # float64 [Ntot]
    c: np.ndarray            # int32 [Ntot]
    offsets: np.ndarray      # int64 [B+1]
    T: np.ndarray            # float64 [B]
    mu: np.ndarray           # float64 [B, M]
    alpha: np.ndarray        # float64 [B, M, M]
    beta: np.ndarray         # float64 [B, M]
    shared_beta: bool
    name: str = ""

    @property
    def B(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def M(self) -> int:
        return int(self.mu.shape[-1])


def spectral_radius(a: np.ndarray, tol: float = 1e-12, max_iter: int = 20000) -> float:
    """Perron root of a non-negative matrix (power iteration on a + I, which
    has the same Perron vector and avoids oscillation on periodic patterns)."""
    a = np.asarray(a, dtype=np.float64)
    m = a.shape[0]
    if m <= 512:
        return float(np.max(np.abs(np.linalg.eigvals(a))))
    x = np.full(m, 1.0 / m)
    r_old = 0.0
    for _ in range(max_iter):
        y = a @ x + x
        r = float(y.sum() / x.sum()) - 1.0
        x = y / np.linalg.norm(y, 1)
        if abs(r - r_old) <= tol * max(1.0, abs(r)):
            break
        r_old = r
    return r


def scale_to_radius(a: np.ndarray, rho: float) -> np.ndarray:
    r = spectral_radius(a)
    if r <= 0.0:
        return a.copy()
    return a * (rho / r)


def _column_sampler(alpha: np.ndarray):
    """Flattened per-column CDF so that one searchsorted draws child marks."""
    m = alpha.shape[0]
    colsum = alpha.sum(axis=0)
    safe = np.where(colsum > 0, colsum, 1.0)
    cum = np.cumsum(alpha, axis=0) / safe[None, :]
    cum[-1, :] = 1.0
    flat = (np.arange(m, dtype=np.float64)[:, None] + cum.T).reshape(-1)  # [j*m + i]
    return colsum, flat


def simulate_cluster(mu, alpha, beta, horizon: float, rng: np.random.Generator):
    """All events on [0, horizon], sorted by time (stable), marks int32."""
    mu = np.asarray(mu, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = mu.shape[0]
    colsum, flat = _column_sampler(np.asarray(alpha, dtype=np.float64))
    counts = rng.poisson(mu * horizon)
    marks = np.repeat(np.arange(m, dtype=np.int32), counts)
    times = rng.uniform(0.0, horizon, size=marks.shape[0])
    all_t, all_c = [times], [marks]
    gen_t, gen_c = times, marks
    while gen_t.shape[0] > 0:
        nkids = rng.poisson(colsum[gen_c])
        par_t = np.repeat(gen_t, nkids)
        par_c = np.repeat(gen_c, nkids)
        if par_t.shape[0] == 0:
            break
        u = rng.random(par_t.shape[0])
        idx = np.searchsorted(flat, par_c.astype(np.float64) + u, side="right")
        kid_c = (idx - par_c.astype(np.int64) * m).clip(0, m - 1).astype(np.int32)
        kid_t = par_t + rng.exponential(1.0, size=par_t.shape[0]) / beta[par_c]
        keep = kid_t <= horizon
        gen_t, gen_c = kid_t[keep], kid_c[keep]
        all_t.append(gen_t)
        all_c.append(gen_c)
    t = np.concatenate(all_t)
    c = np.concatenate(all_c)
    order = np.argsort(t, kind="stable")
    return t[order], c[order]


def stationary_rate(mu, alpha) -> float:
    """Total event rate 1^T (I - alpha)^{-1} mu of a subcritical process."""
    m = mu.shape[0]
    return float(np.linalg.solve(np.eye(m) - alpha, mu).sum())


def simulate_n_events(mu, alpha, beta, n: int, rng: np.random.Generator):
    """First n events of one realisation; T = time of the n-th event."""
    if n == 0:
        return np.zeros(0), np.zeros(0, dtype=np.int32), 0.0
    rate = stationary_rate(mu, alpha)
    horizon = 1.15 * n / rate + 10.0 / float(np.min(beta))
    for _ in range(30):
        t, c = simulate_cluster(mu, alpha, beta, horizon, rng)
        if t.shape[0] >= n:
            t, c = t[:n].copy(), c[:n].copy()
            return t, c, float(t[-1])
        horizon *= 1.5
    raise RuntimeError("simulation did not reach the requested number of events")


def _problem(name, mu, alpha, beta, shared, n, rng, meta=None):
    t, c, T = simulate_n_events(mu, alpha, beta, n, rng)
    return Problem(t=t, c=c, T=T, mu=mu, alpha=alpha, beta=np.asarray(beta, dtype=np.float64),
                   shared_beta=shared, name=name, meta=meta or {})


def workload(n: int, n_events: int | None = None, n_seqs: int | None = None):
    """The five synthetic workloads (see the module docstring).

    ``n_events`` (configs 1, 2, 4, 5) or ``n_seqs`` (config 3) shrink the
    workload while keeping its parameter recipe and seed."""
    rng = np.random.default_rng(n - 1)
    if n == 1:
        m = 4
        mu = np.array([0.2, 0.3, 0.4, 0.5])
        alpha = scale_to_radius(rng.uniform(0.0, 1.0, size=(m, m)), 0.5)
        beta = np.full(m, 1.0)
        return _problem("hawkes_m4_shared_n10k", mu, alpha, beta, True,
                        n_events or 10_000, rng)
    if n == 2:
        m = 64
        beta = rng.uniform(0.5, 2.0, size=m)
        mu = rng.uniform(0.01, 0.1, size=m)
        mask = rng.random((m, m)) < 0.10
        alpha = scale_to_radius(mask * rng.uniform(0.0, 1.0, size=(m, m)), 0.8)
        return _problem("hawkes_m64_persource_n1m", mu, alpha, beta, False,
                        n_events or 1_000_000, rng)
    if n == 3:
        return varlen_workload(rng, n_seqs or 4096)
    if n == 4:
        m = 1024
        w = (np.arange(m) + 1.0) ** -1.1
        mu = 50.0 * w / w.sum()
        alpha = scale_to_radius(rng.uniform(0.0, 1.0, size=(m, m)), 0.7)
        beta = np.full(m, 1.0)
        return _problem("hawkes_m1024_shared_n10m", mu, alpha, beta, True,
                        n_events or 10_000_000, rng)
    if n == 5:
        m = 4096
        beta = rng.uniform(0.2, 5.0, size=m)
        mu = rng.uniform(0.001, 0.01, size=m)
        mask = rng.random((m, m)) < 0.01
        alpha = scale_to_radius(mask * rng.uniform(0.0, 1.0, size=(m, m)), 0.85)
        n_ev = n_events or 50_000_000
        # one common factor on mu so that about n_ev events arrive by T = 1e7
        mu = mu * (n_ev / 1e7) / stationary_rate(mu, alpha)
        return _problem("hawkes_m4096_persource_n50m", mu, alpha, beta, False, n_ev, rng)
    raise ValueError(f"unknown workload {n}")


def varlen_workload(rng: np.random.Generator, n_seqs: int, m: int = 8,
                    median: float = 2000.0, sigma: float = 1.0,
                    lo: int = 50, hi: int = 200_000) -> VarlenProblem:
    lengths = np.clip(np.round(median * np.exp(sigma * rng.standard_normal(n_seqs))),
                      lo, hi).astype(np.int64)
    mus, alphas, betas, ts, cs, Ts = [], [], [], [], [], []
    for s in range(n_seqs):
        beta = rng.uniform(0.5, 3.0, size=m)
        mu = rng.uniform(0.05, 0.5, size=m)
        rho = rng.uniform(0.3, 0.9)
        alpha = scale_to_radius(rng.uniform(0.0, 1.0, size=(m, m)), rho)
        t, c, T = simulate_n_events(mu, alpha, beta, int(lengths[s]), rng)
        mus.append(mu); alphas.append(alpha); betas.append(beta)
        ts.append(t); cs.append(c); Ts.append(T)
    offsets = np.zeros(n_seqs + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    return VarlenProblem(t=np.concatenate(ts) if ts else np.zeros(0),
                         c=np.concatenate(cs).astype(np.int32) if cs else np.zeros(0, np.int32),
                         offsets=offsets, T=np.array(Ts), mu=np.array(mus),
                         alpha=np.array(alphas), beta=np.array(betas), shared_beta=False,
                         name=f"hawkes_varlen_b{n_seqs}_m{m}")


def random_problem(m: int, n: int, seed: int, shared_beta: bool, rho: float = 0.6,
                   density: float = 1.0, beta_range=(0.5, 2.0), mu_range=(0.05, 0.5),
                   time_shift: float = 0.0) -> Problem:
    """A small seeded problem for parity tests (any M, N)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(*mu_range, size=m)
    a = rng.uniform(0.0, 1.0, size=(m, m)) * (rng.random((m, m)) < density)
    alpha = scale_to_radius(a, rho)
    if shared_beta:
        beta = np.full(m, rng.uniform(*beta_range))
    else:
        beta = rng.uniform(*beta_range, size=m)
    p = _problem(f"random_m{m}_n{n}_s{seed}", mu, alpha, beta, shared_beta, n, rng)
    if time_shift:
        p.t = p.t + time_shift
        p.T = p.T + time_shift
    return p


# ------------------------------------------------------------------ several decay kernels
@dataclass
class MultiProblem:
    """One event stream of a K-kernel process: kernel q has alphas[q] (row = target) and
    one decay betas[q] shared by all sources (the paper's multi-kernel model)."""
    t: np.ndarray            # float64 [N]
    c: np.ndarray            # int32 [N]
    T: float
    mu: np.ndarray           # float64 [M]
    alphas: np.ndarray       # float64 [K, M, M]
    betas: np.ndarray        # float64 [K]
    name: str = ""

    @property
    def N(self) -> int:
        return int(self.t.shape[0])

    @property
    def M(self) -> int:
        return int(self.mu.shape[0])

    @property
    def K(self) -> int:
        return int(self.alphas.shape[0])


def simulate_cluster_multi(mu, alphas, betas, horizon: float, rng: np.random.Generator):
    """Cluster representation with several kernels: an event of mark j has
    Poisson(colsum^(q)_j) children through kernel q, marks drawn from column j of
    alphas[q], delays Exp(betas[q])."""
    mu = np.asarray(mu, dtype=np.float64)
    m = mu.shape[0]
    samplers = [_column_sampler(np.asarray(a, dtype=np.float64)) for a in alphas]
    counts = rng.poisson(mu * horizon)
    marks = np.repeat(np.arange(m, dtype=np.int32), counts)
    times = rng.uniform(0.0, horizon, size=marks.shape[0])
    all_t, all_c = [times], [marks]
    gen_t, gen_c = times, marks
    while gen_t.shape[0] > 0:
        new_t, new_c = [], []
        for (colsum, flat), b in zip(samplers, betas):
            nkids = rng.poisson(colsum[gen_c])
            par_t = np.repeat(gen_t, nkids)
            par_c = np.repeat(gen_c, nkids)
            if par_t.shape[0] == 0:
                continue
            u = rng.random(par_t.shape[0])
            idx = np.searchsorted(flat, par_c.astype(np.float64) + u, side="right")
            kid_c = (idx - par_c.astype(np.int64) * m).clip(0, m - 1).astype(np.int32)
            kid_t = par_t + rng.exponential(1.0, size=par_t.shape[0]) / float(b)
            keep = kid_t <= horizon
            new_t.append(kid_t[keep])
            new_c.append(kid_c[keep])
        if not new_t:
            break
        gen_t, gen_c = np.concatenate(new_t), np.concatenate(new_c)
        all_t.append(gen_t)
        all_c.append(gen_c)
    t = np.concatenate(all_t)
    c = np.concatenate(all_c)
    order = np.argsort(t, kind="stable")
    return t[order], c[order]


def random_problem_multi(m: int, n: int, seed: int, kernels: int, rho: float = 0.6,
                         density: float = 1.0, beta_range=(0.3, 3.0),
                         mu_range=(0.05, 0.5)) -> MultiProblem:
    """A seeded K-kernel problem: the summed interaction matrix has spectral radius rho,
    shared among the kernels at random; decays drawn log-uniformly from beta_range."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(*mu_range, size=m)
    parts = [rng.uniform(0.0, 1.0, size=(m, m)) * (rng.random((m, m)) < density)
             for _ in range(kernels)]
    total = sum(parts)
    r = spectral_radius(total)
    scale = rho / r if r > 0 else 0.0
    alphas = np.stack([a * scale for a in parts])
    lo, hi = np.log(beta_range[0]), np.log(beta_range[1])
    betas = np.sort(np.exp(rng.uniform(lo, hi, size=kernels)))
    if n == 0:
        t, c, T = np.zeros(0), np.zeros(0, dtype=np.int32), 0.0
    else:
        rate = stationary_rate(mu, alphas.sum(axis=0))
        horizon = 1.15 * n / rate + 10.0 / float(np.min(betas))
        for _ in range(30):
            t, c = simulate_cluster_multi(mu, alphas, betas, horizon, rng)
            if t.shape[0] >= n:
                t, c = t[:n].copy(), c[:n].copy()
                break
            horizon *= 1.5
        else:
            raise RuntimeError("simulation did not reach the requested number of events")
        T = float(t[-1])
    return MultiProblem(t=t, c=c, T=T, mu=mu, alphas=alphas, betas=betas,
                        name=f"multi_m{m}_k{kernels}_n{n}_s{seed}")
