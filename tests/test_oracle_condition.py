"""Pins of the oracle's conditioning scales with one decay per source.

oracle.condition returns, for the log-likelihood and for every dL/dbeta_j, the sum of
the magnitudes of the terms whose difference is that result (the scale against which a
near-zero result's error is stated).  Here it is checked against the same sums written
out as a brute-force double sum over event pairs with DISTINCT decays beta_j, where a
source/target index slip (a decay taken from the target mark instead of the source)
changes the result; and a planted copy of the oracle with exactly that slip must fail."""
import ctypes
import math
import subprocess

import numpy as np
import pytest

import oracle
from paper_2604_01342_gb300 import synth

from test_oracle_pins import brute_intensity

SRC = oracle._SRC


def brute_condition(t, c, T, mu, alpha, beta):
    """scale_ll = sum_k |log lambda_k| + T sum mu + sum_l colsum_{c_l} (1 - e^{-beta_{c_l}(T - t_l)});
    scale_dbeta[j] = sum_k |alpha[c_k, j] / lambda_k * sum_{l<k, c_l=j} e^{-beta_j d}(1 - beta_j d)|
                     + colsum_j sum_{l: c_l = j} (T - t_l) e^{-beta_j (T - t_l)},  d = t_k - t_l.
    (S - beta G of the source-indexed state, per source j, is the inner sum.)"""
    M = mu.shape[0]
    lam = brute_intensity(t, c, mu, alpha, beta)
    cs = alpha.sum(axis=0)
    sb = np.zeros(M)
    for k in range(len(t)):
        for j in range(M):
            inner = 0.0
            for l in range(k):
                if c[l] == j:
                    d = t[k] - t[l]
                    inner += math.exp(-beta[j] * d) * (1.0 - beta[j] * d)
            sb[j] += abs(alpha[c[k], j] * inner / lam[k])
    for l in range(len(t)):
        x = T - t[l]
        sb[c[l]] += cs[c[l]] * x * math.exp(-beta[c[l]] * x)
    sl = float(np.sum(np.abs(np.log(lam)))) + T * float(mu.sum())
    sl += sum(cs[c[l]] * (1.0 - math.exp(-beta[c[l]] * (T - t[l]))) for l in range(len(t)))
    return sl, sb


def _problem():
    p = synth.random_problem(4, 160, seed=91, shared_beta=False, beta_range=(0.3, 3.0))
    assert np.ptp(p.beta) > 1.0            # decays that differ a lot between sources
    return p


def test_condition_per_source_matches_brute_force():
    p = _problem()
    got = oracle.condition(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    sl, sb = brute_condition(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert abs(got["ll"] - sl) <= 1e-11 * sl
    np.testing.assert_allclose(got["dbeta"], sb, rtol=1e-10)


def test_condition_bounds_the_per_source_gradient():
    p = _problem()
    sc = oracle.condition(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    g = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert np.all(np.abs(g["dbeta"]) <= sc["dbeta"] * (1 + 1e-12))
    assert abs(g["ll"]) <= sc["ll"]


# a decay taken from the target mark i = c_k instead of the source j, in the dbeta scale;
# and the same slip in the compensator part of that scale
MUTANTS = {
    "target_decay_in_scale": (
        "scale_dbeta[j] += fabs(w * arow[j] * (S[j] - beta[j] * G[j]));",
        "scale_dbeta[j] += fabs(w * arow[j] * (S[j] - beta[i] * G[j]));"),
    "row_sum_for_column_sum": (
        "for (int32_t r = 0; r < M; ++r) cs += alpha[(size_t)r * M + j];\n            scale_dbeta[j] += cs * F[j];",
        "for (int32_t r = 0; r < M; ++r) cs += alpha[(size_t)j * M + r];\n            scale_dbeta[j] += cs * F[j];"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_condition.argtypes = [ctypes.c_int64, p, p, ctypes.c_double, ctypes.c_int32,
                                     p, p, p, p, p]
    lib.oracle_condition.restype = ctypes.c_int
    return lib


def _pin_passes(lib):
    p = _problem()
    t = np.ascontiguousarray(p.t)
    c = np.ascontiguousarray(p.c, dtype=np.int32)
    mu, al, be = p.mu.copy(), np.ascontiguousarray(p.alpha), p.beta.copy()
    sl, sb = np.zeros(1), np.zeros(p.M)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.oracle_condition(p.N, P(t), P(c), p.T, p.M, P(mu), P(al), P(be), P(sl), P(sb)) == 0
    ref_l, ref_b = brute_condition(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    return abs(sl[0] - ref_l) <= 1e-11 * ref_l and np.allclose(sb, ref_b, rtol=1e-10, atol=0)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_condition_mutant_is_rejected(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pin_passes(_build(tmp_path, name, old, new))


def test_condition_unmutated_copy_passes(tmp_path):
    assert _pin_passes(_build(tmp_path, "same", "scale_dbeta[j] += cs * F[j];",
                              "scale_dbeta[j] += cs * F[j];"))
