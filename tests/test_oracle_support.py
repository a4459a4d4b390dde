"""Pins of the oracle's lazy per-component form (oracle.loglik_grad_support), the
reference of the per-source path for large, sparse alpha: against the dense sequential
oracle (itself pinned by brute force, quadrature, closed forms and finite differences),
entry by entry on alpha's support; in every entry when alpha has full support; and its L
against the brute-force intensity plus the closed-form compensator.  A planted slip in a
copy of its source (the decay of the target instead of the source) must fail."""
import ctypes
import math
import subprocess

import numpy as np
import pytest

import oracle
from paper_2604_01342_gb300 import synth

from test_oracle_pins import brute_intensity


def _sparse_problem(m, n, seed, density, time_shift=0.0):
    p = synth.random_problem(m, n, seed, False, rho=0.7, density=density, beta_range=(0.2, 5.0),
                             time_shift=time_shift)
    assert np.ptp(p.beta) > 1.0
    return p


@pytest.mark.parametrize("m,n,seed,density", [(12, 800, 1, 0.25), (40, 1500, 2, 0.1),
                                              (5, 400, 3, 0.6), (64, 3000, 4, 0.05)])
def test_support_form_matches_dense_oracle_on_the_support(m, n, seed, density):
    p = _sparse_problem(m, n, seed, density)
    a = oracle.loglik_grad_support(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    b = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert abs(a["ll"] - b["ll"]) <= 1e-12 * abs(b["ll"])
    np.testing.assert_allclose(a["dmu"], b["dmu"], rtol=1e-11, atol=1e-11 * np.abs(b["dmu"]).max())
    np.testing.assert_allclose(a["dbeta"], b["dbeta"], rtol=1e-10,
                               atol=1e-11 * np.abs(b["dbeta"]).max())
    sup = p.alpha != 0
    assert 0 < sup.sum() < m * m
    np.testing.assert_allclose(a["dalpha"][sup], b["dalpha"][sup], rtol=1e-10,
                               atol=1e-11 * np.abs(b["dalpha"]).max())
    assert np.all(a["dalpha"][~sup] == 0.0)


def test_support_form_full_support_equals_dense_oracle():
    p = synth.random_problem(7, 900, 11, False, beta_range=(0.3, 4.0))
    assert np.all(p.alpha > 0)
    a = oracle.loglik_grad_support(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    b = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    for k in ("dmu", "dalpha", "dbeta"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-10, atol=1e-11 * np.abs(b[k]).max())


def test_support_form_loglik_against_brute_force():
    p = _sparse_problem(9, 500, 21, 0.3)
    lam = brute_intensity(p.t, p.c, p.mu, p.alpha, p.beta)
    cs = p.alpha.sum(axis=0)
    comp = p.T * p.mu.sum() + sum(cs[p.c[l]] * -math.expm1(-p.beta[p.c[l]] * (p.T - p.t[l]))
                                  for l in range(p.N))
    a = oracle.loglik_grad_support(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert abs(a["ll"] - (np.sum(np.log(lam)) - comp)) <= 1e-11 * abs(a["ll"])


def test_support_form_ties_and_large_times():
    p = _sparse_problem(6, 600, 31, 0.4, time_shift=1e7)
    p.t = np.round(p.t, 1)                # many equal times, near 1e7
    p.T = float(max(p.T, p.t[-1]))
    a = oracle.loglik_grad_support(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    b = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert abs(a["ll"] - b["ll"]) <= 1e-11 * abs(b["ll"])
    sup = p.alpha != 0
    np.testing.assert_allclose(a["dalpha"][sup], b["dalpha"][sup], rtol=1e-8,
                               atol=1e-10 * np.abs(b["dalpha"]).max())
    np.testing.assert_allclose(a["dbeta"], b["dbeta"], rtol=1e-8, atol=1e-10 * np.abs(b["dbeta"]).max())


def test_support_form_mutant_is_rejected(tmp_path):
    src = open(oracle._SRC).read()
    old = "            const double d = exp(-beta[j] * dt);\n            xs[e - rowp[i]] = S[j] * d;"
    assert src.count(old) == 1
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, old.replace("beta[j]", "beta[i]")))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_loglik_grad_support.argtypes = [ctypes.c_int64, P, P, ctypes.c_double,
                                               ctypes.c_int32, P, P, P, P, P, P, P]
    p = _sparse_problem(12, 800, 1, 0.25)
    t, c = np.ascontiguousarray(p.t), np.ascontiguousarray(p.c, np.int32)
    mu, al, be = p.mu.copy(), np.ascontiguousarray(p.alpha), p.beta.copy()
    ll, dmu, dal, dbe = np.zeros(1), np.zeros(p.M), np.zeros((p.M, p.M)), np.zeros(p.M)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    lib.oracle_loglik_grad_support(p.N, ptr(t), ptr(c), p.T, p.M, ptr(mu), ptr(al), ptr(be),
                                   ptr(ll), ptr(dmu), ptr(dal), ptr(dbe))
    b = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert abs(ll[0] - b["ll"]) > 1e-9 * abs(b["ll"])
