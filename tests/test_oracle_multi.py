"""Pins for the FP64 oracle of several decay kernels (oracle_loglik_grad_multi): each test
checks it against something other than itself (the single-kernel oracle at K = 1, a
brute-force double sum over kernels and event pairs, the identity that kernels sharing
one decay act as one kernel with the summed matrix, adaptive quadrature of the
compensator, central finite differences), and the conditioning sums of several kernels
against the single-kernel ones and a brute-force double sum."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2604_01342_gb300 import synth


def brute_intensity_multi(t, c, mu, alphas, betas):
    """Eq. hawkes_excitation with its sum over kernels, written out: O(N^2 K)."""
    lam = np.empty(len(t))
    for k in range(len(t)):
        s = mu[c[k]]
        for q in range(alphas.shape[0]):
            for l in range(k):
                s += alphas[q, c[k], c[l]] * betas[q] * math.exp(-betas[q] * (t[k] - t[l]))
        lam[k] = s
    return lam


def quad_compensator_multi(t, c, T, mu, alphas, betas):
    def total_rate(x):
        s = float(mu.sum())
        for q in range(alphas.shape[0]):
            for l in range(len(t)):
                if t[l] < x:
                    s += alphas[q, :, c[l]].sum() * betas[q] * math.exp(-betas[q] * (x - t[l]))
        return s
    knots = np.concatenate([[0.0], np.asarray(t), [T]])
    total = 0.0
    for a, b in zip(knots[:-1], knots[1:]):
        if b > a:
            total += integrate.quad(total_rate, a, b, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    return total


def test_one_kernel_equals_single_kernel_oracle():
    p = synth.random_problem(5, 600, seed=41, shared_beta=False)
    a = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    b = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alpha[None], p.beta[None])
    assert a["ll"] == b["ll"]
    np.testing.assert_array_equal(a["dmu"], b["dmu"])
    np.testing.assert_array_equal(a["dalpha"], b["dalpha"][0])
    np.testing.assert_array_equal(a["dbeta"], b["dbeta"][0])


@pytest.mark.parametrize("m,n,k,seed", [(2, 150, 2, 42), (4, 200, 3, 43)])
def test_intensity_matches_brute_force(m, n, k, seed):
    p = synth.random_problem_multi(m, n, seed=seed, kernels=k)
    out = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas, want_lam=True)
    ref = brute_intensity_multi(p.t, p.c, p.mu, p.alphas, p.betas)
    np.testing.assert_allclose(out["lam"], ref, rtol=1e-12)


def test_loglik_matches_quadrature():
    p = synth.random_problem_multi(2, 60, seed=44, kernels=3)
    out = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas, want_lam=True)
    L = float(np.sum(np.log(brute_intensity_multi(p.t, p.c, p.mu, p.alphas, p.betas))))
    L -= quad_compensator_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas)
    assert abs(out["ll"] - L) <= 1e-9 * abs(L)


def test_kernels_with_one_decay_act_as_their_sum():
    p = synth.random_problem_multi(4, 800, seed=45, kernels=2)
    betas = np.array([p.betas[0], p.betas[0]])
    two = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alphas, betas)
    one = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alphas.sum(axis=0), np.full(4, betas[0]))
    assert abs(two["ll"] - one["ll"]) <= 1e-12 * abs(one["ll"])
    np.testing.assert_allclose(two["dmu"], one["dmu"], rtol=1e-11, atol=1e-11)
    for q in range(2):      # dL/dalpha^(q) = dL/d(alpha^(1) + alpha^(2))
        np.testing.assert_allclose(two["dalpha"][q], one["dalpha"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(two["dbeta"].sum(axis=0), one["dbeta"], rtol=1e-10, atol=1e-9)


def test_gradient_matches_finite_differences():
    p = synth.random_problem_multi(3, 400, seed=46, kernels=2)
    out = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas)
    f = lambda mu, al, be: oracle.loglik_grad_multi(p.t, p.c, p.T, mu, al, be,  # noqa: E731
                                                    want_grad=False)["ll"]
    h = 1e-6
    g_mu = np.zeros(3)
    for i in range(3):
        e = np.zeros(3); e[i] = h
        g_mu[i] = (f(p.mu + e, p.alphas, p.betas) - f(p.mu - e, p.alphas, p.betas)) / (2 * h)
    g_al = np.zeros_like(p.alphas)
    for q in range(2):
        for i in range(3):
            for j in range(3):
                e = np.zeros_like(p.alphas); e[q, i, j] = h
                g_al[q, i, j] = (f(p.mu, p.alphas + e, p.betas) - f(p.mu, p.alphas - e, p.betas)) / (2 * h)
    g_be = np.zeros(2)              # one decay per kernel: the sum over sources
    for q in range(2):
        e = np.zeros(2); e[q] = h
        g_be[q] = (f(p.mu, p.alphas, p.betas + e) - f(p.mu, p.alphas, p.betas - e)) / (2 * h)
    for got, ref in ((out["dmu"], g_mu), (out["dalpha"], g_al), (out["dbeta"].sum(axis=1), g_be)):
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert float(np.max(np.abs(got - ref))) / scale < 2e-7


def brute_condition_multi(t, c, T, mu, alphas, betas):
    """The conditioning sums written as double sums over kernels and event pairs."""
    K, M = alphas.shape[0], mu.shape[0]
    lam = brute_intensity_multi(t, c, mu, alphas, betas)
    sb = np.zeros((K, M))
    for k in range(len(t)):
        for q in range(K):
            for j in range(M):
                d = sum(math.exp(-betas[q] * (t[k] - t[l])) * (1.0 - betas[q] * (t[k] - t[l]))
                        for l in range(k) if c[l] == j)
                sb[q, j] += abs(alphas[q, c[k], j] * d / lam[k])
    for q in range(K):
        cs = alphas[q].sum(axis=0)
        for l in range(len(t)):
            x = T - t[l]
            sb[q, c[l]] += cs[c[l]] * x * math.exp(-betas[q] * x)
    sl = float(np.sum(np.abs(np.log(lam)))) + T * float(mu.sum())
    for q in range(K):
        cs = alphas[q].sum(axis=0)
        sl += sum(cs[c[l]] * (1.0 - math.exp(-betas[q] * (T - t[l]))) for l in range(len(t)))
    return sl, sb


def test_condition_multi_one_kernel_equals_condition():
    p = synth.random_problem(6, 500, seed=47, shared_beta=True)
    a = oracle.condition(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    b = oracle.condition_multi(p.t, p.c, p.T, p.mu, p.alpha[None], p.beta[None])
    assert abs(a["ll"] - b["ll"]) <= 1e-13 * a["ll"]
    np.testing.assert_allclose(b["dbeta"][0], a["dbeta"], rtol=1e-13)


def test_condition_multi_matches_brute_force_and_bounds_the_gradient():
    p = synth.random_problem_multi(3, 120, seed=48, kernels=3)
    got = oracle.condition_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas)
    sl, sb = brute_condition_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas)
    assert abs(got["ll"] - sl) <= 1e-11 * sl
    np.testing.assert_allclose(got["dbeta"], sb, rtol=1e-10)
    g = oracle.loglik_grad_multi(p.t, p.c, p.T, p.mu, p.alphas, p.betas)
    assert np.all(np.abs(g["dbeta"]) <= got["dbeta"] * (1 + 1e-12))
    assert abs(g["ll"]) <= got["ll"]
