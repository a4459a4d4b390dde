"""Pins for the FP64 oracle: each test checks it against something other than
itself (a brute-force double sum, quadrature, closed forms, finite
differences, identities and invariances the mathematics fixes)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2604_01342_gb300 import synth


# ---------------------------------------------------------------- helpers
def brute_intensity(t, c, mu, alpha, beta):
    """Eq. hawkes_excitation written out: an O(N^2 M) double sum over earlier
    events (index order l < k, so tied times count as earlier)."""
    n = len(t)
    lam = np.empty(n)
    for k in range(n):
        s = mu[c[k]]
        for l in range(k):
            j = c[l]
            s += alpha[c[k], j] * beta[j] * math.exp(-beta[j] * (t[k] - t[l]))
        lam[k] = s
    return lam


def intensity_at(x, t, c, mu, alpha, beta, strict=True):
    """lambda_m(x) for every m: base rate plus every event strictly before x."""
    lam = mu.copy()
    for l in range(len(t)):
        if (t[l] < x) if strict else (t[l] <= x):
            j = c[l]
            lam += alpha[:, j] * beta[j] * math.exp(-beta[j] * (x - t[l]))
    return lam


def quad_compensator(t, c, T, mu, alpha, beta):
    """int_0^T sum_m lambda_m(s) ds by adaptive quadrature between events."""
    knots = np.concatenate([[0.0], np.asarray(t), [T]])
    total = 0.0
    for a, b in zip(knots[:-1], knots[1:]):
        if b <= a:
            continue
        f = lambda s: float(np.sum(intensity_at(s, t, c, mu, alpha, beta)))  # noqa: E731
        val, _ = integrate.quad(f, a, b, epsabs=1e-13, epsrel=1e-12, limit=200)
        total += val
    return total


def small(m, n, seed, shared, **kw):
    return synth.random_problem(m, n, seed, shared, **kw)


# ------------------------------------------------------ brute force / quadrature
@pytest.mark.parametrize("m,n,seed,shared", [(1, 200, 0, True), (3, 300, 1, False),
                                             (5, 250, 2, True), (8, 400, 3, False)])
def test_intensity_matches_brute_force(m, n, seed, shared):
    p = small(m, n, seed, shared)
    got = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta, want_grad=False,
                             want_lam=True)["lam"]
    ref = brute_intensity(p.t, p.c, p.mu, p.alpha, p.beta)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("m,n,seed,shared", [(2, 40, 4, False), (3, 60, 5, True)])
def test_loglik_matches_quadrature(m, n, seed, shared):
    p = small(m, n, seed, shared)
    ll = oracle.loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    lam = brute_intensity(p.t, p.c, p.mu, p.alpha, p.beta)
    ref = float(np.sum(np.log(lam))) - quad_compensator(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert ll == pytest.approx(ref, rel=1e-10, abs=1e-10)


def test_ties_count_earlier_index():
    # three events at the same time: the second sees the first at full weight
    t = np.array([1.0, 1.0, 1.0, 2.5])
    c = np.array([0, 1, 0, 1], dtype=np.int32)
    mu = np.array([0.3, 0.2]); alpha = np.array([[0.2, 0.5], [0.4, 0.1]]); beta = np.array([1.5, 0.7])
    got = oracle.loglik_grad(t, c, 3.0, mu, alpha, beta, want_grad=False, want_lam=True)["lam"]
    np.testing.assert_allclose(got, brute_intensity(t, c, mu, alpha, beta), rtol=1e-14)
    assert got[1] == pytest.approx(mu[1] + alpha[1, 0] * beta[0], rel=1e-15)


# ------------------------------------------------------------- closed forms
def test_poisson_closed_form():
    p = small(6, 500, 7, False)
    a0 = np.zeros_like(p.alpha)
    out = oracle.loglik_grad(p.t, p.c, p.T, p.mu, a0, p.beta)
    n_i = np.bincount(p.c, minlength=6)
    assert out["ll"] == pytest.approx(float(np.sum(np.log(p.mu[p.c])) - p.T * p.mu.sum()),
                                      rel=1e-13)
    np.testing.assert_allclose(out["dmu"], n_i / p.mu - p.T, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(out["dbeta"], 0.0, atol=1e-12)
    # the Poisson MLE mu_i = n_i / T zeroes dmu
    out2 = oracle.loglik_grad(p.t, p.c, p.T, n_i / p.T, a0, p.beta)
    np.testing.assert_allclose(out2["dmu"], 0.0, atol=1e-8)


def test_one_event_closed_form():
    mu = np.array([0.2, 0.3]); alpha = np.array([[0.1, 0.4], [0.2, 0.3]]); beta = np.array([1.0, 2.0])
    t = np.array([0.5]); c = np.array([1], dtype=np.int32); T = 2.0
    ll = oracle.loglik(t, c, T, mu, alpha, beta)
    colsum1 = alpha[0, 1] + alpha[1, 1]
    ref = math.log(mu[1]) - T * mu.sum() - colsum1 * (1.0 - math.exp(-beta[1] * (T - t[0])))
    assert ll == pytest.approx(ref, rel=1e-15)
    assert ll == pytest.approx(-2.869121856468431, rel=1e-14)


def test_two_event_univariate_closed_form():
    mu, a, b = 0.5, 0.5, 1.0
    t = np.array([1.0, 2.0]); c = np.array([0, 0], dtype=np.int32); T = 3.0
    out = oracle.loglik_grad(t, c, T, [mu], [[a]], [b], want_lam=True)
    e1 = math.exp(-b * (t[1] - t[0]))
    lam2 = mu + a * b * e1
    comp = mu * T + a * ((1 - math.exp(-b * (T - t[0]))) + (1 - math.exp(-b * (T - t[1]))))
    np.testing.assert_allclose(out["lam"], [mu, lam2], rtol=1e-15)
    assert out["ll"] == pytest.approx(math.log(mu) + math.log(lam2) - comp, rel=1e-15)
    assert out["dmu"][0] == pytest.approx(1 / mu + 1 / lam2 - T, rel=1e-14)
    d_alpha = b * e1 / lam2 - ((1 - math.exp(-b * (T - t[0]))) + (1 - math.exp(-b * (T - t[1]))))
    assert out["dalpha"][0, 0] == pytest.approx(d_alpha, rel=1e-14)
    dt = t[1] - t[0]
    d_beta = a * e1 * (1 - b * dt) / lam2 - a * ((T - t[0]) * math.exp(-b * (T - t[0]))
                                                 + (T - t[1]) * math.exp(-b * (T - t[1])))
    assert out["dbeta"][0] == pytest.approx(d_beta, rel=1e-13)
    assert out["ll"] == pytest.approx(-3.32142531139764, rel=1e-13)
    assert out["dbeta"][0] == pytest.approx(-0.31927500382233, rel=1e-11)


# ------------------------------------------------------ gradient derivations
def fd_grad(p, h_rel=1e-6):
    f = lambda mu, al, be: oracle.loglik(p.t, p.c, p.T, mu, al, be)  # noqa: E731
    g_mu = np.zeros_like(p.mu); g_al = np.zeros_like(p.alpha); g_be = np.zeros_like(p.beta)
    for i in range(p.M):
        h = h_rel * max(1.0, abs(p.mu[i])); e = np.zeros_like(p.mu); e[i] = h
        g_mu[i] = (f(p.mu + e, p.alpha, p.beta) - f(p.mu - e, p.alpha, p.beta)) / (2 * h)
        h = h_rel * max(1.0, abs(p.beta[i])); e = np.zeros_like(p.beta); e[i] = h
        g_be[i] = (f(p.mu, p.alpha, p.beta + e) - f(p.mu, p.alpha, p.beta - e)) / (2 * h)
        for j in range(p.M):
            h = h_rel; e = np.zeros_like(p.alpha); e[i, j] = h
            g_al[i, j] = (f(p.mu, p.alpha + e, p.beta) - f(p.mu, p.alpha - e, p.beta)) / (2 * h)
    return g_mu, g_al, g_be


@pytest.mark.parametrize("m,n,seed", [(2, 300, 11), (4, 500, 12)])
def test_gradient_matches_finite_differences(m, n, seed):
    p = small(m, n, seed, False)
    out = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    g_mu, g_al, g_be = fd_grad(p)
    for got, ref in ((out["dmu"], g_mu), (out["dalpha"], g_al), (out["dbeta"], g_be)):
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert float(np.max(np.abs(got - ref))) / scale < 2e-7


@pytest.mark.parametrize("m,n,seed,shared", [(3, 400, 21, False), (7, 600, 22, True),
                                             (16, 300, 23, False)])
def test_adjoint_equals_forward_mode(m, n, seed, shared):
    p = small(m, n, seed, shared)
    f = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    a = oracle.grad_adjoint(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert a["ll"] == pytest.approx(f["ll"], rel=1e-13)
    for k in ("dmu", "dalpha", "dbeta"):
        np.testing.assert_allclose(a[k], f[k], rtol=1e-9, atol=1e-9 * np.max(np.abs(f[k])))


@pytest.mark.parametrize("m,n,seed", [(3, 300, 31), (6, 400, 32)])
def test_paper_formulas_equal_forward_mode(m, n, seed):
    p = small(m, n, seed, True)
    f = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    g = oracle.paper_grad_shared(p.t, p.c, p.T, p.mu, p.alpha, p.beta[0])
    assert g["ll"] == pytest.approx(f["ll"], rel=1e-12)
    np.testing.assert_allclose(g["dmu"], f["dmu"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(g["dalpha"], f["dalpha"], rtol=1e-9, atol=1e-9)
    assert g["dbeta"] == pytest.approx(float(np.sum(f["dbeta"])), rel=1e-7, abs=1e-7)


@pytest.mark.parametrize("shared", [False, True])
def test_euler_identity(shared):
    # lambda and the compensator are 1-homogeneous in (mu, alpha)
    p = small(5, 800, 41, shared)
    out = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta, want_lam=True)
    comp = float(np.sum(np.log(out["lam"]))) - out["ll"]
    lhs = float(np.dot(p.mu, out["dmu"]) + np.sum(p.alpha * out["dalpha"]))
    assert lhs == pytest.approx(p.N - comp, rel=1e-11, abs=1e-9)


# --------------------------------------------------------------- invariances
def test_time_shift():
    p = small(4, 500, 51, False)
    tau = 1e7
    ll0 = oracle.loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    ll1 = oracle.loglik(p.t + tau, p.c, p.T + tau, p.mu, p.alpha, p.beta)
    assert ll1 == pytest.approx(ll0 - tau * p.mu.sum(), rel=1e-9)


def test_time_rescale():
    p = small(4, 500, 52, False)
    a = 3.7
    ll0 = oracle.loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    ll1 = oracle.loglik(a * p.t, p.c, a * p.T, p.mu / a, p.alpha, p.beta / a)
    assert ll1 == pytest.approx(ll0 - p.N * math.log(a), rel=1e-12)


def test_relabel_marks():
    p = small(6, 500, 53, False)
    rng = np.random.default_rng(0)
    perm = rng.permutation(6)          # new label of old mark j is perm[j]
    inv = np.argsort(perm)
    c2 = perm[p.c].astype(np.int32)
    mu2 = p.mu[inv]; beta2 = p.beta[inv]; al2 = p.alpha[np.ix_(inv, inv)]
    f = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    g = oracle.loglik_grad(p.t, c2, p.T, mu2, al2, beta2)
    assert g["ll"] == pytest.approx(f["ll"], rel=1e-13)
    np.testing.assert_allclose(g["dmu"], f["dmu"][inv], rtol=1e-11)
    np.testing.assert_allclose(g["dalpha"], f["dalpha"][np.ix_(inv, inv)], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g["dbeta"], f["dbeta"][inv], rtol=1e-10, atol=1e-12)


def test_varlen_equals_per_sequence():
    rng = np.random.default_rng(5)
    vp = synth.varlen_workload(rng, 7, m=3, median=60, lo=0, hi=400)
    out = oracle.loglik_grad_varlen(vp.t, vp.c, vp.offsets, vp.T, vp.mu, vp.alpha, vp.beta)
    for s in range(vp.B):
        a, b = vp.offsets[s], vp.offsets[s + 1]
        f = oracle.loglik_grad(vp.t[a:b], vp.c[a:b], vp.T[s], vp.mu[s], vp.alpha[s], vp.beta[s])
        assert out["ll"][s] == f["ll"]
        np.testing.assert_array_equal(out["dalpha"][s], f["dalpha"])


def test_empty_and_single():
    mu = np.array([0.4, 0.1]); al = np.array([[0.1, 0.2], [0.3, 0.0]]); be = np.array([1.0, 2.0])
    out = oracle.loglik_grad(np.zeros(0), np.zeros(0, np.int32), 5.0, mu, al, be)
    assert out["ll"] == pytest.approx(-5.0 * mu.sum(), rel=1e-15)
    np.testing.assert_allclose(out["dmu"], [-5.0, -5.0])
    np.testing.assert_array_equal(out["dalpha"], 0.0)


# --------------------------------------------------- integer work, validation
def test_mark_counts_bit_exact():
    rng = np.random.default_rng(9)
    c = rng.integers(0, 37, size=100_000).astype(np.int32)
    np.testing.assert_array_equal(oracle.mark_counts(c, 37), np.bincount(c, minlength=37))


@pytest.mark.parametrize("case,code", [("unsorted", 2), ("mark", 3), ("time", 4), ("param", 5)])
def test_validation_codes(case, code):
    t = np.array([0.1, 0.5, 0.9]); c = np.array([0, 1, 0], dtype=np.int32)
    mu = np.array([0.3, 0.2]); al = np.full((2, 2), 0.1); be = np.array([1.0, 1.0]); T = 1.0
    if case == "unsorted":
        t = t[::-1].copy()
    elif case == "mark":
        c = np.array([0, 2, 0], dtype=np.int32)
    elif case == "time":
        T = 0.8
    elif case == "param":
        al = al.copy(); al[0, 1] = -0.1
    with pytest.raises(oracle.OracleError) as ei:
        oracle.loglik(t, c, T, mu, al, be)
    assert ei.value.code == code


# ----------------------------------------------------------- simulator check
def test_simulated_compensator_is_near_n():
    # time-rescaling: at the true parameters Lambda(T) ~ N +- a few sqrt(N)
    p = synth.workload(1, n_events=4000)
    out = oracle.loglik_grad(p.t, p.c, p.T, p.mu, p.alpha, p.beta, want_grad=False, want_lam=True)
    comp = float(np.sum(np.log(out["lam"]))) - out["ll"]
    assert abs(comp - p.N) < 5 * math.sqrt(p.N)
