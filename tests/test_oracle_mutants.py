"""The pins have teeth: plant a plausible mistake in a copy of the oracle's C
source (on the CPU), rebuild it, and check that at least one pin rejects it."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2604_01342_gb300 import synth

from test_oracle_pins import brute_intensity, fd_grad

SRC = os.path.join(os.path.dirname(oracle.__file__), "hawkes_oracle.c")

MUTANTS = {
    # dropped decay factor beta_j in the intensity
    "drop_beta_in_intensity": ("exc += arow[j] * beta[j] * S[j];", "exc += arow[j] * S[j];"),
    # transposed alpha (row = source instead of target)
    "transposed_alpha": ("const double* arow = alpha + (size_t)i * (size_t)M;",
                         "double arow[4096]; for (int32_t q = 0; q < M; ++q) arow[q] = alpha[(size_t)q * M + i];"),
    # state jump applied after the decay instead of before it
    "jump_after_decay": ("double P = S[j] + (j == prev ? 1.0 : 0.0);",
                         "double P = S[j]; if (j == prev) { S[j] += 1.0 / d; P = S[j]; }"),
    # wrong sign of the G term in dL/dbeta
    "g_sign": ("(S[j] - beta[j] * G[j])", "(S[j] + beta[j] * G[j])"),
    # compensator of the source without the (1 - e) factor
    "compensator_no_decay": ("E[i] += -expm1(-x);", "E[i] += 1.0;"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_loglik_grad.argtypes = [ctypes.c_int64, p, p, ctypes.c_double, ctypes.c_int32,
                                       p, p, p, p, p, p, p, p]
    return lib


def run(lib, prob):
    M, N = prob.M, prob.N
    arrs = dict(t=np.ascontiguousarray(prob.t), c=np.ascontiguousarray(prob.c, np.int32),
                mu=prob.mu.copy(), al=prob.alpha.copy(), be=prob.beta.copy(), ll=np.zeros(1),
                lam=np.zeros(N), dmu=np.zeros(M), dal=np.zeros((M, M)), dbe=np.zeros(M))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    lib.oracle_loglik_grad(N, P(arrs["t"]), P(arrs["c"]), prob.T, M, P(arrs["mu"]), P(arrs["al"]),
                           P(arrs["be"]), P(arrs["ll"]), P(arrs["lam"]), P(arrs["dmu"]),
                           P(arrs["dal"]), P(arrs["dbe"]))
    return arrs


def pins_pass(lib):
    prob = synth.random_problem(3, 150, 77, False)
    out = run(lib, prob)
    if not np.allclose(out["lam"], brute_intensity(prob.t, prob.c, prob.mu, prob.alpha, prob.beta),
                       rtol=1e-10):
        return False
    ref = oracle.loglik_grad(prob.t, prob.c, prob.T, prob.mu, prob.alpha, prob.beta)
    if abs(out["ll"][0] - ref["ll"]) > 1e-9 * abs(ref["ll"]):   # quadrature-pinned value
        return False
    g_mu, g_al, g_be = fd_grad(prob)
    for got, fd in ((out["dmu"], g_mu), (out["dal"], g_al), (out["dbe"], g_be)):
        if np.max(np.abs(got - fd)) > 1e-5 * max(1.0, np.max(np.abs(fd))):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmp_path, name):
    assert not pins_pass(build_mutant(tmp_path, name))


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "same.c"
    path.write_text(src)
    so = tmp_path / "same.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_loglik_grad.argtypes = [ctypes.c_int64, p, p, ctypes.c_double, ctypes.c_int32,
                                       p, p, p, p, p, p, p, p]
    assert pins_pass(lib)
