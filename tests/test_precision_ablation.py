"""Precision ablations of two design choices, measured against the FP64 oracle on CPU:

1. time differences: the kernels subtract event times in FP64 and round the difference to
   FP32; storing times in FP32 and subtracting there loses them once t is large (the
   spacing of FP32 at 1e7 is 1.0);
2. the log-sum: FP64 accumulation of FP32 log-intensities, against a compensated
   (Neumaier) FP32 sum and a plain FP32 sum.

Both use a plain sequential FP32 recurrence (numpy scalars) that mirrors the kernels'
arithmetic: decays exp(-beta dt) in FP32, states and intensities in FP32.  The printed
numbers are the ones quoted in the design notes."""
import numpy as np

import oracle
from paper_2604_01342_gb300 import synth

f32 = np.float32


def fp32_loglik(t, c, T, mu, alpha, beta, dt_in_fp64=True, log_sum="fp64"):
    """Sequential FP32 recurrence S_k = D_k (S_{k-1} + e_{c_{k-1}}) with FP32 parameters."""
    M = mu.shape[0]
    mu32, al32, be32 = mu.astype(f32), alpha.astype(f32), beta.astype(f32)
    t32 = t.astype(f32)
    S = np.zeros(M, dtype=f32)
    acc64 = 0.0
    acc32, comp32 = f32(0.0), f32(0.0)
    for k in range(t.shape[0]):
        if k > 0:
            dt = f32(t[k] - t[k - 1]) if dt_in_fp64 else f32(t32[k] - t32[k - 1])
            S = (S * np.exp(-be32 * dt)).astype(f32)
            S[c[k - 1]] += f32(np.exp(-be32[c[k - 1]] * dt))
        lam = mu32[c[k]] + f32(np.dot(al32[c[k]] * be32, S))
        lg = f32(np.log(lam))
        if log_sum == "fp64":
            acc64 += float(lg)
        elif log_sum == "kahan":
            y = f32(acc32 + lg)
            if abs(acc32) >= abs(lg):
                comp32 = f32(comp32 + f32(f32(acc32 - y) + lg))
            else:
                comp32 = f32(comp32 + f32(f32(lg - y) + acc32))
            acc32 = y
        else:
            acc32 = f32(acc32 + lg)
    logsum = acc64 if log_sum == "fp64" else float(f32(acc32 + comp32))
    # compensator with FP64 T - t (as in the kernels), FP32 expm1
    colsum = al32.sum(axis=0).astype(np.float64)
    rest = T - t if dt_in_fp64 else (f32(T) - t32).astype(np.float64)
    comp = T * float(mu32.astype(np.float64).sum()) + float(
        (colsum[c] * -np.expm1(-be32[c].astype(np.float64) * rest)).sum())
    return logsum - comp


def test_fp64_time_differences_matter_at_large_t():
    p = synth.random_problem(4, 3000, seed=11, shared_beta=False, time_shift=1.0e7)
    ref = oracle.loglik(p.t, p.c, p.T, f32(p.mu), f32(p.alpha), f32(p.beta))
    e64 = abs(fp32_loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta, dt_in_fp64=True) - ref) / abs(ref)
    e32 = abs(fp32_loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta, dt_in_fp64=False) - ref) / abs(ref)
    print(f"times near 1e7: relative L error, FP64 differences {e64:.2e}, FP32 times {e32:.2e}")
    assert e64 < 1e-6
    assert e32 > 100 * e64


def test_log_sum_accumulation():
    rng = np.random.default_rng(5)
    n = 1_000_000
    lg = np.log(rng.uniform(0.01, 5.0, n)).astype(f32)
    exact = float(np.sum(lg.astype(np.float64)))      # FP64 sum of the FP32 terms
    s32 = f32(0.0)
    for x in lg[:200_000]:                            # plain FP32, first 2e5 terms
        s32 = f32(s32 + x)
    acc, comp = f32(0.0), f32(0.0)
    for x in lg[:200_000]:
        y = f32(acc + x)
        comp = f32(comp + (f32(f32(acc - y) + x) if abs(acc) >= abs(x) else f32(f32(x - y) + acc)))
        acc = y
    part = float(np.sum(lg[:200_000].astype(np.float64)))
    e_plain = abs(float(s32) - part) / abs(part)
    e_kahan = abs(float(f32(acc + comp)) - part) / abs(part)
    e64 = abs(float(np.sum(lg.astype(np.float64))) - exact) / abs(exact)
    print(f"log-sum of 2e5 FP32 terms: plain FP32 {e_plain:.2e}, compensated FP32 {e_kahan:.2e}; "
          f"FP64 over 1e6 terms {e64:.2e}")
    assert e_kahan < 1e-7 and e64 < 1e-12
    assert e_plain > 10 * e_kahan


def fp32_log_product(lam, per_thread=64):
    """The kernels' log-sum: per thread, a running product of FP32 intensities kept as an
    FP32 mantissa in [1, 2) and an integer binary exponent (one FP32 rounding per factor),
    one FP64 log per thread, FP64 sum over threads."""
    total = 0.0
    for g in range(0, lam.shape[0], per_thread):
        m, e = f32(1.0), 0
        for x in lam[g:g + per_thread]:
            fx, ex = np.frexp(f32(x))                 # x = fx 2^ex, fx in [0.5, 1)
            m = f32(m * f32(2.0 * fx))
            e += int(ex) - 1
            fm, em = np.frexp(m)
            m = f32(2.0 * fm)
            e += int(em) - 1
        total += float(np.log(np.float64(m))) + e * np.log(2.0)
    return total


def test_log_product_in_fp32_mantissa():
    rng = np.random.default_rng(6)
    lam = rng.uniform(0.01, 5.0, 200_000).astype(f32)
    exact = float(np.sum(np.log(lam.astype(np.float64))))
    e = abs(fp32_log_product(lam) - exact) / abs(exact)
    e_abs = abs(fp32_log_product(lam) - exact)
    print(f"log-sum of 2e5 FP32 intensities as FP32-mantissa products of 64: relative {e:.2e}, "
          f"absolute {e_abs:.2e}")
    assert e < 1e-9
