"""The plain FP64 scan comparator in bench.py (the paper's forward pass as
plain tensor ops) agrees with the oracle; runs on CPU tensors."""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_2604_01342_gb300 import synth


@pytest.mark.parametrize("n,batch", [(300, 1 << 19), (500, 64), (257, 128)])
def test_fp64_scan_matches_oracle(n, batch):
    p = synth.random_problem(6, n, 31 + n, True)
    ll = bench.fp64_scan_loglik(torch.from_numpy(p.t), torch.from_numpy(p.c), p.T,
                                torch.from_numpy(p.mu), torch.from_numpy(p.alpha),
                                float(p.beta[0]), batch=batch)
    ref = oracle.loglik(p.t, p.c, p.T, p.mu, p.alpha, p.beta)
    assert ll == pytest.approx(ref, rel=1e-11)


def test_blelloch_against_sequential_products():
    rng = np.random.default_rng(0)
    n, m = 37, 3
    s = torch.from_numpy(rng.uniform(0.2, 1.0, n))
    v = torch.from_numpy(rng.normal(size=(n, m)))
    Si, Vi = bench._blelloch_inclusive(s, v)
    accS, accV = 1.0, np.zeros(m)
    for i in range(n):            # P_i = M_i P_{i-1}
        accV = s[i].item() * accV + v[i].numpy()
        accS = s[i].item() * accS
        assert Si[i].item() == pytest.approx(accS, rel=1e-13)
        np.testing.assert_allclose(Vi[i].numpy(), accV, rtol=1e-12, atol=1e-13)
