"""The decay factors' exponential (exp_unbiased): against FP64 exp rounded to FP32, its
error stays below one ulp and its mean signed error over each argument range stays near
zero, so products of many factors do not drift (the property the decay chains need)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(x):
    import torch
    from paper_2604_01342_gb300 import binding
    L = binding.lib()
    L.hawkes_test_exp_unbiased.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p]
    L.hawkes_test_exp_unbiased.restype = ctypes.c_int
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty_like(xd)
    assert L.hawkes_test_exp_unbiased(xd.data_ptr(), yd.data_ptr(), x.shape[0],
                                      torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _ulps(x32, y):
    ref = np.exp(x32.astype(np.float64))
    rf = ref.astype(np.float32)
    ulp = np.spacing(rf).astype(np.float64)
    return (y.astype(np.float64) - ref) / ulp


@pytest.mark.parametrize("lo,hi", [(-1e-3, 0.0), (-0.0625, 0.0625), (-0.35, 0.35), (-2.0, -0.2),
                                   (-20.0, -2.0), (-87.0, -20.0), (0.1, 2.0), (2.0, 64.0)])
def test_error_below_one_ulp_and_unbiased(lo, hi):
    n = 1 << 20
    x = (lo + (hi - lo) * (np.arange(n) + 0.5) / n).astype(np.float32)
    e = _ulps(x, _run(x))
    print(f"[{lo}, {hi}]: mean {e.mean():+.4f} ulp, max {np.abs(e).max():.3f} ulp")
    assert np.abs(e).max() < 1.0
    assert abs(e.mean()) < 0.03


def test_special_values():
    x = np.array([0.0, -0.0, -104.5, -200.0, 89.0, -1e-30, 1e-30], dtype=np.float32)
    y = _run(x)
    assert y[0] == 1.0 and y[1] == 1.0
    assert y[2] == 0.0 and y[3] == 0.0
    assert np.isinf(y[4])
    assert y[5] == 1.0 and y[6] == 1.0


def test_product_of_many_factors_does_not_drift():
    """2^16 chained factors exp(-x_i) against exp(-sum x_i): relative drift well below the
    one-signed 2^16 * 0.1 ulp (~4e-4) that a biased factor would give."""
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 0.2, size=1 << 16).astype(np.float32)
    y = _run(-x).astype(np.float64)
    logs = np.log(y) + x.astype(np.float64)            # per-factor relative error
    drift = float(logs.sum())
    print(f"drift over {x.shape[0]} factors: {drift:+.3e}")
    assert abs(drift) < 5e-5
