"""GB300-native exact log-likelihood and gradient of multivariate linear
exponential Hawkes processes (chunked prefix scan of diagonal-affine state
transitions, fused with the intensity, its log and the compensator).

The compute path is the C-ABI library ``libhawkes_gb300.so`` built from
``csrc/`` for sm_103a; ``binding`` loads it with ctypes and ``torch_api``
wraps it in a ``torch.autograd.Function``.  Nothing here falls back to the CPU:
if the library is missing, the first call raises.
"""
from .binding import (HawkesError, hawkes_loglik, hawkes_loglik_grad,  # noqa: F401
                      hawkes_loglik_varlen, hawkes_loglik_grad_varlen,
                      hawkes_workspace_size, hawkes_status_str, library_path)
