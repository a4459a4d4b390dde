"""PyTorch-facing API: tensors in, tensors out, one ``torch.autograd.Function``.

PyTorch is used for device memory (the workspace comes from the caching
allocator) and streams (the current stream is passed to the C ABI); every step
of the computation runs in the CUDA kernels of ``libhawkes_gb300.so``.

    ll = loglik(t, c, T, mu, alpha, beta)            # 0-d float64, differentiable
    ll.backward()                                    # fills mu.grad, alpha.grad, beta.grad
    ll, dmu, dalpha, dbeta = loglik_grad(t, c, T, mu, alpha, beta)
    ll_b = loglik_varlen(t, c, offsets, T, mu, alpha, beta)   # [B], differentiable
    ll = loglik_multi(t, c, T, mu, alphas, betas)     # K decay kernels: alphas [K,M,M], betas [K]

Conventions follow ``include/hawkes_gb300.h``: marks 0-based, alpha[target,
source], beta of shape [] or [1] (shared decay) or [M] (per source), gradients
of L itself.  ``check=True`` synchronises and raises HawkesError if the device
checks found an invalid input.
"""
from __future__ import annotations

import torch

from . import binding as _b

_ws_cache: dict = {}


def _workspace(nbytes: int, device: torch.device) -> torch.Tensor:
    key = (device.index, torch.cuda.current_stream(device).cuda_stream)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=device)
        if buf.data_ptr() % 256:
            raise RuntimeError("workspace is not 256-byte aligned")
        _ws_cache[key] = buf
    return buf


def _shared(beta: torch.Tensor, M: int, beta_shared) -> bool:
    if beta_shared is not None:
        return bool(beta_shared)
    return beta.numel() == 1 and M != 1


def _prep(t, c, mu, alpha, beta):
    if not (t.is_cuda and c.is_cuda and mu.is_cuda and alpha.is_cuda and beta.is_cuda):
        raise ValueError("all tensors must be CUDA tensors")
    t = t.contiguous().to(torch.float64)
    c = c.contiguous().to(torch.int32)
    mu = mu.detach().contiguous().to(torch.float32)
    alpha = alpha.detach().contiguous().to(torch.float32)
    beta = beta.detach().contiguous().to(torch.float32).reshape(-1)
    return t, c, mu, alpha, beta


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def loglik_grad(t, c, T, mu, alpha, beta, beta_shared=None, chunk: int = 0, path: int = 0,
                validate: bool = True, check: bool = True, grad: bool = True,
                support: bool = False, reduce: int = 0, fp32_times: bool = False,
                walk_lanes: int = 0):
    """L (float64 0-d) and, if ``grad``, (dmu, dalpha, dbeta) as float32 tensors.
    ``support=True``: dalpha on alpha's support (entries alpha == 0 get 0).  ``reduce`` and
    ``fp32_times``: the precision options of hawkes_opts (chunk-GEMM path)."""
    t, c, mu, alpha, beta = _prep(t, c, mu, alpha, beta)
    dev = t.device
    N, M = t.shape[0], mu.shape[0]
    shared = _shared(beta, M, beta_shared)
    opts = _b.make_opts(shared, chunk, validate, path, support=support, reduce=reduce,
                        fp32_times=fp32_times, walk_lanes=walk_lanes)
    nbytes = _b.hawkes_workspace_size(N, M, 1, grad, opts)
    ws = _workspace(nbytes, dev)
    out_ll = torch.empty((), dtype=torch.float64, device=dev)
    s = _stream(dev)
    if grad:
        dmu = torch.empty(M, dtype=torch.float32, device=dev)
        dal = torch.empty(M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(1 if shared else M, dtype=torch.float32, device=dev)
        _b.hawkes_loglik_grad(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                              alpha.data_ptr(), beta.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                              out_ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(), dbe.data_ptr(), s)
    else:
        _b.hawkes_loglik(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                         alpha.data_ptr(), beta.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                         out_ll.data_ptr(), s)
    if check:
        rc = _b.hawkes_last_device_status(ws.data_ptr(), s)
        if rc:
            raise _b.HawkesError(rc, "device check")
    if grad:
        return out_ll, dmu, dal, dbe
    return out_ll


def loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta, beta_shared=None, chunk: int = 0,
                       path: int = 0, validate: bool = True, check: bool = True,
                       grad: bool = True, walk_lanes: int = 0):
    """Per-sequence L [B] (float64) and, if ``grad``, dmu [B,M], dalpha [B,M,M], dbeta [B] or [B,M]."""
    t, c, mu, alpha, beta = _prep(t, c, mu, alpha, beta)
    dev = t.device
    offsets = offsets.contiguous().to(torch.int64)
    T = T.contiguous().to(torch.float64)
    B = offsets.shape[0] - 1
    N = t.shape[0]
    M = mu.shape[-1]
    shared = bool(beta_shared) if beta_shared is not None else (beta.numel() == B and M != 1)
    opts = _b.make_opts(shared, chunk, validate, path, walk_lanes=walk_lanes)
    nbytes = _b.hawkes_workspace_size(N, M, B, grad, opts)
    ws = _workspace(nbytes, dev)
    out_ll = torch.empty(B, dtype=torch.float64, device=dev)
    s = _stream(dev)
    if grad:
        dmu = torch.empty(B, M, dtype=torch.float32, device=dev)
        dal = torch.empty(B, M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(B, dtype=torch.float32, device=dev) if shared else \
            torch.empty(B, M, dtype=torch.float32, device=dev)
        _b.hawkes_loglik_grad_varlen(t.data_ptr(), c.data_ptr(), offsets.data_ptr(), B, N,
                                     T.data_ptr(), M, mu.data_ptr(), alpha.data_ptr(),
                                     beta.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                                     out_ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(),
                                     dbe.data_ptr(), s)
    else:
        _b.hawkes_loglik_varlen(t.data_ptr(), c.data_ptr(), offsets.data_ptr(), B, N,
                                T.data_ptr(), M, mu.data_ptr(), alpha.data_ptr(),
                                beta.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                                out_ll.data_ptr(), s)
    if check:
        rc = _b.hawkes_last_device_status(ws.data_ptr(), s)
        if rc:
            raise _b.HawkesError(rc, "device check")
    if grad:
        return out_ll, dmu, dal, dbe
    return out_ll


def loglik_grad_multi(t, c, T, mu, alphas, betas, chunk: int = 0, validate: bool = True,
                      check: bool = True, grad: bool = True):
    """K decay kernels (kernel q: matrix alphas[q] with row = target, one decay betas[q]):
    L (float64 0-d) and, if ``grad``, (dmu [M], dalpha [K,M,M], dbeta [K]) as float32."""
    t, c, mu, alphas, betas = _prep(t, c, mu, alphas, betas)
    dev = t.device
    N, M = t.shape[0], mu.shape[0]
    K = alphas.numel() // (M * M)
    if alphas.numel() != K * M * M or betas.numel() != K:
        raise ValueError("alphas must be [K, M, M] and betas [K]")
    opts = _b.make_opts(True, chunk, validate, 2, K)
    nbytes = _b.hawkes_workspace_size(N, M, 1, grad, opts)
    ws = _workspace(nbytes, dev)
    out_ll = torch.empty((), dtype=torch.float64, device=dev)
    s = _stream(dev)
    if grad:
        dmu = torch.empty(M, dtype=torch.float32, device=dev)
        dal = torch.empty(K, M, M, dtype=torch.float32, device=dev)
        dbe = torch.empty(K, dtype=torch.float32, device=dev)
        _b.hawkes_loglik_grad(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                              alphas.data_ptr(), betas.data_ptr(), opts, ws.data_ptr(),
                              ws.numel(), out_ll.data_ptr(), dmu.data_ptr(), dal.data_ptr(),
                              dbe.data_ptr(), s)
    else:
        _b.hawkes_loglik(t.data_ptr(), c.data_ptr(), N, float(T), M, mu.data_ptr(),
                         alphas.data_ptr(), betas.data_ptr(), opts, ws.data_ptr(), ws.numel(),
                         out_ll.data_ptr(), s)
    if check:
        rc = _b.hawkes_last_device_status(ws.data_ptr(), s)
        if rc:
            raise _b.HawkesError(rc, "device check")
    if grad:
        return out_ll, dmu, dal, dbe
    return out_ll


class HawkesLogLikMulti(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, c, T, mu, alphas, betas, chunk):
        ll, dmu, dal, dbe = loglik_grad_multi(t, c, T, mu, alphas, betas, chunk)
        ctx.save_for_backward(dmu, dal, dbe)
        ctx.shapes = (alphas.shape, betas.shape)
        return ll

    @staticmethod
    def backward(ctx, g):
        dmu, dal, dbe = ctx.saved_tensors
        g32 = g.to(torch.float32)
        return (None, None, None, g32 * dmu, (g32 * dal).reshape(ctx.shapes[0]),
                (g32 * dbe).reshape(ctx.shapes[1]), None)


def loglik_multi(t, c, T, mu, alphas, betas, chunk: int = 0):
    """Differentiable exact log-likelihood with K decay kernels (0-d float64)."""
    return HawkesLogLikMulti.apply(t, c, T, mu, alphas, betas, chunk)


class HawkesLogLik(torch.autograd.Function):
    """L(mu, alpha, beta) for one sequence; the forward pass runs the fused
    log-likelihood + gradient kernels once and the backward pass scales the
    saved gradient by grad_output (no second pass over the events)."""

    @staticmethod
    def forward(ctx, t, c, T, mu, alpha, beta, beta_shared, chunk, path, support):
        need = any(ctx.needs_input_grad[3:6])
        if need:
            ll, dmu, dal, dbe = loglik_grad(t, c, T, mu, alpha, beta, beta_shared, chunk, path,
                                            support=support)
            ctx.save_for_backward(dmu, dal, dbe)
            ctx.beta_shape = beta.shape
        else:
            ll = loglik_grad(t, c, T, mu, alpha, beta, beta_shared, chunk, path, grad=False,
                             support=support)
        return ll

    @staticmethod
    def backward(ctx, g):
        dmu, dal, dbe = ctx.saved_tensors
        g32 = g.to(torch.float32)
        return (None, None, None, g32 * dmu, g32 * dal, (g32 * dbe).reshape(ctx.beta_shape),
                None, None, None, None)


class HawkesLogLikVarlen(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, c, offsets, T, mu, alpha, beta, beta_shared, chunk, path):
        need = any(ctx.needs_input_grad[4:7])
        if need:
            ll, dmu, dal, dbe = loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta,
                                                   beta_shared, chunk, path)
            ctx.save_for_backward(dmu, dal, dbe)
            ctx.beta_shape = beta.shape
        else:
            ll = loglik_grad_varlen(t, c, offsets, T, mu, alpha, beta, beta_shared, chunk, path,
                                    grad=False)
        return ll

    @staticmethod
    def backward(ctx, g):
        dmu, dal, dbe = ctx.saved_tensors
        g32 = g.to(torch.float32)
        gb = g32.reshape(-1, *([1] * (dbe.dim() - 1)))
        return (None, None, None, None, g32[:, None] * dmu, g32[:, None, None] * dal,
                (gb * dbe).reshape(ctx.beta_shape), None, None, None)


def loglik(t, c, T, mu, alpha, beta, beta_shared=None, chunk: int = 0, path: int = 0,
           support: bool = False):
    """Differentiable exact log-likelihood of one sequence (0-d float64).  ``support=True``
    takes the gradient with respect to alpha on its support (entries alpha == 0 get 0)."""
    return HawkesLogLik.apply(t, c, T, mu, alpha, beta, beta_shared, chunk, path, support)


def loglik_varlen(t, c, offsets, T, mu, alpha, beta, beta_shared=None, chunk: int = 0,
                  path: int = 0):
    """Differentiable per-sequence log-likelihoods [B] (float64)."""
    return HawkesLogLikVarlen.apply(t, c, offsets, T, mu, alpha, beta, beta_shared, chunk, path)
