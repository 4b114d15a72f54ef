"""Differentiable AM-QFT: a torch.autograd.Function whose forward and
backward are the library's CUDA kernels.

The DFT of Eq. qft_0A is linear, y = F x, so for a real loss the gradient
with respect to x is F^H times the gradient with respect to y (PyTorch's
convention for complex tensors).  F^H = conj o F o conj is exactly the
library's unnormalised inverse (amqft_exec_inv), so the backward pass is one
launch of the same fused recursion; the backward of the inverse transform is
the forward transform.

Ordering: the transforms run on the current CUDA stream.  A cached plan above
2^16 owns a multi-pass workspace that its calls share, so forward and
backward passes that use one plan must be ordered (one stream, or explicit
synchronisation between streams and host threads).
"""
from __future__ import annotations

import threading
from collections import OrderedDict

from .amqft import Plan

_lock = threading.Lock()
_plans: "OrderedDict[tuple, Plan]" = OrderedDict()

# At most this many cached plans: a plan above 2^16 holds a workspace of up
# to 2 GiB, so the least recently used plan is released beyond the bound.
MAX_CACHED_PLANS = 8


def plan_for(log2n: int, variant: int, batch: int, device_index: int) -> Plan:
    """Cached plan for (length, variant, batch, device): plans own device
    constant tables (and, above 2^16, a workspace), so repeated calls reuse
    them; the cache keeps the MAX_CACHED_PLANS most recently used."""
    import torch

    key = (int(log2n), int(variant), int(batch), int(device_index))
    with _lock:
        p = _plans.get(key)
        if p is not None:
            _plans.move_to_end(key)
            return p
        with torch.cuda.device(device_index):
            p = Plan(log2n, variant, batch)
        _plans[key] = p
        while len(_plans) > MAX_CACHED_PLANS:
            old_key, old = _plans.popitem(last=False)
            with torch.cuda.device(old_key[3]):
                torch.cuda.synchronize()  # no kernel of the released plan is in flight
            old.close()
        return p


def clear_plan_cache() -> None:
    with _lock:
        for p in _plans.values():
            p.close()
        _plans.clear()


def _make_function():
    # created on first use so that importing the package does not import torch
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, variant: int, inverse: bool):
            n = x.shape[-1]
            log2n = n.bit_length() - 1
            xc = x.reshape(-1, n).contiguous()
            p = plan_for(log2n, variant, xc.shape[0], xc.device.index)
            y = p.inv(xc) if inverse else p.fwd(xc)
            ctx.variant, ctx.inverse, ctx.shape = variant, inverse, x.shape
            return y.reshape(x.shape)

        @staticmethod
        def backward(ctx, g):
            n = g.shape[-1]
            log2n = n.bit_length() - 1
            gc = g.reshape(-1, n).contiguous()
            p = plan_for(log2n, ctx.variant, gc.shape[0], gc.device.index)
            # adjoint: F^H g for the forward transform, F g for the inverse
            gx = p.fwd(gc) if ctx.inverse else p.inv(gc)
            return gx.reshape(ctx.shape), None, None

    return _Fn


_FN = None


def amqft(x, variant: int = 4, inverse: bool = False):
    """Differentiable DFT (or unnormalised inverse) over the last axis of a
    complex64 CUDA tensor whose length is a power of two."""
    global _FN
    import torch

    if x.dtype != torch.complex64 or not x.is_cuda:
        raise ValueError("amqft: x must be a complex64 CUDA tensor")
    n = x.shape[-1]
    if n < 1 or n & (n - 1):
        raise ValueError("amqft: the last dimension must be a power of two")
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(x, int(variant), bool(inverse))
