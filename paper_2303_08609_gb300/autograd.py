"""``torch.autograd`` support: chi = M_eo(U) phi with hand-written backward kernels.

Backward of a real loss L with incoming gradient g = dL/dchi (torch's
convention for complex tensors: dL/dRe + i dL/dIm):

* dL/dphi = M_eo^dag g            (``wilson_eo_apply_dag``)
* dL/dU   = link gradient of Re<g, M_eo phi>   (``wilson_eo_link_grad``)

Both run in the library's CUDA kernels. For S = |M_eo phi|^2 the su(3)
projection of dS/dU is the pseudofermion force (``WilsonEO.force``).
"""

from __future__ import annotations

import torch

from . import WilsonEO


def _sync_gauge(op: WilsonEO, U: torch.Tensor, refresh):
    """Repack ``U`` into ``op`` when it may have changed.

    refresh=None: when ``U`` is another tensor or its version counter moved
    (in-place ops); changes made through ``U.data`` are invisible to that
    counter, so pass refresh=True after them. refresh=True: always.
    refresh=False: never (the caller guarantees ``op`` already holds ``U``).
    """
    key = (U.data_ptr(), U._version)
    if refresh is True or (refresh is None and getattr(op, "_gauge_key", None) != key):
        op.set_gauge(U.detach().contiguous())
        op._gauge_key = key


class MeoFunction(torch.autograd.Function):
    """chi = M_eo phi for the gauge field ``U`` (canonical ``(4, V, 3, 3)``).

    ``op`` is a :class:`WilsonEO` handle (FP64 or FP32) on the lattice of
    ``U``; see :func:`_sync_gauge` for when its packed links are refreshed.
    """

    @staticmethod
    def forward(ctx, phi, U, op, refresh=None):
        _sync_gauge(op, U, refresh)
        phi = phi.contiguous()
        ctx.op = op
        ctx.refresh = refresh
        ctx.save_for_backward(phi, U)
        return op.apply(phi)

    @staticmethod
    def backward(ctx, grad_out):
        phi, U = ctx.saved_tensors
        op = ctx.op
        # the handle may hold another forward's links by now
        _sync_gauge(op, U, ctx.refresh)
        g = grad_out.contiguous()
        grad_phi = op.apply(g, dag=True) if ctx.needs_input_grad[0] else None
        grad_U = None
        if ctx.needs_input_grad[1]:
            if phi.dim() != 3:
                raise NotImplementedError("link gradient is provided for one right-hand side")
            grad_U = op.link_grad(g, phi)
        return grad_phi, grad_U, None, None


def meo(phi: torch.Tensor, U: torch.Tensor, op: WilsonEO, refresh=None) -> torch.Tensor:
    """Differentiable M_eo phi (see :class:`MeoFunction`)."""
    return MeoFunction.apply(phi, U, op, refresh)


def pseudofermion_action(phi: torch.Tensor, U: torch.Tensor, op: WilsonEO,
                         refresh=None) -> torch.Tensor:
    """S(U, phi) = |M_eo phi|^2 as a differentiable real scalar."""
    chi = meo(phi, U, op, refresh)
    return torch.sum(chi.real**2 + chi.imag**2)
