"""torch.autograd over a sequence of SBIM traction updates (Section 2.3, Eq. (SBI)).

``sbim_sequence(u, v, **params)`` runs N updates of one half-space from rest
(u, v: [N, 3, n3, n1] CUDA tensors) and returns the tractions [N, 3, n3, n1].
Its backward runs the library's adjoint entry point (sbim_step_adjoint) over the
cotangents in reverse time on a fresh handle: the transpose of the truncated
convolution is the time-reversed correlation with the same kernels.  The map is
linear in (u, v), so the backward needs no forward state: nothing is saved or
recomputed for the boundary operator itself.
"""
from __future__ import annotations

import torch

from .sbim import SBIM


class SBIMSequence(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v, params):
        if u.shape != v.shape or u.dim() != 4 or u.shape[1] != 3:
            raise ValueError("u and v must be [N, 3, n3, n1] tensors of equal shape")
        u = u.contiguous()
        v = v.contiguous()
        h = SBIM(**params)
        try:
            tau = torch.empty_like(u)
            for n in range(u.shape[0]):
                h.step(u[n], v[n], tau[n])
            h.check()
        finally:
            h.close()
        ctx.params = dict(params)
        return tau

    @staticmethod
    def backward(ctx, tau_bar):
        tau_bar = tau_bar.contiguous()
        u_bar = torch.empty_like(tau_bar)
        v_bar = torch.empty_like(tau_bar)
        h = SBIM(**ctx.params)
        try:
            for m in range(tau_bar.shape[0] - 1, -1, -1):
                h.step_adjoint(tau_bar[m], u_bar[m], v_bar[m])
            h.check()
        finally:
            h.close()
        return u_bar, v_bar, None


def sbim_sequence(u, v, *, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, precision="fp32",
                  kahan=True):
    """Differentiable tractions of N consecutive updates from rest."""
    params = dict(n1=n1, n3=n3, L1=L1, L3=L3, cs=cs, cp=cp, rho=rho, dt=dt, n_cut=n_cut,
                  side=side, precision=precision, kahan=kahan)
    return SBIMSequence.apply(u, v, params)
