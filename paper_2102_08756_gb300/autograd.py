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


class HybridRupture(torch.autograd.Function):
    """Fault tractions [N, 3, n3, n1] of N coupled steps from rest (FE slab with a
    slip-weakening fault between two SBIM half-spaces, Section 2.4) as a function
    of the uniform slip-weakening distance Dc (a 0-d tensor).

    Forward: keeps the FE state every K steps and the SBIM boundary tractions of
    every step (the half-spaces' state is a linear function of the boundary
    history, so these replace it).  Backward: for each K-step segment, latest
    first, restores the checkpoint, recomputes the segment's states without the
    half-spaces (sbim_hybrid_step_given), and takes the transpose of its steps in
    reverse order (sbim_hybrid_adjoint_step), accumulating dJ/dDc per fault node
    (summed for the uniform Dc).
    """

    @staticmethod
    def forward(ctx, dc, params, law, steps, every):
        from .hybrid import Hybrid
        dcv = dc.detach().cpu().double().numpy()
        if dcv.ndim:
            raise ValueError("Dc must be a 0-d tensor (a uniform slip-weakening distance)")
        h = Hybrid(**params)
        h.set_fault(law["mu_s"], law["tau0"], law["mu_k"], float(dcv), law["sigma0"])
        ckpt, ttop, tbot, taus = {}, [], [], []
        for n in range(steps):
            if n % every == 0:
                ckpt[n] = h.get_state()
            h.step()
            top, bot = h.boundary_tractions()
            ttop.append(top)
            tbot.append(bot)
            taus.append(h.fault_fields()[2])
        # the handle is reused by the backward sweep: its FE state for the
        # recomputation, its (reset) half-spaces for the SBIM transposes
        ctx.h = h
        ctx.params, ctx.law, ctx.steps, ctx.every, ctx.dc = params, law, steps, every, float(dcv)
        ctx.ckpt, ctx.ttop, ctx.tbot = ckpt, ttop, tbot
        return torch.stack(taus)

    @staticmethod
    def backward(ctx, tau_bar):
        from . import sbim as B
        tau_bar = tau_bar.contiguous()
        h = ctx.h
        _, _, top, bot = B.sbim_hybrid_info(h.h)
        B.sbim_reset(top)                  # the adjoint sweep starts from rest
        B.sbim_reset(bot)
        lu = torch.zeros(h.shape, dtype=h.dtype, device=tau_bar.device)
        lv, la = torch.zeros_like(lu), torch.zeros_like(lu)
        dcb = torch.zeros((h.n3, h.n1), dtype=h.dtype, device=tau_bar.device)
        for s0 in reversed(range(0, ctx.steps, ctx.every)):
            s1 = min(s0 + ctx.every, ctx.steps)
            h.set_state(*ctx.ckpt[s0])
            states = []
            for n in range(s0, s1):
                states.append(h.get_state())
                h.step_given(ctx.ttop[n], ctx.tbot[n])
            for n in range(s1 - 1, s0 - 1, -1):
                u, v, a = states[n - s0]
                h.adjoint_step(u, v, a, ctx.ttop[n], ctx.tbot[n], tau_bar[n], lu, lv, la, dcb)
        return dcb.sum().to(torch.float64), None, None, None, None


def hybrid_rupture(dc, *, n1, n2, n3, h, cs, cp, rho, dt, n_cut, mu_s, tau0, mu_k, sigma0,
                   steps, every=50, precision="fp32"):
    """Differentiable fault tractions of a coupled rupture with respect to Dc."""
    params = dict(n1=n1, n2=n2, n3=n3, h=h, cs=cs, cp=cp, rho=rho, dt=dt, n_cut=n_cut,
                  precision=precision, boundaries=True, fault=True)
    law = dict(mu_s=mu_s, tau0=tau0, mu_k=mu_k, sigma0=sigma0)
    return HybridRupture.apply(dc, params, law, steps, every)


def sbim_sequence(u, v, *, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, precision="fp32",
                  kahan=True):
    """Differentiable tractions of N consecutive updates from rest."""
    params = dict(n1=n1, n3=n3, L1=L1, L3=L3, cs=cs, cp=cp, rho=rho, dt=dt, n_cut=n_cut,
                  side=side, precision=precision, kahan=kahan)
    return SBIMSequence.apply(u, v, params)
