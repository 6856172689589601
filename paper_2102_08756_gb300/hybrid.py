"""torch-facing wrapper of the hybrid FEM-SBIM time step (Section 2.4): an
explicit hexahedral slab (Section 2.2) between two SBIM half-spaces, with an
optional slip-weakening fault on its mid-plane (Section 2.1).  Argument
marshalling only; every step runs in the library's kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from . import sbim as B


class Hybrid:
    def __init__(self, n1, n2, n3, h, cs, cp, rho, dt, n_cut, precision="fp32",
                 boundaries=True, fault=True, stream=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.n1, self.n2, self.n3 = n1, n2, n3
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.h = B.sbim_hybrid_create(n1, n2, n3, float(h), float(cs), float(cp), float(rho),
                                      float(dt), int(n_cut), B.PRECISION[precision],
                                      int(bool(boundaries)), int(bool(fault)),
                                      stream.cuda_stream)
        self.layers = B.sbim_hybrid_info(self.h)[0]
        self.shape = (self.layers, 3, n3, n1)

    def _t(self, x, shape):
        t = self.torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.dtype
                and tuple(x.shape) == shape and x.is_contiguous()):
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of shape {shape}")
        return x.data_ptr()

    def set_fault(self, mu_s, tau0, mu_k, Dc, sigma0):
        plane = (self.n3, self.n1)
        ms = np.ascontiguousarray(np.broadcast_to(np.asarray(mu_s, dtype=np.float64), plane))
        t0 = np.ascontiguousarray(np.broadcast_to(np.asarray(tau0, dtype=np.float64), plane))
        dp = ctypes.POINTER(ctypes.c_double)
        B.sbim_hybrid_set_fault(self.h, ms.ctypes.data_as(dp), t0.ctypes.data_as(dp),
                                float(mu_k), float(Dc), float(sigma0))

    def set_state(self, u=None, v=None, a=None):
        ptr = lambda x: None if x is None else self._t(x, self.shape)  # noqa: E731
        B.sbim_hybrid_set_state(self.h, ptr(u), ptr(v), ptr(a))

    def get_state(self):
        t = self.torch
        out = [t.empty(self.shape, dtype=self.dtype, device=self.stream.device) for _ in range(3)]
        B.sbim_hybrid_get_state(self.h, *[o.data_ptr() for o in out])
        return tuple(out)

    def step(self, force=None):
        B.sbim_hybrid_step(self.h, None if force is None else self._t(force, self.shape))

    def boundary_tractions(self):
        t = self.torch
        top = t.empty((3, self.n3, self.n1), dtype=self.dtype, device=self.stream.device)
        bot = t.empty_like(top)
        B.sbim_hybrid_boundary_tractions(self.h, top.data_ptr(), bot.data_ptr())
        return top, bot

    def step_given(self, tau_top, tau_bot):
        shp = (3, self.n3, self.n1)
        B.sbim_hybrid_step_given(self.h, self._t(tau_top, shp), self._t(tau_bot, shp))

    def adjoint_step(self, u, v, a, tau_top, tau_bot, tau_bar, lu, lv, la, dc_bar):
        shp = (3, self.n3, self.n1)
        B.sbim_hybrid_adjoint_step(
            self.h, self._t(u, self.shape), self._t(v, self.shape), self._t(a, self.shape),
            self._t(tau_top, shp), self._t(tau_bot, shp),
            None if tau_bar is None else self._t(tau_bar, shp),
            self._t(lu, self.shape), self._t(lv, self.shape), self._t(la, self.shape),
            self._t(dc_bar, (self.n3, self.n1)))

    def fault_fields(self):
        t = self.torch
        out = [t.empty((3, self.n3, self.n1), dtype=self.dtype, device=self.stream.device)
               for _ in range(3)]
        B.sbim_hybrid_fault_fields(self.h, *[o.data_ptr() for o in out])
        return tuple(out)

    def save(self):
        """Checkpoint of the coupled state: the slab's u, v, a (host copies) and
        both half-spaces' histories (sbim_save).  The fault law is part of the
        handle's parameters, not of the checkpoint; the slip is u+ - u-."""
        u, v, a = (x.cpu() for x in self.get_state())
        _, _, top, bot = B.sbim_hybrid_info(self.h)
        ck = {"u": u, "v": v, "a": a}
        if top.value:
            ck["top"], ck["bot"] = B.sbim_save(top), B.sbim_save(bot)
        return ck

    def load(self, ck):
        """Restore a checkpoint taken by ``save`` on a handle with the same
        parameters; the run continues as the original did."""
        dev = self.stream.device
        self.set_state(*(ck[k].to(dev).contiguous() for k in ("u", "v", "a")))
        _, _, top, bot = B.sbim_hybrid_info(self.h)
        if top.value:
            B.sbim_load(top, ck["top"])
            B.sbim_load(bot, ck["bot"])

    @property
    def steps(self):
        return B.sbim_hybrid_info(self.h)[1]

    def close(self):
        if self.h is not None:
            B.sbim_hybrid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
