"""torch-facing wrapper of the pure-SBIM planar fault solver: a slip-weakening
fault (Section 2.1) between two elastic half-spaces represented only by their
boundaries (Eq. (SBI)), the reference solver of the TPV3 benchmark (Section 3).
Argument marshalling only; every step runs in the library's kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from . import sbim as B


class FaultSolver:
    def __init__(self, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, precision="fp32",
                 symmetric=False, stream=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.n1, self.n3 = n1, n3
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.shape = (2, 3, n3, n1)
        self.h = B.sbim_fault_create(n1, n3, float(L1), float(L3), float(cs), float(cp),
                                     float(rho), float(dt), int(n_cut), B.PRECISION[precision],
                                     int(bool(symmetric)), stream.cuda_stream)

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
        B.sbim_fault_set_fault(self.h, ms.ctypes.data_as(dp), t0.ctypes.data_as(dp),
                               float(mu_k), float(Dc), float(sigma0))

    def set_state(self, u=None, v=None):
        ptr = lambda x: None if x is None else self._t(x, self.shape)  # noqa: E731
        B.sbim_fault_set_state(self.h, ptr(u), ptr(v))

    def get_state(self):
        t = self.torch
        out = [t.empty(self.shape, dtype=self.dtype, device=self.stream.device) for _ in range(2)]
        B.sbim_fault_get_state(self.h, *[o.data_ptr() for o in out])
        return tuple(out)

    def step(self):
        B.sbim_fault_step(self.h)

    def fault_fields(self):
        """(slip, slip rate, fault traction perturbation), each [3][n3][n1]."""
        t = self.torch
        out = [t.empty((3, self.n3, self.n1), dtype=self.dtype, device=self.stream.device)
               for _ in range(3)]
        B.sbim_fault_fields(self.h, *[o.data_ptr() for o in out])
        return tuple(out)

    def handles(self):
        _, up, lo = B.sbim_fault_info(self.h)
        return up, (lo if lo.value else None)

    def save(self):
        """Checkpoint: both faces' u, v (host copies) and the half-spaces'
        histories (sbim_save)."""
        u, v = (x.cpu() for x in self.get_state())
        up, lo = self.handles()
        ck = {"u": u, "v": v, "up": B.sbim_save(up)}
        if lo is not None:
            ck["lo"] = B.sbim_save(lo)
        return ck

    def load(self, ck):
        dev = self.stream.device
        self.set_state(ck["u"].to(dev).contiguous(), ck["v"].to(dev).contiguous())
        up, lo = self.handles()
        B.sbim_load(up, ck["up"])
        if lo is not None:
            B.sbim_load(lo, ck["lo"])

    @property
    def steps(self):
        return B.sbim_fault_info(self.h)[0]

    def close(self):
        if self.h is not None:
            B.sbim_fault_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
