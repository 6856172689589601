"""Thin Python binding of the C ABI in include/sbim.h (argument marshalling only).

Every entry point of the library has a function of the same name here; they
take plain integers / pointers and raise ``SBIMError`` on a non-zero status.
``SBIM`` wraps a handle for torch CUDA tensors: the tensors supply device
memory and the handle is bound to the current torch stream at creation.  Every
step of the traction update runs in the library's kernels; there is no
fallback when the library is missing -- loading it raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libsbim.so")

SBIM_OK = 0
PRECISION = {"fp64": 0, "fp32": 1, "bf16x2": 2, "bf16": 3}
STAGES = ("fft_forward", "convolution", "assemble", "fft_inverse", "epilogue")

_lib = None


class SBIMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sbim status {code}: {msg}")
        self.code = code


def lib():
    """Load libsbim.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    L.sbim_create.argtypes = [ctypes.POINTER(vp), i, i, d, d, d, d, d, d, i, i, i, i, vp]
    L.sbim_step.argtypes = [vp, vp, vp, vp]
    L.sbim_step_host.argtypes = [vp, vp, vp, vp]
    L.sbim_step_adjoint.argtypes = [vp, vp, vp, vp]
    L.sbim_set_far_field.argtypes = [vp, ctypes.POINTER(d)]
    L.sbim_reset.argtypes = [vp]
    L.sbim_rewind.argtypes = [vp]
    L.sbim_step_repeat.argtypes = [vp, vp, vp, vp]
    L.sbim_get_step.argtypes = [vp, ctypes.POINTER(ll)]
    L.sbim_get_info.argtypes = [vp] + [ctypes.POINTER(ll)] * 4
    L.sbim_plan.argtypes = [i, i, d, d, i, i] + [ctypes.POINTER(ll)] * 3
    L.sbim_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.sbim_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.sbim_set_profiling.argtypes = [vp, i]
    L.sbim_set_check_finite.argtypes = [vp, i]
    L.sbim_set_conv_tile.argtypes = [vp, i]
    L.sbim_batch_set_conv_tile.argtypes = [vp, i]
    L.sbim_hybrid_batch_set_conv_tile.argtypes = [vp, i]
    L.sbim_stage_times.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ll)]
    L.sbim_set_conv_config.argtypes = [vp, i, i]
    L.sbim_set_window.argtypes = [vp, d]
    L.sbim_check_device.argtypes = [vp]
    L.sbim_selftest_wait_timeout.argtypes = [vp]
    L.sbim_spectral_response_noalloc.argtypes = [i, i, d, d, d, d, d, d, i, i, vp, vp, vp]
    L.sbim_destroy.argtypes = [vp]
    L.sbim_fault_create.argtypes = [ctypes.POINTER(vp), i, i, d, d, d, d, d, d, i, i, i, vp]
    L.sbim_fault_set_fault.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d), d, d, d]
    L.sbim_fault_set_state.argtypes = [vp, vp, vp]
    L.sbim_fault_get_state.argtypes = [vp, vp, vp]
    L.sbim_fault_step.argtypes = [vp]
    L.sbim_fault_fields.argtypes = [vp, vp, vp, vp]
    L.sbim_fault_info.argtypes = [vp, ctypes.POINTER(ll), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.sbim_fault_destroy.argtypes = [vp]
    L.sbim_batch_set_conv_config.argtypes = [vp, i, i]
    L.sbim_hybrid_batch_set_conv_config.argtypes = [vp, i, i]
    L.sbim_hybrid_create.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, d, d, d, i, i, i, i, vp]
    L.sbim_hybrid_set_fault.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d), d, d, d]
    L.sbim_hybrid_set_state.argtypes = [vp, vp, vp, vp]
    L.sbim_hybrid_get_state.argtypes = [vp, vp, vp, vp]
    L.sbim_hybrid_step.argtypes = [vp, vp]
    L.sbim_hybrid_fault_fields.argtypes = [vp, vp, vp, vp]
    L.sbim_hybrid_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(ll),
                                   ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.sbim_hybrid_destroy.argtypes = [vp]
    L.sbim_hybrid_boundary_tractions.argtypes = [vp, vp, vp]
    L.sbim_hybrid_step_given.argtypes = [vp, vp, vp]
    L.sbim_hybrid_adjoint_step.argtypes = [vp] * 11
    L.sbim_batch_create.argtypes = [ctypes.POINTER(vp), i] + [vp] * 10 + [i, i, vp]
    L.sbim_batch_step.argtypes = [vp, vp, vp, vp]
    L.sbim_batch_capture.argtypes = [vp, vp, vp, vp]
    L.sbim_batch_replay.argtypes = [vp]
    L.sbim_batch_member.argtypes = [vp, i, ctypes.POINTER(vp)]
    L.sbim_batch_destroy.argtypes = [vp]
    L.sbim_hybrid_batch_create.argtypes = [ctypes.POINTER(vp), i, vp]
    for nm in ("sbim_hybrid_batch_step", "sbim_hybrid_batch_capture", "sbim_hybrid_batch_replay",
               "sbim_hybrid_batch_destroy"):
        getattr(L, nm).argtypes = [vp]
    L.sbim_last_error.argtypes = []
    L.sbim_last_error.restype = ctypes.c_char_p
    for name in ("sbim_create", "sbim_step", "sbim_step_host", "sbim_step_adjoint",
                 "sbim_set_far_field",
                 "sbim_reset", "sbim_get_step", "sbim_get_info", "sbim_plan", "sbim_set_profiling",
                 "sbim_set_check_finite", "sbim_set_conv_tile", "sbim_batch_set_conv_tile",
                 "sbim_hybrid_batch_set_conv_tile",
                 "sbim_stage_times", "sbim_set_conv_config", "sbim_check_device", "sbim_set_window",
                 "sbim_spectral_response_noalloc", "sbim_destroy", "sbim_hybrid_create",
                 "sbim_hybrid_set_fault", "sbim_hybrid_set_state", "sbim_hybrid_get_state",
                 "sbim_hybrid_step", "sbim_hybrid_fault_fields", "sbim_hybrid_info",
                 "sbim_hybrid_destroy", "sbim_hybrid_boundary_tractions", "sbim_hybrid_step_given",
                 "sbim_hybrid_adjoint_step", "sbim_batch_create", "sbim_batch_step",
                 "sbim_batch_capture", "sbim_batch_replay", "sbim_batch_member",
                 "sbim_batch_destroy", "sbim_hybrid_batch_create", "sbim_hybrid_batch_step",
                 "sbim_hybrid_batch_capture", "sbim_hybrid_batch_replay",
                 "sbim_hybrid_batch_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code):
    if code != SBIM_OK:
        raise SBIMError(code, lib().sbim_last_error().decode())


# --- one function per C entry point ------------------------------------------
def sbim_create(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, precision, kahan, stream):
    h = ctypes.c_void_p()
    _check(lib().sbim_create(ctypes.byref(h), n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side,
                             precision, kahan, stream))
    return h


def sbim_step(h, u_ptr, v_ptr, tau_ptr):
    _check(lib().sbim_step(h, u_ptr, v_ptr, tau_ptr))


def sbim_step_host(h, u_ptr, v_ptr, tau_ptr):
    _check(lib().sbim_step_host(h, u_ptr, v_ptr, tau_ptr))


def sbim_step_adjoint(h, tau_bar_ptr, u_bar_ptr, v_bar_ptr):
    _check(lib().sbim_step_adjoint(h, tau_bar_ptr, u_bar_ptr, v_bar_ptr))


def sbim_set_far_field(h, tau_inf):
    arr = (ctypes.c_double * 3)(*tau_inf)
    _check(lib().sbim_set_far_field(h, arr))


def sbim_reset(h):
    _check(lib().sbim_reset(h))


def sbim_step_repeat(h, u_ptr, v_ptr, tau_ptr):
    _check(lib().sbim_step_repeat(h, u_ptr, v_ptr, tau_ptr))


def sbim_rewind(h):
    _check(lib().sbim_rewind(h))


def sbim_get_step(h):
    n = ctypes.c_longlong()
    _check(lib().sbim_get_step(h, ctypes.byref(n)))
    return n.value


def sbim_get_info(h):
    vals = [ctypes.c_longlong() for _ in range(4)]
    _check(lib().sbim_get_info(h, *[ctypes.byref(v) for v in vals]))
    return dict(zip(("n_modes", "n_slots", "hist_bytes", "table_nodes"), (v.value for v in vals)))


def sbim_plan(n1, n3, L1, L3, n_cut, precision):
    """Layout sbim_create would build (host only): n_modes, n_slots, hist_bytes."""
    vals = [ctypes.c_longlong() for _ in range(3)]
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(lib().sbim_plan(int(n1), int(n3), float(L1), float(L3), int(n_cut), prec,
                           *[ctypes.byref(v) for v in vals]))
    return dict(zip(("n_modes", "n_slots", "hist_bytes"), (v.value for v in vals)))


def sbim_save(h):
    """Checkpoint of the handle's state as a numpy uint8 array."""
    import numpy as np
    n = ctypes.c_size_t(0)
    _check(lib().sbim_save(h, None, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib().sbim_save(h, buf.ctypes.data, ctypes.byref(n)))
    return buf[:n.value]


def sbim_load(h, buf):
    import numpy as np
    if isinstance(buf, (bytes, bytearray, memoryview)):
        buf = np.frombuffer(buf, dtype=np.uint8)
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().sbim_load(h, buf.ctypes.data if buf.nbytes else None, buf.nbytes))


def sbim_set_profiling(h, enable):
    _check(lib().sbim_set_profiling(h, int(enable)))


def sbim_set_check_finite(h, enable):
    _check(lib().sbim_set_check_finite(h, int(enable)))


def sbim_set_conv_tile(h, orbits_per_cta):
    _check(lib().sbim_set_conv_tile(h, int(orbits_per_cta)))


def sbim_batch_set_conv_tile(b, orbits_per_cta):
    _check(lib().sbim_batch_set_conv_tile(b, int(orbits_per_cta)))


def sbim_hybrid_batch_set_conv_tile(b, orbits_per_cta):
    _check(lib().sbim_hybrid_batch_set_conv_tile(b, int(orbits_per_cta)))


def sbim_stage_times(h):
    ms = (ctypes.c_double * 5)()
    n = ctypes.c_longlong()
    _check(lib().sbim_stage_times(h, ms, ctypes.byref(n)))
    return dict(zip(STAGES, list(ms))), n.value


def sbim_set_conv_config(h, variant, lags_per_cta=0):
    _check(lib().sbim_set_conv_config(h, int(variant), int(lags_per_cta)))


def sbim_set_window(h, window):
    _check(lib().sbim_set_window(h, float(window)))


def sbim_check_device(h):
    _check(lib().sbim_check_device(h))


def sbim_selftest_wait_timeout(h):
    _check(lib().sbim_selftest_wait_timeout(h))


def sbim_spectral_response_noalloc(n1, n3, L1, L3, cs, cp, rho, dt, side, n_lags, uhat_ptr,
                                   fhat_ptr, stream):
    """Allocation-free non-local traction spectrum for callers that may not
    allocate device memory (see include/sbim.h); device pointers in and out."""
    _check(lib().sbim_spectral_response_noalloc(n1, n3, L1, L3, cs, cp, rho, dt, side, n_lags,
                                                uhat_ptr, fhat_ptr, stream))


def sbim_destroy(h):
    _check(lib().sbim_destroy(h))


def sbim_last_error():
    return lib().sbim_last_error().decode()


def _ptrs(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*ptrs)


def sbim_batch_create(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, precision, kahan, stream):
    """Per-member sequences of equal length nb."""
    import numpy as np
    nb = len(n1)
    ints = [np.ascontiguousarray(x, dtype=np.int32) for x in (n1, n3, n_cut, side)]
    dbls = [np.ascontiguousarray(x, dtype=np.float64) for x in (L1, L3, cs, cp, rho, dt)]
    b = ctypes.c_void_p()
    _check(lib().sbim_batch_create(ctypes.byref(b), nb, ints[0].ctypes.data, ints[1].ctypes.data,
                                   *[d.ctypes.data for d in dbls], ints[2].ctypes.data,
                                   ints[3].ctypes.data, precision, kahan, stream))
    return b


def sbim_batch_set_conv_config(b, shape, lags_per_item=0):
    _check(lib().sbim_batch_set_conv_config(b, int(shape), int(lags_per_item)))


def sbim_hybrid_batch_set_conv_config(b, shape, lags_per_item=0):
    _check(lib().sbim_hybrid_batch_set_conv_config(b, int(shape), int(lags_per_item)))


def sbim_batch_step(b, u_ptrs, v_ptrs, tau_ptrs):
    _check(lib().sbim_batch_step(b, _ptrs(u_ptrs), _ptrs(v_ptrs), _ptrs(tau_ptrs)))


def sbim_batch_capture(b, u_ptrs, v_ptrs, tau_ptrs):
    _check(lib().sbim_batch_capture(b, _ptrs(u_ptrs), _ptrs(v_ptrs), _ptrs(tau_ptrs)))


def sbim_batch_replay(b):
    _check(lib().sbim_batch_replay(b))


def sbim_batch_member(b, i):
    h = ctypes.c_void_p()
    _check(lib().sbim_batch_member(b, i, ctypes.byref(h)))
    return h


def sbim_batch_destroy(b):
    _check(lib().sbim_batch_destroy(b))


def sbim_hybrid_batch_create(members):
    b = ctypes.c_void_p()
    _check(lib().sbim_hybrid_batch_create(ctypes.byref(b), len(members),
                                          _ptrs([m.value if hasattr(m, "value") else m
                                                 for m in members])))
    return b


def sbim_hybrid_batch_step(b):
    _check(lib().sbim_hybrid_batch_step(b))


def sbim_hybrid_batch_capture(b):
    _check(lib().sbim_hybrid_batch_capture(b))


def sbim_hybrid_batch_replay(b):
    _check(lib().sbim_hybrid_batch_replay(b))


def sbim_hybrid_batch_destroy(b):
    _check(lib().sbim_hybrid_batch_destroy(b))


def sbim_fault_create(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, precision, symmetric, stream):
    hh = ctypes.c_void_p()
    _check(lib().sbim_fault_create(ctypes.byref(hh), n1, n3, L1, L3, cs, cp, rho, dt, n_cut,
                                   precision, symmetric, stream))
    return hh


def sbim_fault_set_fault(h, mu_s_ptr, tau0_ptr, mu_k, Dc, sigma0):
    _check(lib().sbim_fault_set_fault(h, mu_s_ptr, tau0_ptr, mu_k, Dc, sigma0))


def sbim_fault_set_state(h, u_ptr, v_ptr):
    _check(lib().sbim_fault_set_state(h, u_ptr, v_ptr))


def sbim_fault_get_state(h, u_ptr, v_ptr):
    _check(lib().sbim_fault_get_state(h, u_ptr, v_ptr))


def sbim_fault_step(h):
    _check(lib().sbim_fault_step(h))


def sbim_fault_fields(h, slip_ptr, rate_ptr, traction_ptr):
    _check(lib().sbim_fault_fields(h, slip_ptr, rate_ptr, traction_ptr))


def sbim_fault_info(h):
    steps = ctypes.c_longlong()
    up, lo = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().sbim_fault_info(h, ctypes.byref(steps), ctypes.byref(up), ctypes.byref(lo)))
    return steps.value, up, lo


def sbim_fault_destroy(h):
    _check(lib().sbim_fault_destroy(h))


def sbim_hybrid_create(n1, n2, n3, h, cs, cp, rho, dt, n_cut, precision, boundaries, fault,
                       stream):
    hh = ctypes.c_void_p()
    _check(lib().sbim_hybrid_create(ctypes.byref(hh), n1, n2, n3, h, cs, cp, rho, dt, n_cut,
                                    precision, boundaries, fault, stream))
    return hh


def sbim_hybrid_set_fault(h, mu_s_ptr, tau0_ptr, mu_k, Dc, sigma0):
    _check(lib().sbim_hybrid_set_fault(h, mu_s_ptr, tau0_ptr, mu_k, Dc, sigma0))


def sbim_hybrid_set_state(h, u_ptr, v_ptr, a_ptr):
    _check(lib().sbim_hybrid_set_state(h, u_ptr, v_ptr, a_ptr))


def sbim_hybrid_get_state(h, u_ptr, v_ptr, a_ptr):
    _check(lib().sbim_hybrid_get_state(h, u_ptr, v_ptr, a_ptr))


def sbim_hybrid_step(h, force_ptr=None):
    _check(lib().sbim_hybrid_step(h, force_ptr))


def sbim_hybrid_fault_fields(h, slip_ptr, rate_ptr, traction_ptr):
    _check(lib().sbim_hybrid_fault_fields(h, slip_ptr, rate_ptr, traction_ptr))


def sbim_hybrid_info(h):
    layers, steps = ctypes.c_int(), ctypes.c_longlong()
    top, bot = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().sbim_hybrid_info(h, ctypes.byref(layers), ctypes.byref(steps),
                                  ctypes.byref(top), ctypes.byref(bot)))
    return layers.value, steps.value, top, bot


def sbim_hybrid_boundary_tractions(h, top_ptr, bot_ptr):
    _check(lib().sbim_hybrid_boundary_tractions(h, top_ptr, bot_ptr))


def sbim_hybrid_step_given(h, top_ptr, bot_ptr):
    _check(lib().sbim_hybrid_step_given(h, top_ptr, bot_ptr))


def sbim_hybrid_adjoint_step(h, u, v, a, tau_top, tau_bot, tau_bar, lu, lv, la, dc_bar):
    _check(lib().sbim_hybrid_adjoint_step(h, u, v, a, tau_top, tau_bot, tau_bar, lu, lv, la,
                                          dc_bar))


def sbim_hybrid_destroy(h):
    _check(lib().sbim_hybrid_destroy(h))


# --- torch-facing wrapper ------------------------------------------------------
class SBIM:
    """One half-space boundary (Section 2.3, Eq. (SBI)) on an n1 x n3 periodic grid.

    ``step(u, v)`` takes CUDA tensors [3, n3, n1] (float64 for precision
    "fp64", float32 otherwise) and returns the traction tensor.
    """

    def __init__(self, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, precision="fp32",
                 kahan=True, stream=None):
        import torch
        self.torch = torch
        self.n1, self.n3, self.n_cut, self.side = n1, n3, n_cut, side
        self.precision = precision
        self.kahan = kahan
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = stream.device
        self.h = sbim_create(n1, n3, float(L1), float(L3), float(cs), float(cp), float(rho),
                             float(dt), int(n_cut), int(side), PRECISION[precision],
                             int(bool(kahan)), stream.cuda_stream)

    def _field(self, x, name):
        t = self.torch
        if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == self.dtype
                and tuple(x.shape) == (3, self.n3, self.n1) and x.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor "
                             f"of shape (3, {self.n3}, {self.n1})")
        return x.data_ptr()

    def step(self, u, v, tau=None):
        if tau is None:
            tau = self.torch.empty_like(u)
        sbim_step(self.h, self._field(u, "u"), self._field(v, "v"), self._field(tau, "tau"))
        return tau

    def step_repeat(self, u, v, tau=None):
        """The last step's level again with a new u, v (see include/sbim.h)."""
        if tau is None:
            tau = self.torch.empty_like(u)
        sbim_step_repeat(self.h, self._field(u, "u"), self._field(v, "v"), self._field(tau, "tau"))
        return tau

    def step_adjoint(self, tau_bar, u_bar=None, v_bar=None):
        """Transpose of one step (reverse-time sweeps, see include/sbim.h)."""
        if u_bar is None:
            u_bar = self.torch.empty_like(tau_bar)
        if v_bar is None:
            v_bar = self.torch.empty_like(tau_bar)
        sbim_step_adjoint(self.h, self._field(tau_bar, "tau_bar"), self._field(u_bar, "u_bar"),
                          self._field(v_bar, "v_bar"))
        return u_bar, v_bar

    def step_host(self, u, v, tau=None):
        """Host numpy arrays in and out (copies inside the call)."""
        import numpy as np
        dt = np.float64 if self.precision == "fp64" else np.float32
        u = np.ascontiguousarray(u, dtype=dt)
        v = np.ascontiguousarray(v, dtype=dt)
        if tau is None:
            tau = np.empty_like(u)
        for a in (u, v, tau):
            if a.shape != (3, self.n3, self.n1) or a.dtype != dt or not a.flags.c_contiguous:
                raise ValueError("host arrays must be C-contiguous (3, n3, n1)")
        sbim_step_host(self.h, u.ctypes.data, v.ctypes.data, tau.ctypes.data)
        return tau

    def set_far_field(self, tau_inf):
        sbim_set_far_field(self.h, tau_inf)

    def save(self):
        """Checkpoint (numpy uint8) of the step counter, far field and history."""
        return sbim_save(self.h)

    def load(self, buf):
        sbim_load(self.h, buf)

    def reset(self):
        sbim_reset(self.h)

    def rewind(self):
        sbim_rewind(self.h)

    @property
    def n(self):
        return sbim_get_step(self.h)

    def info(self):
        return sbim_get_info(self.h)

    def set_profiling(self, enable=True):
        sbim_set_profiling(self.h, enable)

    def set_check_finite(self, enable=True):
        sbim_set_check_finite(self.h, enable)

    def set_conv_tile(self, orbits_per_cta):
        sbim_set_conv_tile(self.h, orbits_per_cta)

    def stage_times(self):
        return sbim_stage_times(self.h)

    def set_conv_config(self, variant, lags_per_cta=0):
        sbim_set_conv_config(self.h, variant, lags_per_cta)

    def set_window(self, window):
        """Mode-dependent truncation window in T = |k| c_s t (0: uniform cutoff)."""
        sbim_set_window(self.h, window)

    def check(self):
        """Wait for the stream; raise if a bounded device wait gave up."""
        sbim_check_device(self.h)

    def close(self):
        if self.h is not None:
            sbim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
