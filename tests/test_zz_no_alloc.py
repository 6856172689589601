"""The allocation-free entry point sbim_spectral_response_noalloc.

Some callers cannot allocate device memory: a solver that runs inside a fixed
memory arena handed to it by its host framework, or a plugin whose device
footprint must stay the same while its host time-steps.  They cannot use
sbim_create, which allocates the history ring, the kernel tables and the FFT
plans, so this entry point takes the displacement-spectrum history and the
output from the caller and works in a static device array.

Both it and the handle-based sbim_step evaluate the non-local traction s of one
half-space.  sbim_step runs a handle with v = 0, so its output tau is s; the
allocation-free entry point gets the same displacement history as caller-owned
spectra and must return the spectrum of that s.  Each case checks two calls in
a row against sbim_step and against the FP64 oracle's per-mode operator
(relative L2 per component <= 1e-5, the float32 parity bound).  The cases
cover both half-spaces, a short history (fewer lags than the handle's cutoff),
and the table rebuilds a new c_p/c_s or a longer lag range force.  Bad
arguments (sizes beyond the static array, misaligned or host pointers) are
rejected before any launch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle.sbim_oracle import KernelTable, Material, ModeSet, apply_modal_operator, trapezoid_weights
from tests._errors import assert_finite

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, RHO = 3464.0, 2670.0


@pytest.fixture(scope="module")
def sbim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2102_08756_gb300 import sbim as mod
    return mod


def _oracle_spectrum(n1, n3, L1, L3, cp, dt, side, spec):
    """The oracle's s spectrum for the lag-major history ``spec`` (L, 3, n3, nh)."""
    modes = ModeSet.build(n1, n3, L1, L3)
    mat = Material(CS, cp, RHO)
    n_lags = spec.shape[0]
    dT = modes.q * CS * dt
    kt = KernelTable(mat.eta, float(dT.max()) * n_lags + 1)
    uniq, inv = np.unique(dT, return_inverse=True)
    w = np.stack([trapezoid_weights(d, n_lags, kt) for d in uniq], axis=1)[:, inv, :]
    hist_rev = spec.reshape(n_lags, 3, -1)
    F = apply_modal_operator(modes, mat, side, w, hist_rev, hist_rev[0])
    return F.reshape(3, n3, n1 // 2 + 1)


# (n1, n3, dx, cp, n_cut, side, steps): the first case is the original check; the
# second flips the side, changes c_p (table rebuild) and stops before the cutoff
# is reached; the third returns to the first c_p with a longer lag range.
CASES = [(32, 24, 100.0, 6000.0, 16, -1, 22),
         (24, 32, 100.0, 5500.0, 40, 1, 12),
         (32, 24, 100.0, 6000.0, 64, -1, 70)]


@pytest.mark.parametrize("n1,n3,dx,cp,n_cut,side,steps", CASES)
def test_noalloc_matches_sbim_step_on_two_calls(sbim, n1, n3, dx, cp, n_cut, side, steps):
    from paper_2102_08756_gb300.synth import separable_history
    L1, L3 = n1 * dx, n3 * dx
    dt = 0.3 * dx / cp
    nh = n1 // 2 + 1
    hist = separable_history(n1, n3, L1, L3, steps, dt, CS, seed=77 + n_cut, spectrum="k2")
    g = sbim.SBIM(n1, n3, L1, L3, CS, cp, RHO, dt, n_cut, side, "fp32", True)
    stream = torch.cuda.current_stream().cuda_stream
    zero = torch.zeros((3, n3, n1), device="cuda")
    fields, checked = [], 0
    for m in range(steps):
        u = hist.u(m).astype(np.float32)
        fields.append(u)
        tau = g.step(torch.from_numpy(u).cuda(), zero)
        if m < steps - 2:
            continue
        n_lags = min(m + 1, n_cut)
        spec = np.stack([np.fft.rfft2(fields[m - k].astype(np.float64)) for k in range(n_lags)])
        dev_hist = torch.from_numpy(np.ascontiguousarray(spec.astype(np.complex64)).view(np.float32)).cuda()
        out = torch.empty((3, n3, 2 * nh), dtype=torch.float32, device="cuda")
        sbim.sbim_spectral_response_noalloc(n1, n3, L1, L3, CS, cp, RHO, dt, side, n_lags,
                                            dev_hist.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex64).astype(np.complex128)
        assert_finite(got, "noalloc spectrum")
        ref = np.fft.rfft2(assert_finite(tau, "sbim_step tau"))
        oracle = _oracle_spectrum(n1, n3, L1, L3, cp, dt, side, spec)
        for c in range(3):
            err = np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c])
            assert err < 1e-5, ("against sbim_step", m, c, err)
            err = np.linalg.norm(got[c] - oracle[c]) / np.linalg.norm(oracle[c])
            assert err < 1e-5, ("against the oracle", m, c, err)
        checked += 1
    g.check()
    g.close()
    assert checked == 2


def test_noalloc_rejects_oversized_requests(sbim):
    """Sizes beyond the static array are rejected.  The buffers are real device
    allocations large enough for the sizes passed, so no launch could leave them
    even if a check were loosened."""
    bins = 2048 * 1025
    h = torch.zeros(4 * 3 * bins * 2, device="cuda")
    o = torch.zeros(3 * bins * 2, device="cuda")
    with pytest.raises(sbim.SBIMError, match="too large"):
        sbim.sbim_spectral_response_noalloc(2048, 2048, 2048e2, 2048e2, CS, 6000.0, RHO, 0.005, 1,
                                            4, h.data_ptr(), o.data_ptr(), None)
    # 64 x 64 at dt = 0.5 s: 77 table units per lag, 200 lags exceed the table
    bins = 64 * 33
    h = torch.zeros(200 * 3 * bins * 2, device="cuda")
    o = torch.zeros(3 * bins * 2, device="cuda")
    with pytest.raises(sbim.SBIMError, match="too long"):
        sbim.sbim_spectral_response_noalloc(64, 64, 6400.0, 6400.0, CS, 6000.0, RHO, 0.5, 1,
                                            200, h.data_ptr(), o.data_ptr(), None)
    torch.cuda.synchronize()


def test_noalloc_rejects_misaligned_and_host_pointers(sbim):
    """Pointers the float2 kernels cannot use come back as SBIM_ERR_ARG before
    any launch: a 4-byte offset into a device buffer, and host memory."""
    n, n_lags = 8, 3
    bins = n * (n // 2 + 1)
    h = torch.zeros(n_lags * 3 * bins * 2 + 2, device="cuda")
    o = torch.zeros(3 * bins * 2 + 2, device="cuda")
    args = (n, n, 800.0, 800.0, CS, 6000.0, RHO, 0.005, 1, n_lags)
    with pytest.raises(sbim.SBIMError, match="aligned") as e:
        sbim.sbim_spectral_response_noalloc(*args, h.data_ptr() + 4, o.data_ptr(), None)
    assert e.value.code == -1
    with pytest.raises(sbim.SBIMError, match="aligned"):
        sbim.sbim_spectral_response_noalloc(*args, h.data_ptr(), o.data_ptr() + 4, None)
    host = np.zeros(3 * bins * 2, dtype=np.float32)
    with pytest.raises(sbim.SBIMError, match="not device memory"):
        sbim.sbim_spectral_response_noalloc(*args, h.data_ptr(),
                                            host.ctypes.data_as(ctypes.c_void_p).value, None)
    # the accepted call on the same buffers still works afterwards
    sbim.sbim_spectral_response_noalloc(*args, h.data_ptr(), o.data_ptr(), None)
    torch.cuda.synchronize()
    assert float(o.abs().max()) == 0.0
