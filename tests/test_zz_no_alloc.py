"""The allocation-free entry point sbim_spectral_response_noalloc, for callers
that may not allocate device memory (a solver handed fixed buffers by its host
framework), against the existing handle-based sbim_step.

Both evaluate the non-local traction s of one half-space.  sbim_step runs a
handle (history, tables and FFT plans it allocated) on a rectangular grid with
v = 0, so its output tau is s; the new entry point gets the same displacement
history as caller-owned spectra and must return the spectrum of that s.  Two
calls in a row are checked, with the parity bound of the float32 path (relative
L2 per component <= 1e-5).  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0


def test_noalloc_matches_sbim_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2102_08756_gb300 import sbim
    from paper_2102_08756_gb300.synth import separable_history

    n1, n3, L1, L3 = 32, 24, 3200.0, 2400.0
    dt, n_cut, side, steps = 0.3 * 100.0 / CP, 16, -1, 22
    nh = n1 // 2 + 1
    hist = separable_history(n1, n3, L1, L3, steps, dt, CS, seed=77, spectrum="k2")
    g = sbim.SBIM(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side, "fp32", True)
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
        sbim.sbim_spectral_response_noalloc(n1, n3, L1, L3, CS, CP, RHO, dt, side, n_lags,
                                            dev_hist.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex64).astype(np.complex128)
        ref = np.fft.rfft2(tau.double().cpu().numpy())
        for c in range(3):
            err = np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c])
            assert err < 1e-5, (m, c, err)
        checked += 1
    g.close()
    assert checked == 2


def test_noalloc_rejects_oversized_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2102_08756_gb300 import sbim
    with pytest.raises(sbim.SBIMError, match="too large"):
        sbim.sbim_spectral_response_noalloc(2048, 2048, 2048e2, 2048e2, CS, CP, RHO, 0.005, 1,
                                            4, 1, 1, None)
    with pytest.raises(sbim.SBIMError, match="too long"):
        sbim.sbim_spectral_response_noalloc(64, 64, 6400.0, 6400.0, CS, CP, RHO, 0.005, 1,
                                            200000, 1, 1, None)
