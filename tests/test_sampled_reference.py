"""Pins of the bin-by-bin references (tests/_sampled.py) that check the GPU at
the full 1024 x 1024 size: on small grids they equal the oracle's full stepper
(forward, Section 2.3 Eq. (SBI)) and its literal transpose (adjoint_sequence),
bin for bin, including the self-conjugate columns, the Nyquist lines, the
corner, k = 0 and ring wrap-around (more steps than the cutoff)."""
import numpy as np
import pytest

from oracle.sbim_oracle import Material, ModeSet, SBIMOracle, adjoint_sequence
from paper_2102_08756_gb300.synth import separable_history
from tests._sampled import adjoint_spectra, forward_spectra

CS, CP, RHO = 3464.0, 6000.0, 2670.0


def _case(n1, n3, L1, L3, steps, seed):
    nh = n1 // 2 + 1
    rng = np.random.default_rng(seed)
    bins = {0, 1, nh, n1 // 2, (n3 // 2) * nh, (n3 // 2) * nh + n1 // 2, (n3 - 1) * nh,
            (n3 - 1) * nh + n1 // 2, 2 * nh + 3}
    bins.update(int(b) for b in rng.choice(n3 * nh, 12, replace=False))
    dt = 0.3 * (L1 / n1) / CP
    hist = separable_history(n1, n3, L1, L3, steps, dt, CS, seed=seed, n_terms=2,
                             spectrum="flat", bins=sorted(bins))
    nz = np.nonzero(np.abs(hist.Uhat).sum(axis=(0, 1)) > 0)
    modes = ModeSet.build(n1, n3, L1, L3, r3=nz[0], j1=nz[1])
    return hist, dt, nz, modes


@pytest.mark.parametrize("n1,n3,L1,L3,n_cut,side", [(16, 12, 1600.0, 1250.0, 7, 1),
                                                    (12, 12, 1200.0, 1200.0, 5, -1)])
def test_forward_reference_equals_the_full_stepper(n1, n3, L1, L3, n_cut, side):
    steps = 2 * n_cut + 3
    hist, dt, (r3, j1), modes = _case(n1, n3, L1, L3, steps, seed=n1 + n_cut)
    o = SBIMOracle(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side)
    check = [n_cut - 1, n_cut, steps - 1]
    ref = forward_spectra(modes, Material(CS, CP, RHO), side, dt, n_cut,
                          hist.Uhat[:, :, r3, j1], hist.g, check)
    for n in range(steps):
        s = o.step(hist.u(n), np.zeros((3, n3, n1)))["s"]
        if n in check:
            got = np.fft.rfft2(s)[:, r3, j1]
            assert np.abs(got - ref[n]).max() <= 1e-11 * np.abs(ref[n]).max(), n
            # the bins outside the set stay empty: the update is diagonal in k
            full = np.fft.rfft2(s)
            full[:, r3, j1] = 0.0
            assert np.abs(full).max() <= 1e-11 * np.abs(ref[n]).max()


@pytest.mark.parametrize("n1,n3,L1,L3,n_cut,side", [(16, 12, 1600.0, 1250.0, 7, -1),
                                                    (12, 12, 1200.0, 1200.0, 5, 1)])
def test_adjoint_reference_equals_the_literal_transpose(n1, n3, L1, L3, n_cut, side):
    N = 2 * n_cut + 3
    hist, dt, (r3, j1), modes = _case(n1, n3, L1, L3, N, seed=3 * n1 + n_cut)
    # the adjoint calls run in reverse time: call k carries the time N - 1 - k
    tau_bar = np.stack([hist.u(N - 1 - m) for m in range(N)])
    u_bar, _ = adjoint_sequence(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side, tau_bar)
    calls = [n_cut - 1, n_cut, N - 1]
    ref = adjoint_spectra(modes, Material(CS, CP, RHO), side, dt, n_cut, n1, n3,
                          hist.Uhat[:, :, r3, j1], hist.g, calls)
    for k in calls:
        got = np.fft.rfft2(u_bar[N - 1 - k])[:, r3, j1]
        assert np.abs(got - ref[k]).max() <= 1e-11 * np.abs(ref[k]).max(), k
    # the modal matrices are Hermitian, so the adjoint spectra equal the forward
    # ones on real fields; a dropped conjugate (A^T for A^H) flips the sign of
    # the in-plane coupling and does not match
    fwd = forward_spectra(modes, Material(CS, CP, RHO), side, dt, n_cut,
                          hist.Uhat[:, :, r3, j1], hist.g, [calls[-1]])[calls[-1]]
    assert np.abs(fwd - ref[calls[-1]]).max() <= 1e-11 * np.abs(ref[calls[-1]]).max()
    bad = adjoint_spectra(modes, Material(CS, CP, RHO), side, dt, n_cut, n1, n3,
                          hist.Uhat[:, :, r3, j1], hist.g, [calls[-1]], conjugate=False)[calls[-1]]
    assert np.abs(bad - ref[calls[-1]]).max() > 1e-3 * np.abs(ref[calls[-1]]).max()
