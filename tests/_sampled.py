"""Bin-by-bin references of the update and of its adjoint, built from the
oracle's per-mode pieces, for grids too large for the oracle's full stepper.

The input is a separable history x(t_n) = sum_r X_r g_r[n] whose half spectra
X_hat_r are known exactly on a set of bins (zero elsewhere).  Each Fourier mode
evolves on its own (Section 2.3: the update is diagonal in the wavenumber), so
the spectrum of the output on those bins needs only those bins' histories.

* forward: the spectrum of s at step n, F = apply_modal_operator on the lag-major
  history  sum_r g_r[n - m] X_hat_r  (the oracle's convolution and assembly);
* adjoint: the spectrum of u_bar after the adjoint call of index n (calls in
  reverse time; the earlier calls carry the later times), from the oracle's
  conjugate-transposed modal matrices A(m)^H.  With the oracle's transposes of
  the DFTs (dft2_inverse_transpose weights the half spectrum by c_k / N, c_k = 2
  off the self-conjugate columns j1 = 0, n1/2; dft2_forward_transpose takes the
  real part of the half-spectrum sum), the forward DFT of u_bar is
      X_k                          off the self-conjugate columns,
      (X_k + conj(X_{k*})) / 2     on them (k* = the bin of -k),
  X_k = sum_m A_k(m)^H sum_r g_r[n - m] X_hat_{r,k}.

Both are pinned against the oracle's full stepper and its literal transpose
(adjoint_sequence) on small grids in tests/test_sampled_reference.py.  (The
modal matrices are Hermitian, A(m)^H = A(m), and on real fields the two
spectra coincide; the adjoint reference is still built from A^H as the
transpose defines it.)
"""
from __future__ import annotations

import numpy as np

from oracle.sbim_oracle import (KernelTable, ModeSet, apply_modal_operator, modal_matrices,
                                trapezoid_weights)


def _weights(modes, mat, dt, n_cut):
    dT = modes.q * mat.cs * dt
    kt = KernelTable(mat.eta, float(dT.max()) * n_cut + 1)
    uniq, inv = np.unique(dT, return_inverse=True)
    wu = np.stack([trapezoid_weights(d, n_cut, kt) for d in uniq], axis=1)
    return wu, inv


def _sub(modes, a, b):
    return ModeSet(modes.r3[a:b], modes.j1[a:b], modes.k1[a:b], modes.k3[a:b], modes.q[a:b],
                   modes.nyq1[a:b], modes.nyq3[a:b])


def _hist_rev(g, Xh, n, n_cut):
    """Lag-major history (L, 3, nsel): sum_r g_r[n - m] X_hat_r, zero before t_0."""
    idx = n - np.arange(n_cut)
    gl = np.where(idx >= 0, g[:, np.maximum(idx, 0)], 0.0)         # (R, L)
    return np.einsum("rl,rcq->lcq", gl, Xh)


def forward_spectra(modes, mat, side, dt, n_cut, Xhat, g, steps, chunk=512):
    """Spectra of s (3, nsel) at each step in ``steps``; Xhat is (R, 3, nsel)."""
    wu, inv = _weights(modes, mat, dt, n_cut)
    out = {n: np.empty((3, len(modes)), dtype=complex) for n in steps}
    for a in range(0, len(modes), chunk):
        b = min(a + chunk, len(modes))
        sub, w = _sub(modes, a, b), wu[:, inv[a:b], :]
        for n in steps:
            hr = _hist_rev(g, Xhat[:, :, a:b], n, n_cut)
            out[n][:, a:b] = apply_modal_operator(sub, mat, side, w, hr, hr[0])
    return out


def adjoint_spectra(modes, mat, side, dt, n_cut, n1, n3, Xhat, g, calls, chunk=256,
                    conjugate=True):
    """Spectra of u_bar (3, nsel) after each adjoint call index in ``calls``.
    The bin set must be closed under k -> -k on the self-conjugate columns.
    ``conjugate=False`` uses A(m)^T instead of A(m)^H (a mistake the pins
    must reject)."""
    wu, inv = _weights(modes, mat, dt, n_cut)
    X = {n: np.empty((3, len(modes)), dtype=complex) for n in calls}
    for a in range(0, len(modes), chunk):
        b = min(a + chunk, len(modes))
        sub = _sub(modes, a, b)
        AH = np.swapaxes(modal_matrices(sub, mat, side, wu[:, inv[a:b], :]), 2, 3)
        if conjugate:
            AH = np.conj(AH)
        for n in calls:
            hr = _hist_rev(g, Xhat[:, :, a:b], n, n_cut)                 # (L, 3, q)
            X[n][:, a:b] = np.einsum("lqab,lbq->aq", AH, hr)
    selfc = (modes.j1 == 0) | (modes.j1 == n1 // 2)
    pos = {(int(r), int(j)): i for i, (r, j) in enumerate(zip(modes.r3, modes.j1))}
    partner = np.array([pos[((-int(r)) % n3, int(j))] if s else i
                        for i, (r, j, s) in enumerate(zip(modes.r3, modes.j1, selfc))])
    out = {}
    for n in calls:
        Y = X[n].copy()
        Y[:, selfc] = 0.5 * (X[n][:, selfc] + np.conj(X[n][:, partner[selfc]]))
        out[n] = Y
    return out
