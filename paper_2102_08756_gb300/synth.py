"""Seeded synthetic boundary-displacement histories.

The paper's runs (Section 3: a planar fault in a homogeneous half-space pair,
rho = 2670 kg/m^3, c_p = 6000 m/s, c_s = 3464 m/s) have no published boundary
data, so stand-in histories are drawn here.  A history is a sum of R separable
terms

    u(x1, x3, t) = sum_r U_r(x1, x3) g_r(t)

with U_r a real random field on the periodic boundary grid (three displacement
components) and g_r a band-limited temporal signal that starts from rest.
Three spatial spectra are offered: ``"band"`` (flat amplitude for
|k| <= k_cut, zero above), ``"k2"`` (amplitude 1 / (1 + (|k|/k0)^2), the
k^-2 falloff of a rupture-like field) and ``"flat"`` (the same amplitude at
every wavenumber).  ``sparse`` keeps only a seeded random subset of Fourier
bins, ``bins`` an explicit one; their exact spectra are returned so that large
grids can be checked bin by bin.

This module is shared input plumbing: it holds none of the boundary-integral
arithmetic and is used identically by the tests, the benchmark and the
smoke check.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SeparableHistory:
    """u(x, t_n) = sum_r U[r] * g[r, n]; U is [R][3][N3][N1] float64."""

    U: np.ndarray            # spatial patterns, [R][3][N3][N1]
    Uhat: np.ndarray         # their unnormalised half spectra, [R][3][N3][N1/2+1]
    g: np.ndarray            # temporal signals, [R][steps]
    dt: float

    @property
    def steps(self) -> int:
        return self.g.shape[1]

    def u(self, n: int) -> np.ndarray:
        return np.tensordot(self.g[:, n], self.U, axes=1)

    def v(self, n: int) -> np.ndarray:
        """Backward-difference velocity (u_n - u_{n-1}) / dt, u_{-1} = 0."""
        gp = self.g[:, n - 1] if n > 0 else np.zeros(self.g.shape[0])
        return np.tensordot((self.g[:, n] - gp) / self.dt, self.U, axes=1)


def _temporal(rng, steps, dt, omega_max, n_sin=8, ramp_steps=20):
    t = np.arange(steps) * dt
    w = rng.uniform(0.05, 1.0, n_sin) * omega_max
    ph = rng.uniform(0.0, 2 * np.pi, n_sin)
    amp = rng.normal(size=n_sin)
    sig = (amp[:, None] * np.sin(w[:, None] * t[None, :] + ph[:, None])).sum(0)
    ramp = np.ones(steps)
    k = np.arange(steps)
    on = k < ramp_steps
    ramp[on] = np.sin(0.5 * np.pi * k[on] / ramp_steps) ** 2
    return sig * ramp


def separable_history(n1, n3, L1, L3, steps, dt, cs, seed, *, n_terms=4,
                      spectrum="band", amp_rms=1e-3, sparse=None, bins=None):
    """Draw a seeded ``SeparableHistory``.

    spectrum : "band" -> flat up to a quarter of the Nyquist wavenumber;
               "k2"   -> amplitude 1/(1+(k/k0)^2), k0 = 2 pi / (32 dx);
               "flat" -> unit amplitude everywhere.
    sparse   : if an int, only that many random half-spectrum bins per term
               are non-zero (their spectra are exact in ``Uhat``).
    bins     : if given, flat indices r3 (n1/2+1) + j1 of the half-spectrum
               bins that are non-zero in every term (plus the partners that
               the real-field symmetry of the j1 = 0 and j1 = n1/2 columns
               adds), exact in ``Uhat``.
    """
    rng = np.random.default_rng(seed)
    nh = n1 // 2 + 1
    j1 = np.arange(nh)[None, :]
    r3 = np.arange(n3)[:, None]
    j3 = np.where(r3 <= n3 // 2, r3, r3 - n3)
    k1 = 2 * np.pi * j1 / L1
    k3 = 2 * np.pi * j3 / L3
    kk = np.hypot(k1, k3)
    dx = min(L1 / n1, L3 / n3)
    k_nyq = np.pi / dx
    if spectrum == "band":
        shape = (kk <= 0.25 * k_nyq).astype(float)
    elif spectrum == "k2":
        k0 = 2 * np.pi / (32 * dx)
        shape = 1.0 / (1.0 + (kk / k0) ** 2)
    elif spectrum == "flat":
        shape = np.ones_like(kk)
    else:
        raise ValueError(spectrum)
    U = np.empty((n_terms, 3, n3, n1))
    Uh = np.empty((n_terms, 3, n3, nh), dtype=complex)
    for r in range(n_terms):
        for c in range(3):
            spec = (rng.normal(size=(n3, nh)) + 1j * rng.normal(size=(n3, nh))) * shape
            if sparse is not None:
                keep = np.zeros(n3 * nh, dtype=bool)
                keep[rng.choice(n3 * nh, size=min(sparse, n3 * nh), replace=False)] = True
                spec = spec * keep.reshape(n3, nh)
            if bins is not None:
                keep = np.zeros(n3 * nh, dtype=bool)
                keep[np.asarray(bins)] = True
                spec = spec * keep.reshape(n3, nh)
            field = np.fft.irfft2(spec, s=(n3, n1))
            sp = np.fft.rfft2(field)                # the spectrum the field really has
            if sparse is not None or bins is not None:   # drop FFT round-off outside the bins
                sp[np.abs(sp) < 1e-9 * np.abs(sp).max()] = 0.0
                field = np.fft.irfft2(sp, s=(n3, n1))
            Uh[r, c] = sp
            U[r, c] = field
    rms = np.sqrt(np.mean(U ** 2)) * np.sqrt(n_terms)
    if rms > 0:
        U *= amp_rms / rms
        Uh *= amp_rms / rms
    omega_max = 0.25 * k_nyq * cs
    g = np.stack([_temporal(rng, steps, dt, omega_max) for _ in range(n_terms)])
    return SeparableHistory(U=U, Uhat=Uh, g=g, dt=dt)


def config_small():
    """Single half-space, 64 x 64 periodic grid, dx = 100 m, c_s = 3464 m/s,
    c_p = 6000 m/s, rho = 2670 kg/m^3, dt = 0.3 dx / c_p, 256-lag cutoff,
    200 steps (the small FP64 comparison case)."""
    dx = 100.0
    return dict(n1=64, n3=64, L1=64 * dx, L3=64 * dx, cs=3464.0, cp=6000.0,
                rho=2670.0, dt=0.3 * dx / 6000.0, n_cut=256, steps=200)


def config_large():
    """Single half-space, 1024 x 1024 grid, dx = 100 m, same material,
    4096-lag cutoff (the bandwidth case)."""
    dx = 100.0
    return dict(n1=1024, n3=1024, L1=1024 * dx, L3=1024 * dx, cs=3464.0,
                cp=6000.0, rho=2670.0, dt=0.3 * dx / 6000.0, n_cut=4096)
