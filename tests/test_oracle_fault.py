"""Pins of the pure-SBIM fault oracle (oracle/fault_oracle.py) against what
the mathematics and the paper fix, not against itself:

* a spatially uniform overstressed fault slides at the rate set by the two
  radiation impedances, V = 2 c_s (tau0 - tau_f)/mu, from its first step (the
  k = 0 mode has no non-local term, Section 2.3);
* a frictionless fault under a sinusoidal prestress converges at second order
  in dt to the continuum solution of the two-half-space problem: for slip
  normal to the wavevector (mode III) delta(t) = (2 A/(mu k)) int_0^{k c_s t} J0,
  and for slip along it (mode II) the inverse Laplace transform of
  2 A/(mu k p M(p)), M = K11 - G^2/K22 (the normal displacement adjusts so
  sigma_22 stays continuous), computed by fixed-Talbot inversion (Abate &
  Valko 2004);
* the predictor-corrector stays bounded at the highest modes, where the
  one-evaluation explicit update grows without bound;
* the symmetry-plane reduction of Section 3 equals the two-half-space solver on
  a symmetric problem, and the normal traction does not change;
* the paper's validation of the hybrid scheme (Section 3): a rupture computed by
  the hybrid FEM-SBIM oracle with a thin slab agrees with the pure-SBIM one, and
  the two approach each other as the grid is refined.
"""
import numpy as np
import pytest
import scipy.special as sp
from scipy.integrate import quad

from oracle.fault_oracle import FaultLaw, PureSBIMOracle
from oracle.fem_oracle import HybridOracle, SlabMesh
from oracle.sbim_oracle import laplace_symbols
from tests._errors import Worst

CS, CP, RHO = 3464.0, 6000.0, 2670.0
MU = RHO * CS * CS
DX = 100.0
DT = 0.3 * DX / CP


def test_uniform_overstress_slides_at_radiation_rate():
    n1, n3 = 8, 6
    tau0, sigma0, mu_f = 80e6, 120e6, 0.5            # strength 60 MPa everywhere
    fl = FaultLaw(np.full((n3, n1), mu_f), mu_f, 0.4, np.full((n3, n1), tau0), sigma0)
    V = 2.0 * CS * (tau0 - mu_f * sigma0) / MU
    for sym in (False, True):
        o = PureSBIMOracle(n1, n3, n1 * DX, n3 * DX, CS, CP, RHO, DT, 16, fl, symmetric=sym)
        for n in range(1, 13):
            o.step()
            np.testing.assert_allclose(o.slip_rate[0], V, rtol=1e-12)
            np.testing.assert_allclose(o.slip_rate[2], 0.0, atol=1e-12 * V)
            np.testing.assert_allclose(o.fault_traction[0], mu_f * sigma0 - tau0, rtol=1e-12)
            # trapezoidal slip from rest: the rate jumps to V in the first step
            np.testing.assert_allclose(o.slip[0], (n - 0.5) * DT * V, rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(o.u[0, 0], -o.u[1, 0], rtol=1e-12)


def _frictionless_slip(n1, n3, tau0, dt, T_end, k, station):
    steps = int(round(T_end / (k * CS * dt)))
    fl = FaultLaw(np.zeros((n3, n1)), 0.0, 0.4, tau0, 1e8)
    o = PureSBIMOracle(n1, n3, n1 * DX, n3 * DX, CS, CP, RHO, dt, steps + 2, fl)
    out = []
    for _ in range(steps):
        o.step()
        out.append(o.slip[0][station])
    return np.array(out)


def _errors(n1, n3, tau0, k, station, exact, T_end):
    """Max error of the runs at dt, dt/2, dt/4, each compared with the continuum
    solution at t_n - dt/2 (trapezoidal start from rest: the prestress acts
    from the first step, whose slip rate jumps to its full value)."""
    out = []
    for f in (1, 2, 4):
        h = DT / f
        x = _frictionless_slip(n1, n3, tau0, h, T_end, k, station)
        ts = (np.arange(len(x)) + 0.5) * h
        out.append(np.abs(x - np.array([exact(k * CS * t) for t in ts])).max())
    return out


def _talbot(F, t, M=48):
    """Fixed-Talbot inverse Laplace transform (Abate & Valko 2004) of F at t."""
    r = 2.0 * M / (5.0 * t)
    th = np.arange(1, M) * np.pi / M
    cot = 1.0 / np.tan(th)
    s = r * th * (cot + 1j)
    sig = th + (th * cot - 1.0) * cot
    total = 0.5 * np.exp(r * t) * F(np.array([r + 0j]))[0]
    total += np.sum((np.exp(t * s) * F(s) * (1.0 + 1j * sig)).real)
    return float((r / M * total).real)


def test_mode_iii_converges_to_closed_form():
    n1, n3, A = 4, 16, 1e6
    k = 2 * np.pi / (n3 * DX)
    x3 = np.arange(n3) * DX
    tau0 = A * np.cos(k * x3)[:, None] * np.ones((n3, n1))      # x1 shear varying along x3
    scale = 2 * A / (MU * k)
    exact = lambda T: scale * quad(sp.j0, 0.0, T, limit=200)[0]  # noqa: E731
    e1, e2, e4 = _errors(n1, n3, tau0, k, (0, 0), exact, 12.0)
    assert e1 < 1e-3 * scale and e4 < 5e-5 * scale
    assert 3.5 < e1 / e2 < 4.5 and 3.5 < e2 / e4 < 4.5        # second order


def test_mode_ii_converges_to_laplace_inversion():
    n1, n3, A = 16, 4, 1e6
    eta = CP / CS
    k = 2 * np.pi / (n1 * DX)
    x1 = np.arange(n1) * DX
    tau0 = A * np.cos(k * x1)[None, :] * np.ones((n3, n1))      # x1 shear varying along x1
    scale = 2 * A / (MU * k)

    def F(p):
        K11, K22, _, G = laplace_symbols(p, eta)
        return 1.0 / (p * (K11 - G * G / K22))

    # the inversion itself: the two node counts agree, and the mode-III symbol
    # reproduces the J0 integral
    for T in (0.5, 3.0, 10.0):
        assert abs(_talbot(F, T, 40) - _talbot(F, T, 48)) < 1e-7
        F3 = lambda p: 1.0 / (p * laplace_symbols(p, eta)[2])  # noqa: E731
        assert abs(_talbot(F3, T) - quad(sp.j0, 0.0, T, limit=200)[0]) < 1e-7
    exact = lambda T: 0.0 if T == 0 else scale * _talbot(F, T)  # noqa: E731
    e1, e2, e4 = _errors(n1, n3, tau0, k, (0, 0), exact, 10.0)
    assert e1 < 2e-3 * scale and e4 < 1e-4 * scale
    assert 3.5 < e1 / e2 < 4.5 and 3.5 < e2 / e4 < 4.5
    # the static limit 1/M(0) = 1/(2 (1 - c_s^2/c_p^2)) is the plane-strain
    # compliance 1 - nu: the time average of the response approaches it
    assert abs(1.0 / (F(np.array([1e-9 + 0j]))[0] * 1e-9) - 2 * (1 - 1 / eta ** 2)) < 1e-6


def test_highest_modes_stay_bounded():
    """Frictionless fault, random prestress on a 4 x 4 grid (every mode at or
    near the Nyquist limit, |k| c_s dt up to 0.77): the slip rate stays at its
    first-step size over 1500 steps."""
    n = 4
    rng = np.random.default_rng(0)
    tau0 = rng.normal(size=(n, n)) * 1e6
    tau0 -= tau0.mean()
    fl = FaultLaw(np.zeros((n, n)), 0.0, 0.4, tau0, 1e8)
    for sym in (True, False):
        o = PureSBIMOracle(n, n, n * DX, n * DX, CS, CP, RHO, DT, 1501, fl, symmetric=sym)
        o.step()
        first = np.abs(o.slip_rate).max()
        peak = Worst()
        for _ in range(1499):
            o.step()
            peak.update(np.abs(o.slip_rate).max())
        assert float(peak) < 2.0 * first, (peak, first)


def _tpv3_like(n, half, Dc, mu_s_out=0.677):
    i3, i1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    patch = (np.abs(i1 - n / 2 + 0.5) < half) & (np.abs(i3 - n / 2 + 0.5) < half)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    return FaultLaw(np.full((n, n), mu_s_out), 0.525, Dc, tau0, 120e6)


def test_symmetric_reduction_equals_two_half_spaces():
    n, steps = 24, 40
    fl = _tpv3_like(n, 4, 0.08)
    a = PureSBIMOracle(n, n, n * DX, n * DX, CS, CP, RHO, DT, steps, fl)
    b = PureSBIMOracle(n, n, n * DX, n * DX, CS, CP, RHO, DT, steps, fl, symmetric=True)
    for _ in range(steps):
        a.step()
        b.step()
        assert np.abs(a.fault_traction[1]).max() < 1e-6   # sigma_22 unchanged (Pa)
        scale = np.abs(a.slip_rate).max() + 1e-30
        assert np.abs(a.slip_rate - b.slip_rate).max() < 1e-9 * scale
    assert np.abs(a.slip_rate).max() > 1.0                 # the rupture runs
    np.testing.assert_allclose(a.u[1], PureSBIMOracle.mirror(a.u[0]), atol=1e-12)
    np.testing.assert_allclose(a.u, b.u, atol=1e-12)


def _arrivals_and_slip(n, half, Dc, steps):
    fl = _tpv3_like(n, half, Dc)
    dt = DT
    hy = HybridOracle(SlabMesh(n, 4, n, DX, fault=True), CS, CP, RHO, dt, n_cut=steps + 1, fault=fl)
    ps = PureSBIMOracle(n, n, n * DX, n * DX, CS, CP, RHO, dt, steps + 1, fl)
    t_h = np.full((n, n), np.inf)
    t_p = np.full((n, n), np.inf)
    for m in range(steps):
        hy.step()
        ps.step()
        d = hy.u[hy.mesh.f + 1] - hy.u[hy.mesh.f]
        s_h = np.hypot(d[0], d[2])
        s_p = np.hypot(ps.slip[0], ps.slip[2])
        t_h = np.where((s_h > 1e-3) & np.isinf(t_h), m, t_h)
        t_p = np.where((s_p > 1e-3) & np.isinf(t_p), m, t_p)
    both = np.isfinite(t_h) & np.isfinite(t_p)
    rms = np.sqrt(np.mean((t_h[both] - t_p[both]) ** 2)) / np.mean(t_p[both])
    slip_diff = np.linalg.norm(s_h - s_p) / np.linalg.norm(s_p)
    agree = both.sum() / max(np.isfinite(t_h).sum(), np.isfinite(t_p).sum())
    return rms, slip_diff, agree


def test_rupture_agrees_with_hybrid_and_converges():
    """Section 3 compares the hybrid scheme (a slab of four elements across, here
    L2 = 4 dx) with an SBIM-only solution of the same rupture.  Same fault, patch
    and prestress at two resolutions (the cohesive zone resolved by ~2.5 and ~5
    cells): rupture arrival times and the final slip agree, and agree better on
    the finer grid."""
    rms32, slip32, agree32 = _arrivals_and_slip(32, 6, 0.16, 80)
    rms64, slip64, agree64 = _arrivals_and_slip(64, 12, 0.32, 150)
    assert agree32 > 0.85 and agree64 > 0.95
    assert rms64 < 0.06 and slip64 < 0.03
    assert slip64 < 0.5 * slip32 and rms64 < 0.5 * rms32
