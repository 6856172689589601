"""GPU pure-SBIM fault solver (include/sbim.h, sbim_fault_*) against the FP64
oracle (oracle/fault_oracle.py), through the C ABI; and the paper's TPV3 check
(Section 3): the hybrid FEM-SBIM run agrees with the SBIM-only run.

Bounds, relative to each field's peak over the run (slip rate, slip, traction)
of a nucleating rupture: FP64 1e-10; FP32 (Kahan-summed float history) 1e-4.
The stick/slip decision is a threshold, so a node that changed regime one step
off would carry an O(1) local error; in these runs no node does (asserted), and
the FP32 slip rate stays within 1e-5 of its peak (measured)."""
import numpy as np
import pytest

from oracle.fault_oracle import FaultLaw, PureSBIMOracle
from tests._errors import assert_finite, max_abs_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0
DX = 100.0
DT = 0.3 * DX / CP


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _law(n1, n3, half, Dc, outside=0.677):
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    patch = (np.abs(i1 - n1 / 2 + 0.5) < half) & (np.abs(i3 - n3 / 2 + 0.5) < half)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    return FaultLaw(np.full((n3, n1), outside), 0.525, Dc, tau0, 120e6)


def _solver(n1, n3, n_cut, fl, precision, symmetric):
    from paper_2102_08756_gb300.fault import FaultSolver
    g = FaultSolver(n1, n3, n1 * DX, n3 * DX, CS, CP, RHO, DT, n_cut, precision, symmetric)
    if fl is not None:
        g.set_fault(fl.mu_s, fl.tau0, fl.mu_k, fl.Dc, fl.sigma0)
    return g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
@pytest.mark.parametrize("symmetric", [False, True])
@pytest.mark.parametrize("n1,n3,n_cut", [(24, 16, 50), (20, 20, 13)])
def test_rupture_matches_oracle(precision, tol, symmetric, n1, n3, n_cut):
    steps = 50
    fl = _law(n1, n3, 3.5, 0.05)
    o = PureSBIMOracle(n1, n3, n1 * DX, n3 * DX, CS, CP, RHO, DT, n_cut, fl, symmetric=symmetric)
    g = _solver(n1, n3, n_cut, fl, precision, symmetric)
    got, ref = {"rate": [], "slip": [], "traction": []}, {"rate": [], "slip": [], "traction": []}
    for _ in range(steps):
        o.step()
        g.step()
        slip, rate, trac = (x.double().cpu().numpy() for x in g.fault_fields())
        for name, x, r in (("rate", rate, o.slip_rate), ("slip", slip, o.slip),
                           ("traction", trac, o.fault_traction)):
            got[name].append(assert_finite(x, name))
            ref[name].append(np.array(r, copy=True))
    worst = {name: max_abs_rel(np.array(got[name]), np.array(ref[name])) for name in got}
    peak = np.abs(np.array(ref["rate"])).max()
    from tests.test_gpu_hybrid import regime_report, regime_stats
    print("\n" + regime_report(f"RUPTURE-REPORT sbim {precision} sym={symmetric} {n1}x{n3}",
                                got["rate"], ref["rate"])
          + f"; slip {worst['slip']:.3e}, traction {worst['traction']:.3e} of their peaks")
    assert peak > 1.0, peak                         # the rupture runs
    assert regime_stats(got["rate"], ref["rate"])[0] == 0
    assert all(w < tol for w in worst.values()), worst
    u, v = (x.double().cpu().numpy() for x in g.get_state())
    assert_finite(v, "v")
    assert max_abs_rel(u, o.u) < tol


def test_uniform_overstress_slides_at_radiation_rate():
    n1, n3 = 16, 8
    tau0, sigma0, mu_f = 80e6, 120e6, 0.5
    fl = FaultLaw(np.full((n3, n1), mu_f), mu_f, 0.4, np.full((n3, n1), tau0), sigma0)
    V = 2.0 * CS * (tau0 - mu_f * sigma0) / (RHO * CS * CS)
    for symmetric in (False, True):
        g = _solver(n1, n3, 16, fl, "fp64", symmetric)
        for n in range(1, 11):
            g.step()
            slip, rate, trac = (x.cpu().numpy() for x in g.fault_fields())
            np.testing.assert_allclose(rate[0], V, rtol=1e-12)
            np.testing.assert_allclose(trac[0], mu_f * sigma0 - tau0, rtol=1e-12)
            np.testing.assert_allclose(slip[0], (n - 0.5) * DT * V, rtol=1e-12, atol=1e-15)
        assert g.steps == 10


@pytest.mark.parametrize("symmetric", [False, True])
def test_highest_modes_stay_bounded(symmetric):
    """Frictionless fault with a zero-mean random prestress on an 8 x 8 grid,
    2000 steps (|k| c_s dt up to 0.77): the predictor-corrector keeps the slip
    rate at its first-step size."""
    n = 8
    rng = np.random.default_rng(0)
    tau0 = rng.normal(size=(n, n)) * 1e6
    tau0 -= tau0.mean()
    g = _solver(n, n, 2000, FaultLaw(np.zeros((n, n)), 0.0, 0.4, tau0, 1e8), "fp32", symmetric)
    g.step()
    first = float(g.fault_fields()[1].abs().max())
    peak = torch.zeros((), device="cuda")
    for _ in range(1999):
        g.step()
        peak = torch.maximum(peak, g.fault_fields()[1].abs().max())
    assert float(peak) < 2.0 * first, (float(peak), first)


def test_symmetric_equals_two_half_spaces_and_keeps_normal_stress():
    n = 32
    fl = _law(n, n, 4, 0.08)
    a = _solver(n, n, 60, fl, "fp64", False)
    b = _solver(n, n, 60, fl, "fp64", True)
    assert b.handles()[1] is None and a.handles()[1] is not None
    for _ in range(60):
        a.step()
        b.step()
    ra, rb = a.fault_fields()[1].cpu().numpy(), b.fault_fields()[1].cpu().numpy()
    assert np.abs(ra).max() > 1.0
    assert np.abs(ra - rb).max() < 1e-9 * np.abs(ra).max()
    assert np.abs(a.fault_fields()[2][1].cpu().numpy()).max() < 1e-3   # tau_2 perturbation (Pa)
    u = a.get_state()[0].cpu().numpy()
    np.testing.assert_allclose(u[1], PureSBIMOracle.mirror(u[0]), atol=1e-12)


def test_state_round_trip_and_welded_default():
    n1, n3 = 16, 16
    g = _solver(n1, n3, 8, None, "fp32", False)     # no law: welded
    rng = np.random.default_rng(3)
    u0 = torch.from_numpy(rng.standard_normal((2, 3, n3, n1)).astype(np.float32) * 1e-3).cuda()
    v0 = torch.from_numpy(rng.standard_normal((2, 3, n3, n1)).astype(np.float32) * 1e-2).cuda()
    g.set_state(u0, v0)
    u, v = g.get_state()
    assert torch.equal(u, u0) and torch.equal(v, v0)
    g.step()
    rate = g.fault_fields()[1]
    assert float(rate.abs().max()) == 0.0           # welded: no slip rate
    s = _solver(n1, n3, 8, None, "fp32", True)
    s.set_state(u0, v0)
    u, _ = s.get_state()
    mirror = torch.tensor([-1.0, 1.0, -1.0], device="cuda").view(3, 1, 1)
    assert torch.equal(u[1], u0[0] * mirror)


def test_tpv3_hybrid_agrees_with_pure_sbim():
    """Section 3 at dx = 100 m (the paper uses 50 m): TPV3's 30 x 15 km fault with
    a 3 km nucleation patch, unbreakable outside, on a 51.2 x 25.6 km periodic
    plane; the hybrid run uses a slab of L2 = 4 dx.  Rupture arrival times
    (slip > 1 mm) and the slip after 3.5 s agree with the pure-SBIM run."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n1, n3, steps = 512, 256, 700
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    x1 = (i1 - n1 / 2 + 0.5) * DX
    x3 = (i3 - n3 / 2 + 0.5) * DX
    inside = (np.abs(x1) < 15e3) & (np.abs(x3) < 7.5e3)
    patch = (np.abs(x1) < 1.5e3) & (np.abs(x3) < 1.5e3)
    mu_s = np.where(inside, 0.677, 1e4)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    law = (mu_s, tau0, 0.525, 0.4, 120e6)
    hy = Hybrid(n1, 4, n3, DX, CS, CP, RHO, DT, steps, "fp32")
    hy.set_fault(*law)
    ps = _solver(n1, n3, steps, None, "fp32", True)
    ps.set_fault(*law)
    t_h = torch.full((n3, n1), float("inf"), device="cuda")
    t_p = torch.full((n3, n1), float("inf"), device="cuda")
    for m in range(steps):
        hy.step()
        ps.step()
        sh = hy.fault_fields()[0]
        sp = ps.fault_fields()[0]
        mag_h = torch.hypot(sh[0], sh[2])
        mag_p = torch.hypot(sp[0], sp[2])
        t_h = torch.where((mag_h > 1e-3) & torch.isinf(t_h), float(m), t_h)
        t_p = torch.where((mag_p > 1e-3) & torch.isinf(t_p), float(m), t_p)
    t_h, t_p = t_h.cpu().numpy(), t_p.cpu().numpy()
    both = np.isfinite(t_h) & np.isfinite(t_p)
    either = np.isfinite(t_h) | np.isfinite(t_p)
    rms = np.sqrt(np.mean((t_h[both] - t_p[both]) ** 2)) / np.mean(t_p[both])
    mag_h, mag_p = mag_h.cpu().numpy(), mag_p.cpu().numpy()
    slip_diff = np.linalg.norm(mag_h - mag_p) / np.linalg.norm(mag_p)
    print(f"TPV3-REPORT ruptured {both.sum()} of {either.sum()} nodes; rms arrival difference "
          f"{rms:.4f} of the mean arrival; final slip rel L2 difference {slip_diff:.4f}; "
          f"max slip {mag_p.max():.3f} m")
    assert both.sum() > 0.35 * inside.sum() and both.sum() > 0.95 * either.sum()
    assert rms < 0.05 and slip_diff < 0.05
