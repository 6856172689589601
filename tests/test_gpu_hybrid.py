"""GPU hybrid FEM-SBIM step (Sections 2.1, 2.2, 2.4) against the FP64 oracle,
through the C ABI, and the non-reflection check of the coupled GPU path."""
import numpy as np
import pytest

from oracle.fem_oracle import FaultLaw, HybridOracle, SlabMesh
from tests._errors import Worst, assert_finite, rel_l2_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


rel = rel_l2_field


def regime_stats(rates, refs, thr=1e-3):
    """Where a lower-precision rupture departs from the FP64 one: the number of
    nodes that slip (|slip rate| > thr m/s) at some step in one run but not in
    the other, and the slip-rate error (max over steps and nodes, relative to the
    FP64 peak) inside and outside that set of nodes."""
    rates, refs = np.array(rates), np.array(refs)
    assert_finite(rates, "slip rate")
    mag = lambda x: np.sqrt((x ** 2).sum(axis=1))           # noqa: E731  (steps, n3, n1)
    a, b = mag(rates) > thr, mag(refs) > thr
    switch = (a != b).any(axis=0)
    peak = np.abs(refs).max()
    d = np.abs(rates - refs).max(axis=(0, 1))
    inside = d[switch].max() / peak if switch.any() else 0.0
    outside = d[~switch].max() / peak if (~switch).any() else 0.0
    return int(switch.sum()), switch.size, inside, outside, d.max() / peak, peak


def regime_report(title, rates, refs, thr=1e-3):
    n, total, inside, outside, overall, peak = regime_stats(rates, refs, thr)
    return (f"{title}: {n} of {total} nodes change regime at another step; "
            f"slip-rate error inside {inside:.3e}, outside {outside:.3e}, overall "
            f"{overall:.3e} of the peak {peak:.3f} m/s")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 5e-6)])
@pytest.mark.parametrize("fault,boundaries", [(False, True), (True, True), (True, False)])
def test_linear_slab_matches_oracle(precision, tol, fault, boundaries):
    """Random initial state, SBIM or free boundaries, welded split plane or none:
    u, v, a after 30 steps equal the oracle's, each within one bound (the map is
    linear, so float rounding stays at its own level: measured 4e-7 to 6e-7 in
    FP32 and 1e-12 in FP64 for all three fields)."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n1, n2, n3, h, n_cut, steps = 8, 4, 6, 50.0, 12, 30
    dt = 0.3 * h / CP
    me = SlabMesh(n1, n2, n3, h, fault=fault)
    o = HybridOracle(me, CS, CP, RHO, dt, n_cut=n_cut, sbim=boundaries)
    rng = np.random.default_rng(3)
    o.u = rng.normal(size=o.u.shape) * 1e-3
    o.v = rng.normal(size=o.u.shape) * 1e-2
    if fault:
        o.u[me.f + 1] = o.u[me.f]
        o.v[me.f + 1] = o.v[me.f]
    dtype = torch.float64 if precision == "fp64" else torch.float32
    g = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, n_cut, precision, boundaries, fault)
    g.set_state(torch.from_numpy(o.u).to("cuda", dtype), torch.from_numpy(o.v).to("cuda", dtype),
                None)
    for _ in range(steps):
        o.step()
        g.step()
    u, v, a = (x.double().cpu().numpy() for x in g.get_state())
    print(f"\nSLAB-REPORT {precision} fault={fault} sbim={boundaries}: relative L2 error "
          f"u {rel(u, o.u):.3e} v {rel(v, o.v):.3e} a {rel(a, o.a):.3e}")
    assert rel(u, o.u) < tol
    assert rel(v, o.v) < tol
    assert rel(a, o.a) < tol
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 5e-6)])
@pytest.mark.parametrize("n1,n3", [(40, 10), (64, 6)])
def test_force_tiles_with_ragged_edges(precision, tol, n1, n3):
    """The force kernel marches columns in tiles of 32 x 4 with a periodic halo:
    grids that span several tiles with a ragged last one in x1 (40) or x3 (10,
    6) and wrap across tile edges, with a split plane and both half-spaces,
    equal the oracle after 20 steps."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n2, h, n_cut, steps = 4, 50.0, 12, 20
    dt = 0.3 * h / CP
    me = SlabMesh(n1, n2, n3, h, fault=True)
    o = HybridOracle(me, CS, CP, RHO, dt, n_cut=n_cut, sbim=True)
    rng = np.random.default_rng(5)
    o.u = rng.normal(size=o.u.shape) * 1e-3
    o.v = rng.normal(size=o.u.shape) * 1e-2
    o.u[me.f + 1] = o.u[me.f]
    o.v[me.f + 1] = o.v[me.f]
    dtype = torch.float64 if precision == "fp64" else torch.float32
    g = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, n_cut, precision, True, True)
    g.set_state(torch.from_numpy(o.u).to("cuda", dtype), torch.from_numpy(o.v).to("cuda", dtype),
                None)
    for _ in range(steps):
        o.step()
        g.step()
    u, v, a = (assert_finite(x.double().cpu().numpy(), "state") for x in g.get_state())
    print(f"\nTILES-REPORT {precision} {n1}x{n3}: relative L2 error u {rel(u, o.u):.3e} "
          f"v {rel(v, o.v):.3e} a {rel(a, o.a):.3e}")
    assert rel(u, o.u) < tol
    assert rel(v, o.v) < tol
    assert rel(a, o.a) < tol
    g.close()


def _rupture_setup(n1, n3):
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    patch = (np.abs(i1 - n1 / 2 + 0.5) < 3) & (np.abs(i3 - n3 / 2 + 0.5) < 3)
    mu_s = np.full((n3, n1), 0.677)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    return mu_s, tau0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_rupture_matches_oracle(precision, tol):
    """Slip-weakening rupture from an overstressed patch (TPV3-like stresses,
    Dc scaled to the small fault): the slip-rate field over 45 steps, within
    `tol` of the FP64 oracle's peak slip rate at every node and step.  The stick
    or slip decision of the fault law is a threshold, so a node whose FP32
    traction crossed the strength one step off would carry an O(1) local error;
    no node does here (every node slips or sticks at the same steps as in the
    oracle), and the FP32 error stays at the float rounding of the coupled
    update (measured 3.4e-6 of the peak)."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n1 = n3 = 32
    n2, h, steps = 4, 100.0, 45
    dt = 0.3 * h / CP
    mu_s, tau0 = _rupture_setup(n1, n3)
    me = SlabMesh(n1, n2, n3, h, fault=True)
    o = HybridOracle(me, CS, CP, RHO, dt, n_cut=steps + 1,
                     fault=FaultLaw(mu_s, 0.525, 0.02, tau0, 120e6))
    g = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, steps + 1, precision, True, True)
    g.set_fault(mu_s, tau0, 0.525, 0.02, 120e6)
    worst, peak = Worst(), Worst()
    rates, refs = [], []
    for _ in range(steps):
        o.step()
        g.step()
        slip, rate, trac = (x.double().cpu().numpy() for x in g.fault_fields())
        assert_finite(slip, "slip")
        assert_finite(trac, "traction")
        peak.update(np.abs(o.slip_rate).max())
        rates.append(rate)
        refs.append(o.slip_rate.copy())
        if np.linalg.norm(o.slip_rate) > 0:
            worst.update(rel(rate, o.slip_rate))
    print("\n" + regime_report(f"RUPTURE-REPORT hybrid {precision}", rates, refs))
    switched, _, _, _, overall, _ = regime_stats(rates, refs)
    assert float(peak) > 1.0
    assert switched == 0
    assert overall < tol, overall
    g.close()


def test_fault_solution_independent_of_strip_width():
    """The paper's validation of the hybrid scheme by varying the strip width
    L2 (Sections 3 and 4): the slip rate at a station off the nucleation patch
    is the same for L2 = 4 dx and 8 dx, and each GPU run (FP64) follows the
    oracle's run of the same slab."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n1 = n3 = 32
    h, steps = 100.0, 45
    dt = 0.3 * h / CP
    mu_s, tau0 = _rupture_setup(n1, n3)
    station = (n3 // 2, n1 // 2 + 4)
    traces = {}
    for n2 in (4, 8):
        o = HybridOracle(SlabMesh(n1, n2, n3, h, fault=True), CS, CP, RHO, dt, n_cut=steps + 1,
                         fault=FaultLaw(mu_s, 0.525, 0.02, tau0, 120e6))
        g = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, steps + 1, "fp64", True, True)
        g.set_fault(mu_s, tau0, 0.525, 0.02, 120e6)
        got, ref = [], []
        for _ in range(steps):
            o.step()
            g.step()
            got.append(float(assert_finite(g.fault_fields()[1])[0][station]))
            ref.append(o.slip_rate[0][station])
        g.close()
        got, ref = np.array(got), np.array(ref)
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()
        traces[n2] = got
    a, b = traces[4], traces[8]
    assert np.abs(a).max() > 1.0                     # the rupture reached the station
    assert np.abs(a - b).max() < 0.1 * np.abs(a).max()


def test_gpu_sbim_boundaries_reproduce_an_unbounded_slab():
    """The coupled GPU path: a force pulse in a thin slab with SBIM half-spaces
    moves like the same pulse in a thick free slab until reflections return."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n1 = n3 = 16
    n2, pad, h, steps = 8, 16, 50.0, 60
    dt = 0.3 * h / CP
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")

    def source(layers, first, n):
        out = np.zeros((layers, 3, n3, n1), dtype=np.float32)
        if n <= 12:
            L = np.arange(layers)[:, None, None] - first
            g = np.exp(-((i1 - n1 / 2) ** 2 + (i3 - n3 / 2) ** 2 + (L - n2 / 2) ** 2) / 4.5)
            amp = np.sin(np.pi * n / 12) ** 2 * 1e9
            out[:, 1] = amp * g
            out[:, 0] = 0.5 * amp * g
        return torch.from_numpy(out).cuda()

    thin = Hybrid(n1, n2, n3, h, CS, CP, RHO, dt, steps + 1, "fp32", True, False)
    thick = Hybrid(n1, n2 + 2 * pad, n3, h, CS, CP, RHO, dt, steps + 1, "fp32", False, False)
    worst = Worst()
    for n in range(1, steps + 1):
        thin.step(source(n2 + 1, 0, n))
        thick.step(source(n2 + 2 * pad + 1, pad, n))
        ut = thin.get_state()[0].double().cpu().numpy()
        ur = thick.get_state()[0].double().cpu().numpy()[pad:pad + n2 + 1]
        worst.update(rel(ut, ur))
    assert worst.value < 0.08, worst


def test_coupled_configuration_fp32_against_fp64_and_mirror_symmetry():
    """The coupled configuration at full size: 512 x 16 x 512 slab, two 512²
    half-spaces with 2000-lag cutoffs, TPV3 stresses.  Over the first 60 steps
    of the rupture the FP32 path follows the FP64 path (the one checked against
    the oracle at small sizes) within the rupture tolerance, and the FP64
    solution keeps the mirror symmetry of the setup about the fault plane: the
    top and bottom SBIM tractions are mirror images (tau_1,3 equal, tau_2
    opposite), and the fault's normal traction perturbation stays at rounding."""
    from paper_2102_08756_gb300.hybrid import Hybrid
    n, n2, h, n_cut, steps = 512, 16, 100.0, 2000, 60
    dt = 0.3 * h / CP
    x = (np.arange(n) - n / 2 + 0.5) * h
    X3, X1 = np.meshgrid(x, x, indexing="ij")
    inside = (np.abs(X1) <= 15e3) & (np.abs(X3) <= 7.5e3)
    patch = (np.abs(X1) <= 1.5e3) & (np.abs(X3) <= 1.5e3)
    law = (np.where(inside, 0.677, 1e4), np.where(patch, 1.005 * 0.677 * 120e6, 70e6),
           0.525, 0.4, 120e6)
    runs = {}
    for prec in ("fp64", "fp32"):
        g = Hybrid(n, n2, n, h, CS, CP, RHO, dt, n_cut, prec)
        g.set_fault(*law)
        rates = []
        for _ in range(steps):
            g.step()
            rates.append(g.fault_fields()[1].double())
        top, bot = (t.double() for t in g.boundary_tractions())
        trac = g.fault_fields()[2].double()
        runs[prec] = (torch.stack(rates), top, bot, trac)
        g.close()
    r64, top, bot, trac = runs["fp64"]
    r32 = runs["fp32"][0]
    print("\n" + regime_report("RUPTURE-REPORT coupled 512x16x512 fp32 vs fp64",
                                list(r32.cpu().numpy()), list(r64.cpu().numpy())))
    assert float(r64.abs().max()) > 1.0                          # the rupture runs
    assert float((r32 - r64).abs().max()) < 3e-3 * float(r64.abs().max())
    scale = float(top.abs().max())
    assert float((top[0] - bot[0]).abs().max()) < 1e-9 * scale
    assert float((top[2] - bot[2]).abs().max()) < 1e-9 * scale
    assert float((top[1] + bot[1]).abs().max()) < 1e-9 * scale
    assert float(trac[1].abs().max()) < 1e-9 * float(trac.abs().max())
