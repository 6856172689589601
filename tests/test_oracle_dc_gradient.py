"""Pins of the oracle's gradient of a fault-traction functional with respect to
the slip-weakening distance Dc through the coupled FEM-SBIM run (Sections 2.1,
2.2, 2.4): central finite differences in Dc (uniform and one node), and in the
initial displacement, with a check that no node changes its stick/slip regime
between the perturbed runs.  Also: the step-wise SBIM adjoint equals the
whole-sequence transpose."""
import numpy as np

from oracle.fem_oracle import FaultLaw, HybridOracle, SlabMesh, dc_gradient, forward_record
from oracle.sbim_oracle import SBIMAdjointOracle, adjoint_sequence

CS, CP, RHO = 3464.0, 6000.0, 2670.0


def test_stepwise_sbim_adjoint_equals_sequence_transpose():
    rng = np.random.default_rng(0)
    n1, n3, n_cut, steps = 8, 6, 5, 11
    dt = 0.3 * 100.0 / CP
    tb = rng.normal(size=(steps, 3, n3, n1))
    ub, vb = adjoint_sequence(n1, n3, 800.0, 600.0, CS, CP, RHO, dt, n_cut, -1, tb)
    adj = SBIMAdjointOracle(n1, n3, 800.0, 600.0, CS, CP, RHO, dt, n_cut, -1)
    for m in range(steps - 1, -1, -1):
        u, v = adj.step(tb[m])
        np.testing.assert_allclose(u, ub[m], rtol=1e-12, atol=1e-12 * np.abs(ub).max())
        np.testing.assert_allclose(v, vb[m], rtol=1e-14)


def _setup(Dc, n1=16, n2=4, n3=16, steps=30):
    h = 100.0
    dt = 0.3 * h / CP
    me = SlabMesh(n1, n2, n3, h, fault=True)
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    patch = (np.abs(i1 - n1 / 2 + 0.5) < 3) & (np.abs(i3 - n3 / 2 + 0.5) < 3)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    fl = FaultLaw(np.full((n3, n1), 0.677), 0.525, Dc, tau0, 120e6)
    return me, dt, fl, steps


def _run(Dc, u0=None, n_cut=31):
    me, dt, fl, steps = _setup(Dc)
    o = HybridOracle(me, CS, CP, RHO, dt, n_cut=n_cut, fault=fl)
    if u0 is not None:
        o.u = u0.copy()
    xs, taus = forward_record(o, steps)
    return me, dt, fl, xs, taus


def _regimes(Dc, u0=None):
    """Slip (over-stressed) flags of every step, from a replay."""
    me, dt, fl, xs, _ = _run(Dc, u0)
    flags = []
    p, q = me.f + 1, me.f
    for (u, v, a) in xs:
        du = (u + dt * v + 0.5 * dt * dt * a)
        flags.append(np.hypot(du[p, 0] - du[q, 0], du[p, 2] - du[q, 2]))
    return np.array(flags)


def test_dc_gradient_matches_central_differences():
    Dc, eps = 0.05, 1e-7
    me, dt, fl, xs, taus = _run(Dc)
    rng = np.random.default_rng(3)
    tb = rng.normal(size=taus.shape)
    dDc, _ = dc_gradient(me, CS, CP, RHO, dt, 31, fl, xs, tb)
    assert np.abs(dDc).max() > 0
    Jp = np.sum(_run(Dc + eps)[4] * tb)
    Jm = np.sum(_run(Dc - eps)[4] * tb)
    fd = (Jp - Jm) / (2 * eps)
    an = dDc.sum()
    assert abs(fd - an) < 1e-6 * abs(an), (fd, an)


def test_initial_state_gradient_matches_central_differences():
    Dc = 0.05
    me, dt, fl, xs, taus = _run(Dc)
    rng = np.random.default_rng(4)
    tb = rng.normal(size=taus.shape)
    _, (lu, lv, la) = dc_gradient(me, CS, CP, RHO, dt, 31, fl, xs, tb)
    d = rng.normal(size=xs[0][0].shape) * 1e-6
    d[me.f + 1] = d[me.f]          # keep the fault closed at t = 0
    eps = 1.0
    Jp = np.sum(_run(Dc, u0=eps * d)[4] * tb)
    Jm = np.sum(_run(Dc, u0=-eps * d)[4] * tb)
    fd = (Jp - Jm) / (2 * eps)
    an = np.sum(lu * d)
    assert abs(fd - an) < 1e-4 * abs(an), (fd, an)
