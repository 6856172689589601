"""GPU gradient of a fault-traction functional with respect to Dc through the
coupled run (checkpointed reverse sweep, through the C ABI), against the FP64
oracle's literal transpose and central finite differences."""
import numpy as np
import pytest

from oracle.fem_oracle import FaultLaw, HybridOracle, SlabMesh, dc_gradient, forward_record
from tests._errors import assert_finite

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _case(n1=16, n2=4, n3=16):
    i3, i1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    patch = (np.abs(i1 - n1 / 2 + 0.5) < 3) & (np.abs(i3 - n3 / 2 + 0.5) < 3)
    tau0 = np.where(patch, 1.005 * 0.677 * 120e6, 70e6)
    return dict(n1=n1, n2=n2, n3=n3, h=100.0, cs=CS, cp=CP, rho=RHO, dt=0.3 * 100.0 / CP,
                n_cut=31, mu_s=np.full((n3, n1), 0.677), tau0=tau0, mu_k=0.525, sigma0=120e6)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_dc_gradient_matches_oracle(precision, tol):
    from paper_2102_08756_gb300.autograd import hybrid_rupture
    c = _case()
    steps, Dc = 30, 0.05
    me = SlabMesh(c["n1"], c["n2"], c["n3"], c["h"], fault=True)
    fl = FaultLaw(c["mu_s"], c["mu_k"], Dc, c["tau0"], c["sigma0"])
    o = HybridOracle(me, CS, CP, RHO, c["dt"], n_cut=c["n_cut"], fault=fl)
    xs, taus = forward_record(o, steps)
    rng = np.random.default_rng(3)
    tb = rng.normal(size=taus.shape)
    ref, _ = dc_gradient(me, CS, CP, RHO, c["dt"], c["n_cut"], fl, xs, tb)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    dc = torch.tensor(Dc, dtype=torch.float64, requires_grad=True)
    out = hybrid_rupture(dc, steps=steps, every=7, precision=precision, **c)
    assert out.dtype == dtype
    J = (out.double() * torch.from_numpy(tb).to(out.device)).sum()
    (g,) = torch.autograd.grad(J, dc)
    assert_finite(out, "boundary tractions")
    assert_finite(g, "dJ/dDc")
    print(f"\nGRADIENT-REPORT {precision}: dJ/dDc {float(g):.6e} oracle {ref.sum():.6e} "
          f"relative error {abs(float(g) - ref.sum()) / abs(ref.sum()):.3e}; traction error "
          f"{np.abs(out.detach().double().cpu().numpy() - taus).max() / np.abs(taus).max():.3e} "
          f"of the peak")
    np.testing.assert_allclose(out.detach().double().cpu().numpy(), taus, rtol=0,
                               atol=(1e-10 if precision == "fp64" else 1e-4) * np.abs(taus).max())
    assert abs(float(g) - ref.sum()) < tol * abs(ref.sum()), (float(g), ref.sum())


def test_dc_gradient_central_differences_fp64():
    from paper_2102_08756_gb300.autograd import hybrid_rupture
    c = _case()
    steps, Dc, eps = 30, 0.05, 1e-7
    rng = np.random.default_rng(5)
    tb = torch.from_numpy(rng.normal(size=(steps, 3, c["n3"], c["n1"]))).cuda()
    dc = torch.tensor(Dc, dtype=torch.float64, requires_grad=True)
    J = (hybrid_rupture(dc, steps=steps, every=10, precision="fp64", **c) * tb).sum()
    (g,) = torch.autograd.grad(J, dc)
    with torch.no_grad():
        Jp = (hybrid_rupture(torch.tensor(Dc + eps, dtype=torch.float64), steps=steps, every=10,
                             precision="fp64", **c) * tb).sum()
        Jm = (hybrid_rupture(torch.tensor(Dc - eps, dtype=torch.float64), steps=steps, every=10,
                             precision="fp64", **c) * tb).sum()
    fd = float(Jp - Jm) / (2 * eps)
    assert abs(fd - float(g)) < 1e-5 * abs(fd), (fd, float(g))
