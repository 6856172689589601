"""GPU adjoint of the SBIM traction update against the oracle's literal
transpose, the dot-product identity on the GPU, and autograd against central
finite differences (through the C ABI: sbim_step_adjoint)."""
import numpy as np
import pytest

from oracle.sbim_oracle import adjoint_sequence
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


def _params(n1, n3, n_cut, side, precision, dx=100.0):
    return dict(n1=n1, n3=n3, L1=n1 * dx, L3=n3 * dx, cs=CS, cp=CP, rho=RHO, dt=0.3 * dx / CP,
                n_cut=n_cut, side=side, precision=precision, kahan=True)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-9)])
@pytest.mark.parametrize("n1,n3,n_cut,steps,side,variant", [(8, 8, 5, 12, 1, 1), (16, 12, 24, 20, -1, 1),
                                                            (8, 8, 5, 12, -1, 0), (4, 4, 1, 5, 1, 1)])
def test_adjoint_matches_oracle_transpose(precision, tol, n1, n3, n_cut, steps, side, variant):
    from paper_2102_08756_gb300.sbim import SBIM
    p = _params(n1, n3, n_cut, side, precision)
    rng = np.random.default_rng(n1 * 7 + n_cut)
    tb = rng.normal(size=(steps, 3, n3, n1))
    ub_ref, vb_ref = adjoint_sequence(p["n1"], p["n3"], p["L1"], p["L3"], CS, CP, RHO, p["dt"],
                                      n_cut, side, tb)
    dt_ = torch.float64 if precision == "fp64" else torch.float32
    tbd = torch.from_numpy(tb).to("cuda", dt_)
    h = SBIM(**p)
    h.set_conv_config(variant)
    ub = torch.empty_like(tbd)
    vb = torch.empty_like(tbd)
    for m in range(steps - 1, -1, -1):
        h.step_adjoint(tbd[m], ub[m], vb[m])
    h.check()
    h.close()
    ub, vb = assert_finite(ub, "u_bar"), assert_finite(vb, "v_bar")
    for m in range(steps):
        for c in range(3):
            e = np.linalg.norm(ub[m, c] - ub_ref[m, c]) / np.linalg.norm(ub_ref[m, c])
            assert e < tol, (m, c, e)
    np.testing.assert_allclose(vb, vb_ref, rtol=1e-6 if precision == "fp32" else 1e-13)


def test_gpu_dot_product_identity_fp64():
    from paper_2102_08756_gb300.sbim import SBIM
    n1 = n3 = 16
    steps, n_cut, side = 30, 20, -1
    p = _params(n1, n3, n_cut, side, "fp64")
    g = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn((steps, 3, n3, n1), device="cuda", dtype=torch.float64, generator=g) * 1e-3
    v = torch.randn_like(u)
    tb = torch.randn_like(u)
    fwd = SBIM(**p)
    tau = torch.stack([fwd.step(u[n], v[n]) for n in range(steps)])
    adj = SBIM(**p)
    ub = torch.empty_like(u)
    vb = torch.empty_like(u)
    for m in range(steps - 1, -1, -1):
        adj.step_adjoint(tb[m], ub[m], vb[m])
    lhs = float((tau * tb).sum())
    rhs = float((u * ub).sum() + (v * vb).sum())
    assert abs(lhs - rhs) <= 1e-10 * float((tau * tb).abs().sum())
    fwd.close()
    adj.close()


def test_autograd_against_central_differences():
    """J = 1/2 sum_n |tau_n - tau*_n|^2 over 40 steps of a 16 x 16 boundary with
    truncation after 24 lags, FP64 handles: dJ/du . d and dJ/dv . d from
    autograd against central differences."""
    from paper_2102_08756_gb300.autograd import sbim_sequence
    n1 = n3 = 16
    steps, n_cut, side = 40, 24, 1
    p = _params(n1, n3, n_cut, side, "fp64")
    g = torch.Generator(device="cuda").manual_seed(11)
    u = (torch.randn((steps, 3, n3, n1), device="cuda", dtype=torch.float64, generator=g) * 1e-3)
    v = torch.randn_like(u) * 1e-1
    target = torch.randn_like(u) * 1e6
    du = torch.randn_like(u) * 1e-3
    dv = torch.randn_like(u) * 1e-1

    def J(uu, vv):
        return 0.5 * ((sbim_sequence(uu, vv, **p) - target) ** 2).sum()

    uu = u.clone().requires_grad_(True)
    vv = v.clone().requires_grad_(True)
    Jv = J(uu, vv)
    gu, gv = torch.autograd.grad(Jv, (uu, vv))
    eps = 1e-2
    with torch.no_grad():
        fd = (J(u + eps * du, v + eps * dv) - J(u - eps * du, v - eps * dv)) / (2 * eps)
    an = float((gu * du).sum() + (gv * dv).sum())
    assert abs(float(fd) - an) < 1e-8 * abs(an), (float(fd), an)


def test_dot_product_identity_at_the_gradient_configuration():
    """The gradient configuration's full size: 256 x 256 boundary, 1024-lag
    cutoff, 500 steps, FP32 history with Kahan sums and the default launch.
    sum_n <tau_n, tau_bar_n> = sum_m <u_m, u_bar_m> + <v_m, v_bar_m> (far field
    excluded) holds at any size; float rounding bounds the gap."""
    from paper_2102_08756_gb300.sbim import SBIM
    n, steps = 256, 500
    p = _params(n, n, 1024, 1, "fp32")
    g = torch.Generator(device="cuda").manual_seed(11)
    u = torch.randn((steps, 3, n, n), device="cuda", generator=g) * 1e-3
    v = torch.randn((steps, 3, n, n), device="cuda", generator=g) * 1e-2
    tb = torch.randn((steps, 3, n, n), device="cuda", generator=g)
    fwd = SBIM(**p)
    lhs = 0.0
    for m in range(steps):
        lhs += float((fwd.step(u[m], v[m]).double() * tb[m].double()).sum())
    adj = SBIM(**p)
    ub = torch.empty_like(u[0])
    vb = torch.empty_like(u[0])
    rhs = 0.0
    for m in range(steps - 1, -1, -1):
        adj.step_adjoint(tb[m], ub, vb)
        rhs += float((u[m].double() * ub.double()).sum() + (v[m].double() * vb.double()).sum())
    fwd.check()
    adj.check()
    scale = abs(lhs) + abs(rhs)
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs)
