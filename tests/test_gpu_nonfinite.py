"""The opt-in input check (sbim_set_check_finite, SBIM_ERR_NONFINITE), through
the C ABI.  Non-finite values are written into host-made input fields only; a
refused call must leave the handle untouched, so that the steps that follow
are bit-identical to a handle that never saw the bad input."""
import numpy as np
import pytest

from paper_2102_08756_gb300.synth import separable_history
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


def _bad(x, where, value):
    y = x.copy()
    y.reshape(-1)[where] = value
    return y


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16x2"])
def test_nonfinite_input_is_refused_and_the_handle_continues(precision):
    from paper_2102_08756_gb300.sbim import SBIM, SBIMError
    n1, n3, n_cut, steps = 24, 16, 9, 16
    dt = 0.3 * 100.0 / CP
    ndt = np.float64 if precision == "fp64" else np.float32
    hist = separable_history(n1, n3, n1 * 100.0, n3 * 100.0, steps, dt, CS, seed=5, spectrum="k2")
    ref = SBIM(n1, n3, n1 * 100.0, n3 * 100.0, CS, CP, RHO, dt, n_cut, -1, precision, True)
    g = SBIM(n1, n3, n1 * 100.0, n3 * 100.0, CS, CP, RHO, dt, n_cut, -1, precision, True)
    g.set_check_finite(True)
    bad_values = [np.nan, np.inf, -np.inf]
    for m in range(steps):
        u, v = hist.u(m).astype(ndt), hist.v(m).astype(ndt)
        if m in (3, 7, 12):
            # refused device-buffer and host-buffer steps, each leaving the state alone
            k = (3, 7, 12).index(m)
            bu = _bad(u, 17 * m + 5, bad_values[k])
            bv = _bad(v, 3 * n1 * n3 - 1 - m, bad_values[(k + 1) % 3])
            for uu, vv in ((bu, v), (u, bv)):
                with pytest.raises(SBIMError) as e:
                    g.step(torch.from_numpy(uu).cuda(), torch.from_numpy(vv).cuda())
                assert e.value.code == -6 and "non-finite" in str(e.value)
                with pytest.raises(SBIMError) as e:
                    g.step_host(uu, vv)
                assert e.value.code == -6
            assert g.n == m
        a = ref.step(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
        b = g.step(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
        assert_finite(b, "tau after a refused step")
        np.testing.assert_array_equal(a, b)
        if m == 10:
            # a refused re-evaluation keeps the level it would have replaced
            with pytest.raises(SBIMError) as e:
                g.step_repeat(torch.from_numpy(_bad(u, 0, np.nan)).cuda(), torch.from_numpy(v).cuda())
            assert e.value.code == -6 and g.n == m + 1
    ref.check()
    g.check()
    ref.close()
    g.close()


def test_nonfinite_adjoint_input_is_refused():
    from paper_2102_08756_gb300.sbim import SBIM, SBIMError
    n, n_cut = 16, 6
    dt = 0.3 * 100.0 / CP
    rng = np.random.default_rng(1)
    tb = rng.normal(size=(8, 3, n, n)).astype(np.float32)
    ref = SBIM(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, 1, "fp32", True)
    g = SBIM(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, 1, "fp32", True)
    g.set_check_finite(True)
    for m in range(8):
        if m == 4:
            with pytest.raises(SBIMError) as e:
                g.step_adjoint(torch.from_numpy(_bad(tb[m], 11, np.inf)).cuda())
            assert e.value.code == -6 and g.n == 4
        ua, va = ref.step_adjoint(torch.from_numpy(tb[m]).cuda())
        ub, vb = g.step_adjoint(torch.from_numpy(tb[m]).cuda())
        assert torch.equal(ua, ub) and torch.equal(va, vb)
    ref.close()
    g.close()


def test_check_off_by_default_and_switchable():
    """With the check off (the default) a NaN input is not inspected: it flows
    into the output; switching the check on then refuses the same input."""
    from paper_2102_08756_gb300.sbim import SBIM, SBIMError
    n = 8
    g = SBIM(n, n, n * 100.0, n * 100.0, CS, CP, RHO, 0.005, 4, 1, "fp32", True)
    u = np.zeros((3, n, n), np.float32)
    u[1, 2, 3] = np.nan
    z = torch.zeros((3, n, n), device="cuda")
    t = g.step(torch.from_numpy(u).cuda(), z)
    torch.cuda.synchronize()
    assert not bool(torch.isfinite(t).all())
    g.reset()
    g.set_check_finite(True)
    with pytest.raises(SBIMError) as e:
        g.step(torch.from_numpy(u).cuda(), z)
    assert e.value.code == -6 and g.n == 0
    g.set_check_finite(False)
    g.close()
