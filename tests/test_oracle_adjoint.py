"""Pins of the oracle's adjoint of a sequence of traction updates: the
dot-product identity against the oracle's forward stepper (which uses the
convolve-then-assemble form, not the explicit matrices of the adjoint), the
transposes of the DFT stages, and a central finite difference of a quadratic
misfit."""
import numpy as np
import pytest

from oracle.sbim_oracle import (SBIMOracle, adjoint_sequence, dft2_forward,
                                dft2_forward_transpose, dft2_inverse,
                                dft2_inverse_transpose)

CS, CP, RHO = 3464.0, 6000.0, 2670.0


def test_dft_stage_transposes():
    rng = np.random.default_rng(0)
    n3, n1 = 6, 8
    u = rng.normal(size=(3, n3, n1))
    Ub = rng.normal(size=(3, n3, n1 // 2 + 1)) + 1j * rng.normal(size=(3, n3, n1 // 2 + 1))
    lhs = np.sum((np.conj(dft2_forward(u)) * Ub).real)
    rhs = np.sum(u * dft2_forward_transpose(Ub, n1))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # inverse stage: only Hermitian-consistent half spectra are in its domain
    F = dft2_forward(rng.normal(size=(3, n3, n1)))
    g = rng.normal(size=(3, n3, n1))
    lhs = np.sum(dft2_inverse(F, n1)[0] * g)
    rhs = np.sum((np.conj(F) * dft2_inverse_transpose(g)).real)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("n1,n3,n_cut,steps,side", [(8, 8, 5, 12, 1), (8, 6, 16, 10, -1),
                                                     (4, 4, 1, 6, 1)])
def test_dot_product_identity(n1, n3, n_cut, steps, side):
    rng = np.random.default_rng(n1 + n_cut)
    dx = 100.0
    L1, L3 = n1 * dx, n3 * dx
    dt = 0.3 * dx / CP
    u = rng.normal(size=(steps, 3, n3, n1)) * 1e-3
    v = rng.normal(size=(steps, 3, n3, n1))
    tb = rng.normal(size=(steps, 3, n3, n1))
    o = SBIMOracle(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side)
    tau = np.stack([o.step(u[k], v[k])["tau"] for k in range(steps)])
    ub, vb = adjoint_sequence(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side, tb)
    lhs = np.sum(tau * tb)
    rhs = np.sum(u * ub) + np.sum(v * vb)
    assert abs(lhs - rhs) < 1e-12 * (np.abs(tau * tb).sum()), (lhs, rhs)


def test_finite_difference_of_quadratic_misfit():
    """J = 1/2 sum_n |tau_n - tau*_n|^2; dJ/du_m . d by central differences."""
    rng = np.random.default_rng(5)
    n1 = n3 = 8
    dx, steps, n_cut, side = 100.0, 8, 6, -1
    dt = 0.3 * dx / CP
    u = rng.normal(size=(steps, 3, n3, n1)) * 1e-3
    v = rng.normal(size=(steps, 3, n3, n1))
    target = rng.normal(size=(steps, 3, n3, n1)) * 1e6

    def run(uu):
        o = SBIMOracle(n1, n3, n1 * dx, n3 * dx, CS, CP, RHO, dt, n_cut, side)
        return np.stack([o.step(uu[k], v[k])["tau"] for k in range(steps)])

    tau = run(u)
    ub, _ = adjoint_sequence(n1, n3, n1 * dx, n3 * dx, CS, CP, RHO, dt, n_cut, side, tau - target)
    d = rng.normal(size=u.shape) * 1e-3
    eps = 1e-3
    J = lambda t: 0.5 * np.sum((t - target) ** 2)  # noqa: E731
    fd = (J(run(u + eps * d)) - J(run(u - eps * d))) / (2 * eps)
    an = np.sum(ub * d)
    assert abs(fd - an) < 1e-7 * abs(an), (fd, an)
