"""Pins of the oracle's half-space kernels (Section 2.3, Eq. (SBI); the kernels
are derived because the paper defers them to its references).

Each test checks the oracle against something other than itself: a Bessel
function closed form, an independent numerical solution of Navier's equations,
an independent elastostatic solution, the initial-value theorem, or the
Laplace transform of the time-domain kernels computed by separate quadrature.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from tests._elastic import static_traction
from oracle.sbim_oracle import (KernelTable, kernels_direct, laplace_kernels,
                                laplace_symbols, real_axis_densities)

ETA = 6000.0 / 3464.0      # c_p / c_s of the paper's material (Section 3.1)


def test_h33_is_bessel_j1_over_t():
    """Antiplane kernel: the inverse transform of sqrt(1+p^2) - p is J1(T)/T."""
    special = pytest.importorskip("scipy.special")
    T = np.concatenate([[1e-6, 1e-3], np.linspace(0.1, 50, 137), [100.3, 777.7, 2999.9]])
    H = kernels_direct(T, ETA)
    np.testing.assert_allclose(H[2], special.j1(T) / T, rtol=0, atol=2e-14)


def _navier_traction(p, eta, D):
    """Independent solution of the upper half-space problem for one mode.

    Units q = mu = rho = c_s = 1 so s = p and lambda = eta^2 - 2.  Solutions
    V exp(-kappa x2) of Navier's equations make a 2x2 matrix singular; its
    determinant is a polynomial in kappa whose roots with Re kappa > 0 are
    found numerically, the null vectors combined to match D at x2 = 0, and the
    traction sigma_2j(0) formed from the stress-strain law.
    """
    lam = eta * eta - 2.0
    c = lam + 1.0
    P = np.polynomial.Polynomial
    kap = P([0, 1])
    m11 = kap ** 2 - 1 - c - p * p
    m12 = -1j * c * kap
    m22 = kap ** 2 * (1 + c) - 1 - p * p
    det = m11 * m22 - m12 * m12
    roots = det.roots()
    roots = roots[roots.real > 0]
    assert roots.size == 2
    vecs = []
    for k in roots:
        M = np.array([[m11(k), m12(k)], [m12(k), m22(k)]])
        _, _, vh = np.linalg.svd(M)
        vecs.append(vh[-1].conj())
    V = np.array(vecs).T                      # columns: (V_xi, V_2) per root
    coef = np.linalg.solve(V, D)
    du = -(V * roots[None, :]) @ coef         # d/dx2 at 0
    u0 = V @ coef
    s2xi = du[0] + 1j * u0[1]                 # mu (du_xi/dx2 + du_2/dxi)
    s22 = lam * (1j * u0[0] + du[1]) + 2.0 * du[1]
    kap_sh = np.sqrt(1 + p * p + 0j)
    kap_sh = kap_sh if kap_sh.real > 0 else -kap_sh
    return s2xi, s22, -kap_sh                 # antiplane: sigma = -kappa D_perp


@pytest.mark.parametrize("p", [0.37 + 0.0j, 1.3 + 0.8j, 0.2 - 2.5j, 4.0 + 9.0j])
def test_laplace_symbols_solve_navier(p):
    rng = np.random.default_rng(7)
    D = rng.normal(size=2) + 1j * rng.normal(size=2)
    s2xi, s22, s33 = _navier_traction(p, ETA, D)
    K11, K22, K33, G = laplace_symbols(p, ETA)
    np.testing.assert_allclose(s2xi, -K11 * D[0] + 1j * G * D[1], rtol=1e-9)
    np.testing.assert_allclose(s22, -1j * G * D[0] - K22 * D[1], rtol=1e-9)
    np.testing.assert_allclose(s33, -K33, rtol=1e-12)


def test_static_limit_matches_elastostatics():
    rng = np.random.default_rng(3)
    D = rng.normal(size=2) + 1j * rng.normal(size=2)
    s2xi, s22 = static_traction(ETA, D, +1)
    K11, K22, K33, G = laplace_symbols(1e-7 + 0j, ETA)
    np.testing.assert_allclose(s2xi, -K11 * D[0] + 1j * G * D[1], rtol=1e-9)
    np.testing.assert_allclose(s22, -1j * G * D[0] - K22 * D[1], rtol=1e-9)


def test_initial_values_from_initial_value_theorem():
    """H(0+) = lim p Hhat(p) (and H12'(0+) = lim p^2 Hhat12(p))."""
    H0 = kernels_direct([0.0], ETA)[:, 0]

    def lim(f):
        # p f(p) = L + c/p + O(1/p^2): one Richardson step removes c/p
        p1, p2 = 2000.0, 4000.0
        return 2.0 * f(p2) - f(p1)

    ivt = [lim(lambda p, k=k: np.real(p * laplace_kernels(p, ETA)[k])) for k in range(3)]
    np.testing.assert_allclose(H0[:3], ivt, rtol=1e-6)
    assert abs(H0[3]) < 1e-15
    eps = 1e-5
    slope = kernels_direct([eps], ETA)[3, 0] / eps
    np.testing.assert_allclose(slope, lim(lambda p: np.real(p * p * laplace_kernels(p, ETA)[3])), rtol=1e-5)
    # and the closed forms of those limits
    np.testing.assert_allclose(H0[:3], [(2 * ETA - 1) / 2, ETA ** 2 * (2 - ETA) / 2, 0.5], rtol=1e-13)
    np.testing.assert_allclose(slope, ETA * (ETA - 1) ** 2 / 2, rtol=1e-7)


@pytest.mark.parametrize("p", [0.3, 1.0, 3.0])
def test_laplace_transform_of_time_kernels(p):
    """int_0^inf H(T) exp(-p T) dT, by separate composite quadrature over the
    memoised kernels, equals the Laplace-domain kernels."""
    x, w = leggauss(60)
    edges = np.linspace(0.0, 80.0 / p, 161)
    a, b = edges[:-1, None], edges[1:, None]
    T = ((a + b) / 2 + (b - a) / 2 * x[None, :]).ravel()
    W = ((b - a) / 2 * w[None, :]).ravel()
    kt = KernelTable(ETA, T.max() + 1)
    num = kt(T) @ (W * np.exp(-p * T))
    ref = np.real(np.array(laplace_kernels(p, ETA)))
    np.testing.assert_allclose(num, ref, rtol=1e-10, atol=1e-13)


def test_static_integrals():
    """int_0^inf H = Hhat(0): 2 eta^2/(1+eta^2) for H11, H22; 1 for H33;
    2/(1+eta^2) - (2 - eta) for H12 (by the p -> 0 limit of the symbols)."""
    small = 1e-8
    ref = np.real(np.array(laplace_kernels(small, ETA)))
    np.testing.assert_allclose(ref, [2 * ETA ** 2 / (1 + ETA ** 2)] * 2 + [1.0, 2 / (1 + ETA ** 2) - (2 - ETA)],
                               rtol=1e-6)
    # the time integral up to T = 600 approaches the same values
    T = np.linspace(0, 600, 600 * 64 + 1)
    kt = KernelTable(ETA, 601)
    H = kt(T)
    h = T[1] - T[0]
    integ = h * (H.sum(axis=1) - 0.5 * (H[:, 0] + H[:, -1]))
    np.testing.assert_allclose(integ, ref, atol=2e-3)


def test_densities_are_boundary_values_of_transforms():
    y = np.array([0.05, 0.3, 0.77, 0.999, 1.001, 1.2, 1.5, 1.73, 1.9, 3.0])
    R11, R22, R33, X12 = real_axis_densities(y, ETA)
    Hh = laplace_kernels(1e-12 + 1j * y, ETA)
    np.testing.assert_allclose(R11, Hh[0].real, atol=1e-8)
    np.testing.assert_allclose(R22, Hh[1].real, atol=1e-8)
    np.testing.assert_allclose(R33, Hh[2].real, atol=1e-8)
    np.testing.assert_allclose(X12, -Hh[3].imag, atol=1e-8)


def test_quadrature_matches_plain_density_integral():
    """The mapped Gauss-Legendre quadrature equals a brute midpoint sum of the
    unmapped densities (coarse tolerance: the densities have square-root ends)."""
    y = (np.arange(2_000_000) + 0.5) * (ETA / 2_000_000)
    dy = ETA / 2_000_000
    R11, R22, R33, X12 = real_axis_densities(y, ETA)
    for T in (0.0, 2.5, 11.0):
        c, s = np.cos(y * T), np.sin(y * T)
        brute = 2 / np.pi * dy * np.array([R11 @ c, R22 @ c, R33 @ c, X12 @ s])
        np.testing.assert_allclose(kernels_direct([T], ETA)[:, 0], brute, atol=2e-6)


def test_table_matches_direct():
    rng = np.random.default_rng(11)
    T = np.concatenate([rng.uniform(0, 3200, 400), rng.uniform(0, 1, 50), [0.0]])
    kt = KernelTable(ETA, 3201)
    np.testing.assert_allclose(kt(T), kernels_direct(T, ETA), rtol=0, atol=5e-15)
