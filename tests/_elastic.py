"""Independent elastostatic half-space solution for one Fourier mode, used as a
pin of the oracle (shared by the kernel and the step tests)."""
import numpy as np


def static_traction(eta, D, sigma):
    """Traction sigma_2j at the boundary of an elastostatic half-space with
    boundary displacement D = (D_xi, D_2) e^{i xi}, in units q = mu = 1.

    Ansatz u_j = (a_j + b_j x2) exp(-sigma x2), sigma = +1 for the half-space
    x2 > 0 and -1 for x2 < 0; the b_j are solved from Navier's static
    equations mu lap u + (lambda + mu) grad div u = 0 at two depths.
    """
    lam = eta * eta - 2.0
    c = lam + 1.0
    D = np.asarray(D, dtype=complex)

    def fields(b, y):
        e = np.exp(-sigma * y)
        f = (D + b * y) * e
        f1 = (b - sigma * (D + b * y)) * e
        f2 = (-2 * sigma * b + (D + b * y)) * e
        return f, f1, f2

    def residual(b):
        out = []
        for y in (0.0, 0.7 * sigma):
            f, f1, f2 = fields(b, y)
            div = 1j * f[0] + f1[1]
            ddiv = 1j * f1[0] + f2[1]
            out += [f2[0] - f[0] + c * 1j * div, f2[1] - f[1] + c * ddiv]
        return np.array(out)

    r0 = residual(np.zeros(2, complex))
    A = np.stack([residual(np.eye(2)[k].astype(complex)) - r0 for k in range(2)], axis=1)
    b = np.linalg.lstsq(A, -r0, rcond=None)[0]
    assert np.max(np.abs(residual(b))) < 1e-12
    f, f1, _ = fields(b, 0.0)
    s2xi = f1[0] + 1j * f[1]
    s22 = lam * (1j * f[0] + f1[1]) + 2 * f1[1]
    return s2xi, s22
