"""FP64 CPU oracle of the spectral-boundary-integral (SBIM) traction update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library behind ``include/sbim.h`` and its Python
binding) never imports, links or executes anything under ``oracle/``, and this
module imports nothing from the product package.

What is computed (Albertini, Elbanna & Kammer, arXiv:2102.08756, Section 2.3,
Eq. (SBI)):

    tau_i(x1, x3, t) = tau_i^inf - eta_ij (mu / c_s) du_j/dt + s_i(x1, x3, t)

where the non-local term s_i is evaluated spectrally: a 2D Fourier transform of
the boundary displacement in (x1, x3) and, for every Fourier mode, a time
convolution of that mode's displacement history with the elastodynamic
half-space kernels of the "independent formulation" (one half-space at a
time).  The paper defers the kernels to its references; they are derived here
from half-space elastodynamics (Laplace transform in time, Helmholtz
potentials), and every piece of that derivation is pinned by tests against
closed forms and an independent elastostatic solution.

Readings of the paper used here (the paper is silent or inconsistent):
  * eta_22 = c_p / c_s (the P-wave impedance; Eq. (SBI) prints c_s / c_p).
  * Upper half-space (side +1, material at x2 > 0): radiation term -(mu/c_s);
    lower half-space (side -1): the diagonal terms and the radiation term flip
    sign, the in-plane coupling terms do not.
  * The convolution is the trapezoid rule in T = q c_s t with the current step
    included, D[j] = 0 before the first step (equilibrium start, Section 2.1),
    and a hard cutoff after ``n_cut`` lags.
  * On the Nyquist lines (j1 = N1/2 or j3 = N3/2) the modal operator keeps only
    its part that is even in the aliased wavenumber component; |k| keeps pi/dx.
  * Mode k = 0 has s = 0.
  * Forward DFT unnormalised, inverse DFT scaled by 1/(N1 N3).

Everything is float64 / complex128.  Parity unpinned: none -- every function
here is pinned by a test in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from numpy.polynomial.legendre import leggauss

__all__ = [
    "Material", "laplace_symbols", "laplace_kernels", "real_axis_densities",
    "kernels_direct", "KernelTable", "trapezoid_weights", "dft2_forward",
    "dft2_inverse", "ModeSet", "apply_modal_operator", "SBIMOracle",
]


# ---------------------------------------------------------------------------
# Material constants (Section 2.1 Eq. (linelasticity), Section 2.3 Eq. (SBI))
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Material:
    """Isotropic elastic half-space: shear modulus mu = rho c_s^2 and the wave
    speed ratio eta = c_p / c_s (Section 2.3, the eta_ij of Eq. (SBI))."""

    cs: float
    cp: float
    rho: float

    @property
    def mu(self) -> float:
        return self.rho * self.cs * self.cs

    @property
    def eta(self) -> float:
        return self.cp / self.cs

    @property
    def impedance(self) -> np.ndarray:
        """Diagonal of eta_ij in Eq. (SBI) read as (1, c_p/c_s, 1)."""
        return np.array([1.0, self.eta, 1.0])


# ---------------------------------------------------------------------------
# Laplace-domain response of one half-space to one Fourier mode (Section 2.3;
# kernels derived here because the paper defers them to its references).
#
# Upper half-space x2 > 0, boundary displacement D e^{i q xi + s t}, with
# p = s / (q c_s).  Decaying P and S potentials exp(-q a x2), exp(-q b x2) with
# a = sqrt(1 + p^2/eta^2), b = sqrt(1 + p^2) (branches with Re >= 0) give
#   sigma_2xi  = -mu q K11 D_xi + i mu q G D_2
#   sigma_22   = -i mu q G D_xi - mu q K22 D_2
#   sigma_2perp = -mu q K33 D_perp
# ---------------------------------------------------------------------------
def laplace_symbols(p, eta):
    """K11, K22, K33, G of the upper half-space at complex p (Re p > 0)."""
    p = np.asarray(p, dtype=complex)
    a = np.sqrt(p - 1j * eta) * np.sqrt(p + 1j * eta) / eta
    b = np.sqrt(p - 1j) * np.sqrt(p + 1j)
    ab = a * b
    # K11 = a p^2 / (ab - 1), K22 = b p^2 / (ab - 1) and
    # G = (2 + p^2 - 2ab) / (1 - ab), each multiplied through by (1 + ab):
    # a^2 b^2 - 1 = p^2 (1 + 1/eta^2 + p^2/eta^2) and
    # (2 + p^2)^2 - 4 a^2 b^2 = p^2 (p^2 (1 - 4/eta^2) - 4/eta^2),
    # which removes the 0/0 at small p.
    den = 1.0 + 1.0 / eta ** 2 + p * p / eta ** 2
    K11 = a * (1.0 + ab) / den
    K22 = b * (1.0 + ab) / den
    K33 = b
    G = ((1.0 + ab) * (4.0 / eta ** 2 + p * p * (4.0 / eta ** 2 - 1.0))
         / (den * (2.0 + p * p + 2.0 * ab)))
    return K11, K22, K33, G


def laplace_kernels(p, eta):
    """Laplace transforms of the convolution kernels H11, H22, H33, H12.

    The parts of K that are instantaneous in time are removed: p (shear
    radiation damping), eta p (P-wave radiation damping, so eta_22 = c_p/c_s)
    and the constant in-plane coupling 2 - eta.
    """
    K11, K22, K33, G = laplace_symbols(p, eta)
    p = np.asarray(p, dtype=complex)
    return K11 - p, K22 - eta * p, K33 - p, G - (2.0 - eta)


def real_axis_densities(y, eta):
    """Boundary values on p = i y of the kernel transforms.

    Returns (R11, R22, R33, X12) with R = Re Hhat(i y) for the diagonal
    kernels and X12 = -Im Hhat12(i y).  All vanish for y > eta.
    """
    y = np.asarray(y, dtype=float)
    R11 = np.zeros_like(y)
    R22 = np.zeros_like(y)
    R33 = np.zeros_like(y)
    X12 = np.zeros_like(y)
    lo = (y >= 0) & (y <= 1.0)
    hi = (y > 1.0) & (y <= eta)
    yl = y[lo]
    a = np.sqrt(1.0 - (yl / eta) ** 2)
    b = np.sqrt(1.0 - yl * yl)
    D = 1.0 + (1.0 - yl * yl) / eta ** 2
    R11[lo] = a * (1.0 + a * b) / D
    R22[lo] = b * (1.0 + a * b) / D
    R33[lo] = b
    yh = y[hi]
    A = np.sqrt(1.0 - (yh / eta) ** 2)
    B = np.sqrt(yh * yh - 1.0)
    den = 1.0 + (A * B) ** 2
    R11[hi] = A * yh * yh / den
    R22[hi] = -A * B * B * yh * yh / den
    X12[hi] = A * B * yh * yh / den
    return R11, R22, R33, X12


# ---------------------------------------------------------------------------
# Time-domain kernels by real-axis inversion of the causal transforms:
#   H_jj(T) = (2/pi) int_0^eta R_jj(y) cos(y T) dy
#   H_12(T) = (2/pi) int_1^eta X_12(y) sin(y T) dy
# Both y-intervals are mapped so that the square-root end points become
# smooth (y = sin(theta) on [0, 1]; y = 1 + (eta-1) sin^2(phi) on [1, eta]),
# then integrated by composite 16-point Gauss-Legendre panels whose phase
# change y*T stays below 8 rad per panel.
# ---------------------------------------------------------------------------
_GL_X, _GL_W = leggauss(16)


def _panels(npan):
    edges = np.linspace(0.0, 0.5 * np.pi, npan + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    half = 0.5 * (edges[1:] - edges[:-1])
    x = (mid[:, None] + half[:, None] * _GL_X[None, :]).ravel()
    w = (half[:, None] * _GL_W[None, :]).ravel()
    return x, w


def _lower_segment(theta, eta):
    """y = sin(theta): integrands of H11, H22, H33 times dy/dtheta."""
    y = np.sin(theta)
    b = np.cos(theta)
    a = np.sqrt(1.0 - (y / eta) ** 2)
    D = 1.0 + (1.0 - y * y) / eta ** 2
    jac = b
    return y, a * (1 + a * b) / D * jac, b * (1 + a * b) / D * jac, b * jac


def _upper_segment(phi, eta):
    """y = 1 + (eta-1) sin^2(phi): integrands of H11, H22, H12 times dy/dphi."""
    s, c = np.sin(phi), np.cos(phi)
    y = 1.0 + (eta - 1.0) * s * s
    B = math.sqrt(eta - 1.0) * s * np.sqrt(y + 1.0)
    A = math.sqrt(eta - 1.0) * c * np.sqrt(eta + y) / eta
    jac = 2.0 * (eta - 1.0) * s * c
    den = 1.0 + (A * B) ** 2
    return (y, A * y * y / den * jac, -A * B * B * y * y / den * jac,
            A * B * y * y / den * jac)


def kernels_direct(T, eta):
    """H11, H22, H33, H12 at T >= 0 by quadrature; returns shape (4, len(T))."""
    T = np.atleast_1d(np.asarray(T, dtype=float))
    if np.any(T < 0):
        raise ValueError("kernels_direct takes T >= 0")
    out = np.empty((4, T.size))
    need = np.ceil(T * (0.5 * np.pi) / 8.0).astype(np.int64) + 2
    key = np.ceil(np.log2(np.maximum(need, 4))).astype(np.int64)
    for k in np.unique(key):
        idx = np.nonzero(key == k)[0]
        x, w = _panels(int(2 ** k))
        yl, r11l, r22l, r33l = _lower_segment(x, eta)
        yu, r11u, r22u, x12u = _upper_segment(x, eta)
        chunk = max(1, 4_000_000 // x.size)
        for s0 in range(0, idx.size, chunk):
            sel = idx[s0:s0 + chunk]
            Tc = T[sel][:, None]
            cl = np.cos(Tc * yl[None, :]) * w[None, :]
            cu = np.cos(Tc * yu[None, :]) * w[None, :]
            su = np.sin(Tc * yu[None, :]) * w[None, :]
            out[0, sel] = cl @ r11l + cu @ r11u
            out[1, sel] = cl @ r22l + cu @ r22u
            out[2, sel] = cl @ r33l
            out[3, sel] = su @ x12u
    return out * (2.0 / np.pi)


class KernelTable:
    """Memoised kernels: ``kernels_direct`` on the grid T_j = j h (h = 1/16),
    evaluated elsewhere by 12-point Lagrange interpolation.

    The kernels are entire functions of T (compactly supported spectra on
    [0, eta]); with h = 1/16 the interpolation error is below 1e-15 for
    eta < 2 (pinned against ``kernels_direct``).  Nodes at negative T use the
    even extension of H11, H22, H33 and the odd extension of H12, which the
    cosine/sine representations make exact.
    """

    NPTS = 12

    def __init__(self, eta, t_max, h=1.0 / 16.0):
        self.eta = float(eta)
        self.h = float(h)
        half = self.NPTS // 2
        self.j0 = -(half - 1)
        j_hi = int(math.ceil(t_max / h)) + half + 1
        jj = np.arange(self.j0, j_hi + 1)
        vals = kernels_direct(np.abs(jj) * h, eta)
        vals[3] *= np.sign(jj)
        self.vals = vals
        self.t_max = (j_hi - half) * h
        offs = np.arange(-(half - 1), half + 1, dtype=float)
        self._offs = offs
        self._den = np.array([np.prod([o - p for p in offs if p != o])
                              for o in offs])

    def __call__(self, T):
        T = np.atleast_1d(np.asarray(T, dtype=float))
        if T.size and (T.min() < 0 or T.max() > self.t_max):
            raise ValueError("T outside the kernel table")
        out = np.empty((4, T.size))
        chunk = 1 << 20
        for s0 in range(0, T.size, chunk):
            Tc = T[s0:s0 + chunk]
            u = Tc / self.h
            i = np.floor(u).astype(np.int64)
            t = u - i
            diff = t[:, None] - self._offs[None, :]
            basis = np.empty_like(diff)
            for k in range(self.NPTS):
                others = np.delete(diff, k, axis=1)
                basis[:, k] = np.prod(others, axis=1) / self._den[k]
            cols = (i[:, None] + self._offs[None, :].astype(np.int64)) - self.j0
            for r in range(4):
                out[r, s0:s0 + chunk] = np.sum(basis * self.vals[r][cols], axis=1)
        return out


def trapezoid_weights(dT, n_lags, kernel):
    """Convolution weights w_ab(m), m = 0..n_lags-1, for one mode spacing dT.

    Trapezoid rule in T = q c_s t of int_0^t H(q c_s t') D(t - t') q c_s dt'
    (reading of Section 2.3; the paper does not state the quadrature):
    w(0) = H(0) dT / 2 and w(m) = H(m dT) dT.  Returns shape (4, n_lags) in
    the order (11, 22, 33, 12).
    """
    m = np.arange(n_lags, dtype=float)
    w = kernel(m * dT) * dT
    w[:, 0] *= 0.5
    return w


# ---------------------------------------------------------------------------
# Direct 2D DFT on the periodic boundary plane (Section 2.3 "Fourier transform
# in space"): forward unnormalised over x1 (fastest) and x3, inverse scaled by
# 1/(N1 N3).  Fields are [3][N3][N1]; half spectra are [3][N3][N1/2+1].
# ---------------------------------------------------------------------------
def _dft_matrix(n_out, n_in, sign):
    j = np.arange(n_out)[:, None]
    x = np.arange(n_in)[None, :]
    return np.exp(sign * 2j * np.pi * ((j * x) % n_in) / n_in)


def dft2_forward(u):
    u = np.asarray(u, dtype=float)
    _, n3, n1 = u.shape
    E3 = _dft_matrix(n3, n3, -1.0)            # [r3][x3]
    E1 = _dft_matrix(n1 // 2 + 1, n1, -1.0)   # [j1][x1]
    return np.stack([E3 @ u[c] @ E1.T for c in range(u.shape[0])])


def dft2_inverse(F, n1):
    """Real field from a half spectrum, via the explicit Hermitian extension
    F(-j1, -j3) = conj F(j1, j3) and a full complex inverse DFT.  Returns the
    real part and the largest imaginary part (zero for a consistent half
    spectrum)."""
    F = np.asarray(F, dtype=complex)
    nc, n3, nh = F.shape
    full = np.zeros((nc, n3, n1), dtype=complex)
    full[:, :, :nh] = F
    neg_r3 = (-np.arange(n3)) % n3
    for j1 in range(1, n1 - nh + 1):
        full[:, :, n1 - j1] = np.conj(F[:, neg_r3, j1])
    E3 = _dft_matrix(n3, n3, +1.0)
    E1 = _dft_matrix(n1, n1, +1.0)
    out = np.stack([E3 @ full[c] @ E1.T for c in range(nc)]) / (n1 * n3)
    return out.real, float(np.max(np.abs(out.imag), initial=0.0))


# ---------------------------------------------------------------------------
# The per-mode operator (Section 2.3): Cartesian form of the half-space
# response, Fourier mode by Fourier mode.
# ---------------------------------------------------------------------------
@dataclass
class ModeSet:
    """A set of half-spectrum bins (r3, j1) with their wavevectors."""

    r3: np.ndarray
    j1: np.ndarray
    k1: np.ndarray
    k3: np.ndarray
    q: np.ndarray
    nyq1: np.ndarray
    nyq3: np.ndarray

    @classmethod
    def build(cls, n1, n3, L1, L3, r3=None, j1=None):
        if r3 is None:
            r3, j1 = np.meshgrid(np.arange(n3), np.arange(n1 // 2 + 1), indexing="ij")
            r3, j1 = r3.ravel(), j1.ravel()
        r3 = np.asarray(r3, dtype=np.int64)
        j1 = np.asarray(j1, dtype=np.int64)
        j3 = np.where(r3 <= n3 // 2, r3, r3 - n3)
        k1 = 2.0 * np.pi * j1 / L1
        k3 = 2.0 * np.pi * j3 / L3
        return cls(r3, j1, k1, k3, np.hypot(k1, k3), j1 == n1 // 2, r3 == n3 // 2)

    def __len__(self):
        return self.r3.size


def apply_modal_operator(modes, mat, side, weights, hist_rev, current):
    """Non-local spectral traction F = FT(s) for each mode in ``modes``.

    weights  : (4, nmodes, L) convolution weights (11, 22, 33, 12)
    hist_rev : (L, 3, nmodes) Cartesian displacement spectra, lag-major,
               hist_rev[m] = Uhat at step n - m
    current  : (3, nmodes) Uhat at step n (the instantaneous coupling)

    With e = k/q the in-plane direction and e_perp = (-e3, e1):
      F_h = -side mu q [e e^T (H11*U_h) + e_perp e_perp^T (H33*U_h)]
            + i mu q e [(2 - eta) U_2 + H12*U_2]
      F_2 = -i mu q e^T [(2 - eta) U_h + H12*U_h] - side mu q (H22*U_2)
    On the Nyquist lines the factors odd in the aliased component are zero.
    """
    mu, eta = mat.mu, mat.eta
    q = modes.q
    qs = np.where(q > 0, q, 1.0)
    e1, e3 = modes.k1 / qs, modes.k3 / qs
    odd = modes.nyq1 | modes.nyq3
    e11, e33 = e1 * e1, e3 * e3
    e13 = np.where(odd, 0.0, e1 * e3)
    c1 = np.where(modes.nyq1, 0.0, e1)
    c3 = np.where(modes.nyq3, 0.0, e3)
    # Z[a, c, mode] = sum_m w_a(mode, m) * Uhat_c(n - m, mode)
    Z = np.einsum("aqm,mcq->acq", weights, hist_rev)
    Z11, Z22, Z33, Z12 = Z[0], Z[1], Z[2], Z[3]
    inst = 2.0 - eta
    F = np.empty((3, len(modes)), dtype=complex)
    F[0] = (-side * mu * q * (e11 * Z11[0] + e13 * Z11[2] + e33 * Z33[0] - e13 * Z33[2])
            + 1j * mu * q * c1 * (inst * current[1] + Z12[1]))
    F[2] = (-side * mu * q * (e13 * Z11[0] + e33 * Z11[2] - e13 * Z33[0] + e11 * Z33[2])
            + 1j * mu * q * c3 * (inst * current[1] + Z12[1]))
    F[1] = (-1j * mu * q * (c1 * (inst * current[0] + Z12[0]) + c3 * (inst * current[2] + Z12[2]))
            - side * mu * q * Z22[1])
    F[:, q == 0] = 0.0
    return F


def lag_limits(dT, n_cut, window):
    """Lags kept per mode under a truncation window in T: floor(window/dT) + 1,
    at most n_cut (all n_cut for k = 0)."""
    dT = np.asarray(dT, dtype=float)
    safe = np.where(dT > 0, dT, 1.0)
    lim = np.floor(window / safe) + 1
    return np.where(dT > 0, np.minimum(lim, n_cut), n_cut).astype(np.int64)


class SBIMOracle:
    """Time stepper of Eq. (SBI) for one half-space on a periodic N1 x N3 grid.

    ``step(u, v)`` takes the boundary displacement u_n and velocity v_n
    ([3][N3][N1], x1 fastest; step 3 of the hybrid loop in Section 2.4 passes
    u_{t+1} and the predicted velocity) and returns the traction tau_n
    ([3][N3][N1]) with the non-local term s_n and its half spectrum.
    """

    def __init__(self, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side,
                 tau_inf=(0.0, 0.0, 0.0), kernel="table", window=0.0):
        if n1 % 2 or n3 % 2 or n1 < 2 or n3 < 2:
            raise ValueError("n1, n3 must be even and >= 2")
        if side not in (1, -1):
            raise ValueError("side must be +1 or -1")
        if not (cp > cs > 0 and rho > 0 and dt > 0 and n_cut >= 1):
            raise ValueError("bad material / time step / cutoff")
        self.n1, self.n3, self.n_cut, self.side = n1, n3, n_cut, side
        self.mat = Material(cs, cp, rho)
        self.dt = dt
        self.tau_inf = np.asarray(tau_inf, dtype=float)
        self.modes = ModeSet.build(n1, n3, L1, L3)
        self.dT = self.modes.q * cs * dt
        t_max = float(self.dT.max()) * max(n_cut - 1, 1) + 1.0
        if kernel == "table":
            kern = KernelTable(self.mat.eta, t_max)
        elif kernel == "direct":
            kern = lambda T: kernels_direct(T, self.mat.eta)  # noqa: E731
        else:
            raise ValueError(kernel)
        # weights per distinct mode spacing, scattered back to all modes
        uniq, inv = np.unique(self.dT, return_inverse=True)
        wu = np.stack([trapezoid_weights(d, n_cut, kern) for d in uniq], axis=1)
        self.weights = wu[:, inv, :]             # (4, nmodes, n_cut)
        if window > 0:
            # mode-dependent truncation (the convolution truncation the paper cites
            # from Lapusta et al.): mode q keeps the lags with m dT_q <= window,
            # i.e. a window fixed in T = |k| c_s t, so a fixed number of periods
            self.lags = lag_limits(self.dT, n_cut, window)
            m = np.arange(n_cut)[None, :]
            self.weights = self.weights * (m < self.lags[:, None])[None]
        else:
            self.lags = np.full(self.dT.shape, n_cut)
        self.history = []                         # list of (3, nmodes) complex
        self.n = 0

    def step(self, u, v):
        u = np.asarray(u, dtype=float)
        v = np.asarray(v, dtype=float)
        U = dft2_forward(u).reshape(3, -1)
        self.history.append(U)
        L = min(self.n + 1, self.n_cut)
        hist_rev = np.stack(self.history[::-1][:L])      # (L, 3, nmodes)
        F = apply_modal_operator(self.modes, self.mat, self.side,
                                 self.weights[:, :, :L], hist_rev, U)
        F = F.reshape(3, self.n3, self.n1 // 2 + 1)
        s, imag = dft2_inverse(F, self.n1)
        coef = self.side * self.mat.mu / self.mat.cs
        tau = (self.tau_inf[:, None, None]
               - coef * self.mat.impedance[:, None, None] * v + s)
        self.n += 1
        return {"tau": tau, "s": s, "F": F, "imag": imag}

    def rewind(self):
        """Forget the last step (its displacement leaves the history), so that
        the next ``step`` evaluates the same time level again."""
        if self.n == 0:
            raise ValueError("nothing to rewind")
        self.history.pop()
        self.n -= 1


# ---------------------------------------------------------------------------
# Adjoint (transpose) of a sequence of traction updates, built as the literal
# transpose of each stage of the forward map for the real inner products
# <a, b> = sum_x a(x) b(x) on fields and sum over (Re, Im) parts on half spectra.
# ---------------------------------------------------------------------------
def modal_matrices(modes, mat, side, weights):
    """Cartesian 3x3 modal matrices A(m) with F_n = sum_m A(m) Uhat_{n-m}
    (Section 2.3; the same operator as ``apply_modal_operator``, written out
    entry by entry).  weights: (4, nmodes, L); returns (L, nmodes, 3, 3)."""
    mu, eta = mat.mu, mat.eta
    q = modes.q
    qs = np.where(q > 0, q, 1.0)
    e1, e3 = modes.k1 / qs, modes.k3 / qs
    odd = modes.nyq1 | modes.nyq3
    e11, e33 = e1 * e1, e3 * e3
    e13 = np.where(odd, 0.0, e1 * e3)
    c1 = np.where(modes.nyq1, 0.0, e1)
    c3 = np.where(modes.nyq3, 0.0, e3)
    L = weights.shape[2]
    A = np.zeros((L, len(modes), 3, 3), dtype=complex)
    for m in range(L):
        w11, w22, w33, w12 = (weights[k][:, m] for k in range(4))
        cpl = w12 + ((2.0 - eta) if m == 0 else 0.0)
        d = -side * mu * q
        A[m, :, 0, 0] = d * (e11 * w11 + e33 * w33)
        A[m, :, 0, 2] = d * (e13 * w11 - e13 * w33)
        A[m, :, 2, 0] = d * (e13 * w11 - e13 * w33)
        A[m, :, 2, 2] = d * (e33 * w11 + e11 * w33)
        A[m, :, 1, 1] = d * w22
        A[m, :, 0, 1] = 1j * mu * q * c1 * cpl
        A[m, :, 2, 1] = 1j * mu * q * c3 * cpl
        A[m, :, 1, 0] = -1j * mu * q * c1 * cpl
        A[m, :, 1, 2] = -1j * mu * q * c3 * cpl
    A[:, q == 0] = 0.0
    return A


def _half_column_weights(n1, n3):
    """c_k of the real inner product of half spectra: 1 on the self-conjugate
    columns j1 = 0 and j1 = n1/2, 2 elsewhere."""
    c = np.full((n3, n1 // 2 + 1), 2.0)
    c[:, 0] = 1.0
    c[:, n1 // 2] = 1.0
    return c


def dft2_inverse_transpose(g):
    """Transpose of ``dft2_inverse`` (half spectrum -> real field):
    F_bar = (c_k / (n1 n3)) x forward DFT of g."""
    g = np.asarray(g, dtype=float)
    _, n3, n1 = g.shape
    return dft2_forward(g) * (_half_column_weights(n1, n3) / (n1 * n3))[None]


def dft2_forward_transpose(Ub, n1):
    """Transpose of ``dft2_forward`` (real field -> half spectrum):
    u_bar(x) = Re sum_{half k} Ub_k e^{+i k x} (no doubling, no 1/N)."""
    Ub = np.asarray(Ub, dtype=complex)
    nc, n3, nh = Ub.shape
    E3 = _dft_matrix(n3, n3, +1.0)                     # [x3][r3]
    E1 = _dft_matrix(n1, n1, +1.0)[:, :nh]             # [x1][j1]
    return np.stack([(E3 @ Ub[c] @ E1.T).real for c in range(nc)])


def adjoint_sequence(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, tau_bar, kernel="table"):
    """Transpose of N consecutive updates started from rest: given tau_bar_n
    (N, 3, n3, n1), returns (u_bar, v_bar) with
    sum_n <tau_n, tau_bar_n> = sum_m <u_m, u_bar_m> + <v_m, v_bar_m>."""
    tau_bar = np.asarray(tau_bar, dtype=float)
    N = tau_bar.shape[0]
    mat = Material(cs, cp, rho)
    modes = ModeSet.build(n1, n3, L1, L3)
    dT = modes.q * cs * dt
    if kernel == "table":
        kern = KernelTable(mat.eta, float(dT.max()) * max(n_cut - 1, 1) + 1.0)
    else:
        kern = lambda T: kernels_direct(T, mat.eta)  # noqa: E731
    uniq, inv = np.unique(dT, return_inverse=True)
    wu = np.stack([trapezoid_weights(d, n_cut, kern) for d in uniq], axis=1)
    A = modal_matrices(modes, mat, side, wu[:, inv, :])           # (L, nm, 3, 3)
    AH = np.conj(np.swapaxes(A, 2, 3))
    nh = n1 // 2 + 1
    G = [dft2_inverse_transpose(tb).reshape(3, -1) for tb in tau_bar]
    u_bar = np.empty_like(tau_bar)
    for m in range(N):
        Ub = np.zeros((3, n3 * nh), dtype=complex)
        for lag in range(min(n_cut, N - m)):
            Ub += np.einsum("qab,bq->aq", AH[lag], G[m + lag])
        u_bar[m] = dft2_forward_transpose(Ub.reshape(3, n3, nh), n1)
    coef = side * mat.mu / cs
    v_bar = -coef * mat.impedance[None, :, None, None] * tau_bar
    return u_bar, v_bar


class SBIMAdjointOracle:
    """Transpose of a sequence of updates taken one step at a time in reverse
    time: ``step(tau_bar_m)`` for m = N-1, N-2, ... returns (u_bar_m, v_bar_m),
    the same stage transposes as ``adjoint_sequence`` (which it equals)."""

    def __init__(self, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, side, kernel="table"):
        self.n1, self.n3, self.n_cut, self.side = n1, n3, n_cut, side
        self.mat = Material(cs, cp, rho)
        modes = ModeSet.build(n1, n3, L1, L3)
        dT = modes.q * cs * dt
        kt = KernelTable(self.mat.eta, float(dT.max()) * max(n_cut - 1, 1) + 1.0)
        uniq, inv = np.unique(dT, return_inverse=True)
        wu = np.stack([trapezoid_weights(d, n_cut, kt) for d in uniq], axis=1)
        A = modal_matrices(modes, self.mat, side, wu[:, inv, :])
        self.AH = np.conj(np.swapaxes(A, 2, 3))
        self.future = []          # G of the steps after the current one, nearest first

    def step(self, tau_bar):
        G = dft2_inverse_transpose(tau_bar).reshape(3, -1)
        self.future.insert(0, G)
        del self.future[self.n_cut:]
        Ub = np.zeros_like(G)
        for lag, Gl in enumerate(self.future):
            Ub += np.einsum("qab,bq->aq", self.AH[lag], Gl)
        nh = self.n1 // 2 + 1
        u_bar = dft2_forward_transpose(Ub.reshape(3, self.n3, nh), self.n1)
        v_bar = -(self.side * self.mat.mu / self.mat.cs) * self.mat.impedance[:, None, None] * tau_bar
        return u_bar, v_bar
