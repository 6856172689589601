"""Pins of the oracle's full traction update (Section 2.3, Eq. (SBI)): the
direct DFT against numpy's FFT and a brute-force sum, the k = 0 plane-wave
limit, the antiplane impulse response against J1(T)/T, the quasi-static limit
against an independent elastostatic solution (both half-spaces), passivity,
and exact symmetries."""
import numpy as np
import pytest

from oracle.sbim_oracle import SBIMOracle, dft2_forward, dft2_inverse
from paper_2102_08756_gb300.synth import separable_history
from tests._elastic import static_traction

CS, CP, RHO = 3464.0, 6000.0, 2670.0
MU = RHO * CS * CS
ETA = CP / CS


def test_dft_matches_fft_and_brute_force():
    rng = np.random.default_rng(0)
    u = rng.normal(size=(3, 6, 8))
    F = dft2_forward(u)
    np.testing.assert_allclose(F, np.fft.rfft2(u), rtol=0, atol=1e-12)
    # brute force O(N^4) on the same grid
    n3, n1 = 6, 8
    x3, x1 = np.meshgrid(np.arange(n3), np.arange(n1), indexing="ij")
    for c in range(3):
        for r3 in range(n3):
            for j1 in range(n1 // 2 + 1):
                ref = np.sum(u[c] * np.exp(-2j * np.pi * (j1 * x1 / n1 + r3 * x3 / n3)))
                assert abs(F[c, r3, j1] - ref) < 1e-11
    back, imag = dft2_inverse(F, n1)
    np.testing.assert_allclose(back, u, atol=1e-13)
    assert imag < 1e-13
    np.testing.assert_allclose(back, np.fft.irfft2(F, s=(n3, n1)), atol=1e-13)


def _oracle(n=8, side=1, n_cut=64, dt=None, L=None):
    dx = 100.0
    L = L or n * dx
    return SBIMOracle(n, n, L, L, CS, CP, RHO, dt or 0.3 * dx / CP, n_cut, side)


@pytest.mark.parametrize("side", [1, -1])
def test_uniform_mode_is_plane_wave_radiation(side):
    """k = 0: s = 0 and tau = -side (rho c_s v1, rho c_p v2, rho c_s v3)."""
    o = _oracle(side=side)
    rng = np.random.default_rng(1)
    for _ in range(5):
        u = np.ones((3, 8, 8)) * rng.normal(size=(3, 1, 1))
        v = np.ones((3, 8, 8)) * rng.normal(size=(3, 1, 1))
        out = o.step(u, v)
        assert np.max(np.abs(out["s"])) < 1e-6 * MU * 1e-3
        imp = np.array([RHO * CS, RHO * CP, RHO * CS])
        np.testing.assert_allclose(out["tau"], -side * imp[:, None, None] * v, rtol=1e-12)


@pytest.mark.parametrize("side", [1, -1])
def test_antiplane_impulse_response_is_bessel(side):
    """u3 = delta_{n0} cos(k1 x1) on a mode along x1 is pure antiplane; the
    non-local traction is -side mu q w33(n) cos(k1 x1) with the trapezoid
    weights of J1(T)/T: w(0) = dT/4, w(n) = dT J1(n dT)/(n dT)."""
    special = pytest.importorskip("scipy.special")
    n, dx, steps = 8, 100.0, 40
    o = _oracle(n=n, side=side, n_cut=64)
    k1 = 2 * np.pi / (n * dx)
    x1 = np.arange(n) * dx
    dT = k1 * CS * o.dt
    pat = np.cos(k1 * x1)[None, :] * np.ones((n, 1))
    for m in range(steps):
        u = np.zeros((3, n, n))
        if m == 0:
            u[2] = pat
        out = o.step(u, np.zeros_like(u))
        T = m * dT
        w = dT / 4 if m == 0 else dT * special.j1(T) / T
        np.testing.assert_allclose(out["s"][2], -side * MU * k1 * w * pat, rtol=1e-10, atol=1e-6 * MU * k1 * dT)
        assert np.max(np.abs(out["s"][:2])) < 1e-9 * MU * k1 * dT


@pytest.mark.parametrize("side", [1, -1])
def test_quasistatic_limit_matches_elastostatics(side):
    """A slowly ramped, then held, oblique single mode: once the 3000-lag
    window holds only the constant displacement, the traction equals the
    elastostatic half-space traction up to the truncated tail and the
    trapezoid error (both below 3e-3 here)."""
    n, dx = 4, 100.0
    dt, n_cut, ramp = 1e-3, 3000, 100
    o = _oracle(n=n, side=side, n_cut=n_cut, dt=dt)
    L = n * dx
    k = np.array([2 * np.pi / L, 2 * np.pi / L])
    q = np.hypot(*k)
    e1, e3 = k / q
    Dxi, D2, Dp = 0.7 - 0.2j, -0.4 + 0.5j, 0.3 + 0.1j
    D = np.array([e1 * Dxi - e3 * Dp, D2, e3 * Dxi + e1 * Dp]) * 1e-3
    x3, x1 = np.meshgrid(np.arange(n) * dx, np.arange(n) * dx, indexing="ij")
    phase = np.exp(1j * (k[0] * x1 + k[1] * x3))
    field = np.real(D[:, None, None] * phase[None])
    for m in range(n_cut + ramp + 2):
        r = np.sin(0.5 * np.pi * min(m, ramp) / ramp) ** 2
        out = o.step(r * field, np.zeros_like(field))
    sxi, s22 = static_traction(ETA, np.array([Dxi, D2]) * 1e-3, side)
    sp = -side * Dp * 1e-3
    sig = MU * q * np.array([e1 * sxi - e3 * sp, s22, e3 * sxi + e1 * sp])
    ref = np.real(sig[:, None, None] * phase[None])
    err = np.max(np.abs(out["tau"] - ref)) / np.max(np.abs(ref))
    assert err < 3e-3, err


@pytest.mark.parametrize("side", [1, -1])
def test_passivity(side):
    """Work done on the half-space from rest, -side sum tau . (u_n - u_{n-1}),
    is non-negative at every step (no truncation inside the run)."""
    n, dx, steps = 16, 100.0, 60
    dt = 0.3 * dx / CP
    o = SBIMOracle(n, n, n * dx, n * dx, CS, CP, RHO, dt, 64, side)
    hist = separable_history(n, n, n * dx, n * dx, steps, dt, CS, seed=5)
    work, prev = 0.0, np.zeros((3, n, n))
    for m in range(steps):
        u = hist.u(m)
        out = o.step(u, hist.v(m))
        work += -side * np.sum(out["tau"] * (u - prev))
        prev = u
        assert work >= -1e-12 * MU * 1e-6
    assert work > 0
    assert out["imag"] < 1e-9 * np.max(np.abs(out["s"]))


def test_linearity_translation_and_swap():
    n, dx, steps = 8, 100.0, 12
    dt = 0.3 * dx / CP
    h1 = separable_history(n, n, n * dx, n * dx, steps, dt, CS, seed=1, spectrum="k2")
    h2 = separable_history(n, n, n * dx, n * dx, steps, dt, CS, seed=2, spectrum="k2")

    def run(fu, fv):
        o = SBIMOracle(n, n, n * dx, n * dx, CS, CP, RHO, dt, 8, 1)
        return [o.step(fu(m), fv(m)) for m in range(steps)]

    a = run(h1.u, h1.v)
    b = run(h2.u, h2.v)
    ab = run(lambda m: 2 * h1.u(m) - 3 * h2.u(m), lambda m: 2 * h1.v(m) - 3 * h2.v(m))
    scale = np.max(np.abs(ab[-1]["tau"]))
    for x, y, z in zip(a, b, ab):
        np.testing.assert_allclose(z["tau"], 2 * x["tau"] - 3 * y["tau"], atol=1e-10 * scale)
    # translation by (1, 2) cells
    sh = run(lambda m: np.roll(h1.u(m), (2, 1), axis=(1, 2)), lambda m: np.roll(h1.v(m), (2, 1), axis=(1, 2)))
    for x, y in zip(a, sh):
        np.testing.assert_allclose(y["tau"], np.roll(x["tau"], (2, 1), axis=(1, 2)), atol=1e-10 * scale)
    # swap x1 <-> x3 together with components 1 <-> 3 (square grid)
    perm = [2, 1, 0]
    sw = run(lambda m: np.swapaxes(h1.u(m)[perm], 1, 2), lambda m: np.swapaxes(h1.v(m)[perm], 1, 2))
    for x, y in zip(a, sw):
        np.testing.assert_allclose(y["tau"], np.swapaxes(x["tau"][perm], 1, 2), atol=1e-10 * scale)


def test_nyquist_content_gives_real_output():
    """White-noise input fills the Nyquist lines; the Hermitian extension of the
    oracle's half spectrum must still be consistent (real inverse)."""
    n, dx = 8, 100.0
    o = SBIMOracle(n, 6, n * dx, 6 * dx, CS, CP, RHO, 0.3 * dx / CP, 8, -1)
    rng = np.random.default_rng(4)
    for _ in range(6):
        out = o.step(rng.normal(size=(3, 6, n)) * 1e-3, rng.normal(size=(3, 6, n)))
        assert out["imag"] < 1e-12 * np.max(np.abs(out["s"]))


def test_truncation_window_keeps_the_early_lags():
    """A window of 3 (in T) keeps the lags with m dT <= 3: the antiplane
    impulse response is the untruncated one up to there and zero after."""
    n, dx = 8, 100.0
    full = _oracle(n=n, n_cut=64)
    cut = SBIMOracle(n, n, n * dx, n * dx, CS, CP, RHO, 0.3 * dx / CP, 64, 1, window=3.0)
    k1 = 2 * np.pi / (n * dx)
    dT = k1 * CS * full.dt
    keep = int(np.floor(3.0 / dT)) + 1
    pat = np.cos(k1 * np.arange(n) * dx)[None, :] * np.ones((n, 1))
    for m in range(keep + 5):
        u = np.zeros((3, n, n))
        if m == 0:
            u[2] = pat
        a = full.step(u, np.zeros_like(u))["s"][2]
        b = cut.step(u, np.zeros_like(u))["s"][2]
        if m < keep:
            np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12 * np.max(np.abs(a)))
        else:
            assert np.max(np.abs(b)) < 1e-9 * np.max(np.abs(a)) + 1e-300


def test_rewind_evaluates_the_same_level_again():
    """``rewind`` withdraws the last step: stepping a, rewinding and stepping b
    gives what a handle that only ever saw b at that level gives."""
    rng = np.random.default_rng(11)
    args = (8, 6, 800.0, 600.0, 3464.0, 6000.0, 2670.0, 0.005, 5, 1)
    x = [rng.normal(size=(3, 6, 8)) for _ in range(9)]
    a = SBIMOracle(*args)
    b = SBIMOracle(*args)
    for m in range(7):
        a.step(x[m], x[m + 1])
        b.step(x[m], x[m + 1])
    a.step(x[8], x[0])
    a.rewind()
    assert a.n == 7
    ra = a.step(x[0], x[1])["tau"]
    rb = b.step(x[0], x[1])["tau"]
    assert np.array_equal(ra, rb)
