"""Independent physics pin of the SBIM oracle's in-plane kernels: a single
Fourier mode e^{i k x1} of the upper half-space, solved directly from the
Navier equations (Section 2.1, Eq. (linelasticity) with the momentum balance)
by finite differences along x2, against Eq. (SBI) as the oracle evaluates it.

The boundary x2 = 0 follows a prescribed smooth displacement history of both
in-plane components (a C2 ramp); the column is deep enough that no wave returns
from its far end before t_end.  Its boundary traction sigma_2i(x2 = 0) must
equal the oracle's tau_i, which adds the radiation terms -(mu/c_s)(1, c_p/c_s)
v to the convolution with H11, H22, H12 and the (2 - eta) coupling, for the
same input.  The FD solution converges at second order in dx2 (checked), so the
agreement bounds any error in the kernels, their signs and the coupling."""
import numpy as np

from oracle.sbim_oracle import SBIMOracle
from tests._errors import Worst, max_abs_rel

CS, CP, RHO = 3464.0, 6000.0, 2670.0
MU = RHO * CS * CS
LAM = RHO * CP * CP - 2 * MU
N1, N3, DX = 8, 2, 100.0
K = 2 * np.pi / (N1 * DX)
T_RAMP = 0.03
U = np.array([1e-3, 0.2e-3 + 0.7e-3j])      # complex amplitudes of u1, u2


def _ramp(t):
    x = np.clip(t / T_RAMP, 0.0, 1.0)
    return x ** 3 * (10 - 15 * x + 6 * x * x)


def _dramp(t):
    x = np.clip(t / T_RAMP, 0.0, 1.0)
    return 30 * x * x * (1 - x) ** 2 / T_RAMP


def _column(t_end, dz):
    """Plane-strain Navier equations for u(x2) e^{i k x1}, central differences
    in x2 and time (leapfrog), Dirichlet data at x2 = 0, fixed far end."""
    depth = CP * t_end * 1.1 + 50.0
    nz = int(depth / dz) + 1
    nt = int(np.ceil(t_end / (0.4 * dz / CP)))
    dt = t_end / nt
    u = np.zeros((2, nz), complex)
    up = u.copy()
    ts, tr = [], []
    for n in range(nt + 1):
        t = n * dt
        u[:, 0] = U * _ramp(t)
        d0 = (-3 * u[:, 0] + 4 * u[:, 1] - u[:, 2]) / (2 * dz)
        tr.append([MU * (d0[0] + 1j * K * u[1, 0]), (LAM + 2 * MU) * d0[1] + 1j * K * LAM * u[0, 0]])
        ts.append(t)
        d2 = (u[:, 2:] - 2 * u[:, 1:-1] + u[:, :-2]) / dz ** 2
        d1 = (u[:, 2:] - u[:, :-2]) / (2 * dz)
        a = np.zeros_like(u)
        a[0, 1:-1] = (MU * d2[0] - (LAM + 2 * MU) * K * K * u[0, 1:-1] + 1j * K * (LAM + MU) * d1[1]) / RHO
        a[1, 1:-1] = ((LAM + 2 * MU) * d2[1] - MU * K * K * u[1, 1:-1] + 1j * K * (LAM + MU) * d1[0]) / RHO
        u, up = 2 * u - up + dt * dt * a, u
    return np.array(ts), np.array(tr)


def _oracle_errors(ts, tr, dt, t_end):
    steps = int(round(t_end / dt))
    o = SBIMOracle(N1, N3, N1 * DX, N3 * DX, CS, CP, RHO, dt, steps + 1, +1)
    ph = np.exp(1j * K * np.arange(N1) * DX)
    scale = np.abs(tr).max()
    worst = Worst()
    for n in range(steps):
        t = n * dt
        u = np.zeros((3, N3, N1))
        v = np.zeros((3, N3, N1))
        for c in (0, 1):
            u[c] = (U[c] * _ramp(t) * ph).real[None, :]
            v[c] = (U[c] * _dramp(t) * ph).real[None, :]
        tau = o.step(u, v)["tau"]
        amp = np.array([(tau[c, 0] * np.conj(ph)).sum() * 2 / N1 for c in (0, 1)])
        ref = np.array([np.interp(t, ts, tr[:, c].real) + 1j * np.interp(t, ts, tr[:, c].imag)
                        for c in (0, 1)])
        worst.update(max_abs_rel(amp, ref, scale))
    return worst.value


def test_in_plane_mode_matches_finite_difference_column():
    t_end = 8.0 / (K * CS)                     # T = k c_s t up to 8
    ts, tr = _column(t_end, 0.5)
    assert _oracle_errors(ts, tr, 1e-3, t_end) < 5e-4
    # the residual is the column's own discretisation error: the coarser column
    # is further from the oracle by the second-order factor
    ts2, tr2 = _column(t_end, 1.0)
    assert _oracle_errors(ts2, tr2, 1e-3, t_end) > 2.5 * _oracle_errors(ts, tr, 1e-3, t_end)
