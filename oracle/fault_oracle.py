"""FP64 CPU oracle of the pure-SBIM planar-fault solver.

TEST INFRASTRUCTURE ONLY (same rules as ``oracle/sbim_oracle.py``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
it; it imports nothing from the product package.

What is computed (Albertini, Elbanna & Kammer, Sections 2.1, 2.3 and 3):
a planar fault x2 = 0 with the linear slip-weakening law (Eq. (slipweak))
between two identical elastic half-spaces, each one represented only by its
boundary through Eq. (SBI).  The TPV3 benchmark of Section 3 has no off-fault
nonlinearity, so a boundary-only solver of this kind is the reference the paper
checks the hybrid scheme against; the paper gives no steps for it, and these are
written from Section 2.1's fault conditions and Eq. (SBI).

Per step n -> n+1, with the two faces' displacements u+, u- and velocities v+-,
the second-order predictor-corrector of Lapusta et al. (2000):
  1. predictor u*+- = u+-_n + dt v+-_n; solve (below) -> v*+-;
  2. corrector u+-_{n+1} = u+-_n + dt (v+-_n + v*+-)/2; the predictor's evaluation
     is withdrawn from the half-spaces' histories and the solve is repeated at
     u+-_{n+1} -> v+-_{n+1}.
The solve at face displacements u+-:
  a. S+- = the non-local tractions of Eq. (SBI) of the upper (side +1) and lower
     (side -1) half-spaces for u+- (radiation term left out: velocity 0).
  b. The faces carry one traction tau = S+ - z v+ = S- + z v- (z_i = eta_i mu/c_s,
     the radiation impedances of Eq. (SBI)); the normal velocities are equal (no
     opening, no interpenetration).  With V = v+ - v- and vbar = (v+ + v-)/2 this
     gives vbar = (S+ - S-)/(2z) and tau = tau_stick - z V/2, tau_stick = (S+ + S-)/2.
  c. Stick/slip on the shear traction vector as in the hybrid scheme: the fault
     sticks (V = 0) while |tau0 + tau_stick| <= sigma^n mu(|delta|),
     sigma^n = sigma0 - tau_stick_2, delta = u+ - u-; otherwise the shear traction
     is the strength along tau0 + tau_stick and V = 2 (tau_stick - tau)/z.
  d. v+- = vbar +- V/2.

Readings (the paper is silent):
  * The time stepping is Lapusta et al.'s predictor-corrector (two evaluations of
    each half-space per step); the one-evaluation explicit update u_{n+1} = u_n +
    dt v_n is unstable here: its highest modes (|k| c_s dt = 0.77 at
    dt = 0.3 dx/c_p) grow without bound over a few hundred steps.  The velocity
    enters Eq. (SBI) only through the radiation term, as in the paper.
  * ``symmetric=True`` is the paper's symmetry-plane reduction of TPV3
    (Section 3: only x2 > 0 is modelled, [u2] = 0 and sigma_22 constant): the
    lower face is the mirror image of the upper one (u-_1,3 = -u+_1,3,
    u-_2 = u+_2), so S-_1,3 = S+_1,3 and S-_2 = -S+_2 and only the upper
    half-space is evaluated.
Parity unpinned: none -- pinned by ``tests/test_oracle_fault.py``.
"""
from __future__ import annotations

import numpy as np

from .fem_oracle import FaultLaw
from .sbim_oracle import SBIMOracle

__all__ = ["PureSBIMOracle", "FaultLaw"]


class PureSBIMOracle:
    """Planar slip-weakening fault between two SBIM half-spaces (Section 3).

    State: ``u``, ``v`` of shape (2, 3, n3, n1), face 0 the upper (+) face and
    face 1 the lower (-) one, perturbations from the prestressed equilibrium.
    """

    def __init__(self, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, fault, symmetric=False,
                 window=0.0):
        self.n1, self.n3, self.dt = n1, n3, dt
        self.fault, self.symmetric = fault, symmetric
        mu = rho * cs * cs
        self.z = (mu / cs) * np.array([1.0, cp / cs, 1.0])[:, None, None]
        self.up = SBIMOracle(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, +1, window=window)
        self.lo = None if symmetric else SBIMOracle(n1, n3, L1, L3, cs, cp, rho, dt, n_cut, -1,
                                                    window=window)
        self.u = np.zeros((2, 3, n3, n1))
        self.v = np.zeros((2, 3, n3, n1))
        self.fault_traction = np.zeros((3, n3, n1))
        self.slip_rate = np.zeros((3, n3, n1))
        self.n = 0

    @staticmethod
    def mirror(x):
        """Mirror image across x2 = 0 of a face field: components 1, 3 change sign."""
        return np.stack([-x[0], x[1], -x[2]])

    @property
    def slip(self):
        return self.u[0] - self.u[1]

    def _solve(self, u_new):
        """Steps a-d at face displacements u_new: (v, traction, slip rate)."""
        z, fl = self.z, self.fault
        zero = np.zeros((3, self.n3, self.n1))
        s_up = self.up.step(u_new[0], zero)["s"]                       # step a
        if self.symmetric:                                             # mirror image
            s_lo = np.stack([s_up[0], -s_up[1], s_up[2]])
        else:
            s_lo = self.lo.step(u_new[1], zero)["s"]
        stick = 0.5 * (s_up + s_lo)                                    # step b
        vbar = (s_up - s_lo) / (2.0 * z)
        tau = stick.copy()
        if fl is not None:                                             # step c
            d = u_new[0] - u_new[1]
            slip = np.hypot(d[0], d[2])
            strength = (fl.sigma0 - stick[1]) * fl.friction(slip)
            t1, t3 = fl.tau0 + stick[0], stick[2]
            mag = np.hypot(t1, t3)
            over = mag > strength
            scale = np.where(over, strength / np.where(mag > 0, mag, 1.0), 1.0)
            tau[0] = np.where(over, t1 * scale, t1) - fl.tau0
            tau[2] = np.where(over, t3 * scale, t3)
        V = np.zeros_like(stick)
        V[0] = 2.0 * (stick[0] - tau[0]) / z[0]
        V[2] = 2.0 * (stick[2] - tau[2]) / z[2]
        return np.stack([vbar + 0.5 * V, vbar - 0.5 * V]), tau, V       # step d

    def _mirrored(self, u):
        if self.symmetric:
            u = u.copy()
            u[1] = self.mirror(u[0])
        return u

    def step(self):
        dt = self.dt
        u_pred = self._mirrored(self.u + dt * self.v)                  # predictor
        v_pred, _, _ = self._solve(u_pred)
        self.up.rewind()
        if self.lo is not None:
            self.lo.rewind()
        u_new = self._mirrored(self.u + 0.5 * dt * (self.v + v_pred))  # corrector
        self.v, self.fault_traction, self.slip_rate = self._solve(u_new)
        self.u = u_new
        self.n += 1
        return self.fault_traction
