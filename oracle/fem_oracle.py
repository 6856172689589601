"""FP64 CPU oracle of the hybrid FEM-SBIM time step.

TEST INFRASTRUCTURE ONLY (same rules as ``oracle/sbim_oracle.py``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import
it; it imports nothing from the product package.

What is computed (Albertini, Elbanna & Kammer):
  * Section 2.1: linear isotropic elasticity (Eq. (linelasticity)), momentum
    balance, a planar fault with the linear slip-weakening law (Eq. (slipweak)),
    fault strength tau^s = sigma^n mu(delta).
  * Section 2.2: 8-node trilinear hexahedra on a regular mesh, lumped mass,
    explicit predictor-corrector (Eqs. (fepred), (feintdisp), (tintf),
    (fecorr)), fault traction by the forward Lagrange-multiplier method: free
    slip-rate predictor (Eq. (freeslip)), stick traction through the fault
    impedance (Eq. (sticktraction)), stick/slip selection (Eq. (stickslip)).
  * Section 2.4: the staggered Neumann coupling: predict, hand u_{t+1} and the
    predicted velocity to the two SBIM half-spaces, apply f = +-A tau^SBI on the
    top / bottom boundary nodes, friction, acceleration increment, correction.

Readings (the paper is silent or inconsistent):
  * Eq. (feintdisp) as printed advances u by dt * v^pred = dt v + dt^2 a; the
    central-difference update u_{t+1} = u_t + dt v_t + dt^2/2 a_t is used, with
    the printed predictor and corrector (so v_{t+1} = v_t + dt/2 (a_t + a_{t+1})).
  * Stick/slip acts on the shear traction vector: |tau| <= tau^s sticks, else
    tau = tau^s tau/|tau|; the normal component always sticks (no opening or
    interpenetration, Section 2.1).
  * Perturbation formulation: FE fields are departures from the prestressed
    equilibrium; the fault shear traction is tau0 + tau, the normal stress
    (compression positive) sigma0 - tau_2.
  * The mesh is periodic in x1 and x3 (matching the periodic SBIM planes); the
    fault is the node plane at mid-depth, split into a minus copy (belongs to
    the elements below) and a plus copy (elements above).
  * f = +A tau^(+) on the top boundary (SBIM side +1, half-space above), and
    f = -A tau^(-) on the bottom boundary (side -1), A = h^2 per node.
Parity unpinned: none -- pinned by ``tests/test_oracle_fem.py``.
"""
from __future__ import annotations

import numpy as np

from .sbim_oracle import SBIMAdjointOracle, SBIMOracle


# ---------------------------------------------------------------------------
# Element matrices (Section 2.2: 8-node hexahedra; Section 2.1 Eq. (linelasticity))
# ---------------------------------------------------------------------------
def local_nodes():
    """Local node a = i + 2 j + 4 k at reference coordinates (2i-1, 2j-1, 2k-1)
    along (x1, x2, x3)."""
    return np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                     for a in range(8)], dtype=float)


def hex8_stiffness(h, lam, mu):
    """24 x 24 stiffness of a cube of side h (dof 3a + c), 2x2x2 Gauss."""
    xa = local_nodes()
    g = 1.0 / np.sqrt(3.0)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    K = np.zeros((24, 24))
    for gp in np.array(np.meshgrid([-g, g], [-g, g], [-g, g], indexing="ij")).reshape(3, -1).T:
        dN = np.zeros((8, 3))
        for a in range(8):
            f = 1 + xa[a] * gp
            for d in range(3):
                others = [e for e in range(3) if e != d]
                dN[a, d] = xa[a, d] * f[others[0]] * f[others[1]] / 8.0 * (2.0 / h)
        B = np.zeros((6, 24))
        for a in range(8):
            B[0, 3 * a + 0] = dN[a, 0]
            B[1, 3 * a + 1] = dN[a, 1]
            B[2, 3 * a + 2] = dN[a, 2]
            B[3, 3 * a + 0] = dN[a, 1]; B[3, 3 * a + 1] = dN[a, 0]   # 2 eps_12
            B[4, 3 * a + 1] = dN[a, 2]; B[4, 3 * a + 2] = dN[a, 1]   # 2 eps_23
            B[5, 3 * a + 0] = dN[a, 2]; B[5, 3 * a + 2] = dN[a, 0]   # 2 eps_13
        K += B.T @ D @ B * (h / 2.0) ** 3
    return K


class SlabMesh:
    """n1 x n2 x n3 cubes of side h, periodic in x1 and x3.  Node layers are
    numbered from the bottom; with a fault at element layer f = n2 // 2 the node
    plane there is split: layer f is the minus copy, layer f + 1 the plus copy."""

    def __init__(self, n1, n2, n3, h, fault=True):
        self.n1, self.n2, self.n3, self.h, self.fault = n1, n2, n3, h, fault
        self.f = n2 // 2
        self.layers = n2 + 2 if fault else n2 + 1
        e1, e2, e3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
        e1, e2, e3 = e1.ravel(), e2.ravel(), e3.ravel()
        conn = np.empty((e1.size, 8), dtype=np.int64)
        for a, (i, j, k) in enumerate(((a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8))):
            lay = e2 + j
            if fault:
                lay = np.where(e2 >= self.f, lay + 1, lay)
            conn[:, a] = self.node((e1 + i) % n1, lay, (e3 + k) % n3)
        self.conn = conn
        self.n_nodes = self.layers * n3 * n1

    def node(self, i1, layer, i3):
        return (layer * self.n3 + i3) * self.n1 + i1

    @property
    def top(self):
        return self.layers - 1


class FEMOracle:
    """State u, v, a as [layers][3][n3][n1] arrays; ``internal_force`` = K u."""

    def __init__(self, mesh, cs, cp, rho):
        self.mesh = mesh
        mu = rho * cs * cs
        lam = rho * cp * cp - 2 * mu
        self.Ke = hex8_stiffness(mesh.h, lam, mu)
        m = np.zeros(mesh.n_nodes)
        np.add.at(m, mesh.conn.ravel(), rho * mesh.h ** 3 / 8.0)
        self.mass = m.reshape(mesh.layers, 1, mesh.n3, mesh.n1)

    def internal_force(self, u):
        """K u by element-by-element assembly."""
        me = self.mesh
        flat = u.transpose(0, 2, 3, 1).reshape(-1, 3)           # node-major (node, comp)
        ue = flat[me.conn].reshape(-1, 24)
        fe = ue @ self.Ke.T
        out = np.zeros_like(flat)
        np.add.at(out, me.conn.ravel(), fe.reshape(-1, 3))
        return out.reshape(me.layers, me.n3, me.n1, 3).transpose(0, 3, 1, 2)


class FaultLaw:
    """Linear slip-weakening fault on the split plane (Section 2.1, Eq. (slipweak)).
    mu_s, tau0: [n3][n1] maps (Pa for tau0, the x1 shear prestress); mu_k, Dc,
    sigma0 scalars (sigma0 compression positive)."""

    def __init__(self, mu_s, mu_k, Dc, tau0, sigma0):
        self.mu_s = np.asarray(mu_s, dtype=float)
        self.mu_k, self.Dc, self.sigma0 = float(mu_k), float(Dc), float(sigma0)
        self.tau0 = np.asarray(tau0, dtype=float)

    def friction(self, slip):
        return np.where(slip < self.Dc, self.mu_s - (self.mu_s - self.mu_k) * slip / self.Dc,
                        self.mu_k)


class HybridOracle:
    """Hybrid FEM-SBIM step of Section 2.4 (``sbim=False``: free top and bottom
    surfaces; ``fault=None``: no fault traction, the split plane is welded by
    giving it the stick traction)."""

    def __init__(self, mesh, cs, cp, rho, dt, n_cut=None, fault=None, sbim=True):
        self.mesh, self.dt, self.fault = mesh, dt, fault
        self.fem = FEMOracle(mesh, cs, cp, rho)
        shape = (mesh.layers, 3, mesh.n3, mesh.n1)
        self.u, self.v, self.a = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        self.A = mesh.h ** 2
        self.sbim = sbim
        if sbim:
            L1, L3 = mesh.n1 * mesh.h, mesh.n3 * mesh.h
            self.top = SBIMOracle(mesh.n1, mesh.n3, L1, L3, cs, cp, rho, dt, n_cut, +1)
            self.bot = SBIMOracle(mesh.n1, mesh.n3, L1, L3, cs, cp, rho, dt, n_cut, -1)
        self.fault_traction = np.zeros((3, mesh.n3, mesh.n1))
        self.slip_rate = np.zeros((3, mesh.n3, mesh.n1))
        self.source = None      # optional callable: step index -> nodal force at t_{n+1}
        self.n = 0

    def step(self):
        me, dt, A = self.mesh, self.dt, self.A
        m = self.fem.mass
        v_pred = self.v + dt * self.a                                  # Eq. (fepred)
        u_new = self.u + dt * self.v + 0.5 * dt * dt * self.a          # central difference
        f = np.zeros_like(self.u) if self.source is None else self.source(self.n + 1).copy()
        if self.sbim:                                                  # steps 2-4 of Section 2.4
            t_top = self.top.step(u_new[me.top], v_pred[me.top])["tau"]
            t_bot = self.bot.step(u_new[0], v_pred[0])["tau"]
            f[me.top] += A * t_top
            f[0] -= A * t_bot
            self.last_tau_top, self.last_tau_bot = t_top, t_bot
        kint = self.fem.internal_force(u_new)
        if me.fault:                                                   # step 5
            p, q = me.f + 1, me.f
            a_free = (-kint + f) / m
            vfree = (v_pred - 0.5 * dt * self.a + dt * a_free)         # Eq. (freeslip)
            jump = vfree[p] - vfree[q]
            tau_stick = jump / (dt * A * (1.0 / m[p] + 1.0 / m[q]))   # Eq. (sticktraction)
            tau = tau_stick.copy()
            if self.fault is not None:                                 # Eq. (stickslip)
                fl = self.fault
                dslip = u_new[p] - u_new[q]
                slip = np.hypot(dslip[0], dslip[2])
                sigma_n = fl.sigma0 - tau_stick[1]
                strength = sigma_n * fl.friction(slip)
                t1 = fl.tau0 + tau_stick[0]
                t3 = tau_stick[2]
                mag = np.hypot(t1, t3)
                over = mag > strength
                scale = np.where(over, strength / np.where(mag > 0, mag, 1.0), 1.0)
                tau[0] = np.where(over, t1 * scale, t1) - fl.tau0
                tau[2] = np.where(over, t3 * scale, t3)
            f[p] -= A * tau
            f[q] += A * tau
            self.fault_traction = tau
        a_new = (-kint + f) / m                                        # Eq. (tintf)
        self.v = v_pred + 0.5 * dt * (a_new - self.a)                  # Eq. (fecorr)
        self.u, self.a = u_new, a_new
        if me.fault:
            self.slip_rate = self.v[me.f + 1] - self.v[me.f]
        self.n += 1

    def energy(self):
        """Kinetic + strain energy of the slab."""
        kin = 0.5 * np.sum(self.fem.mass * self.v ** 2)
        strain = 0.5 * np.sum(self.u * self.fem.internal_force(self.u))
        return kin, strain


# ---------------------------------------------------------------------------
# Gradient of a fault-traction misfit with respect to the slip-weakening
# distance Dc through the coupled run (reverse sweep of Section 2.4's step).
# ---------------------------------------------------------------------------
def forward_record(o, steps):
    """Run ``steps`` hybrid steps of the HybridOracle ``o`` and return the
    states before each step and the fault tractions after each step."""
    xs, taus = [], []
    for _ in range(steps):
        xs.append((o.u.copy(), o.v.copy(), o.a.copy()))
        o.step()
        taus.append(o.fault_traction.copy())
    return xs, np.array(taus)


def dc_gradient(mesh, cs, cp, rho, dt, n_cut, fault, xs, tau_bar):
    """d/dDc of sum_n <tau_n, tau_bar_n> (tau_n: fault traction after step n),
    per fault node, by the literal transpose of each step in reverse order.
    xs: states (u, v, a) before each step (a forward run from these states with
    the same parameters reproduces tau_n); tau_bar: [N][3][n3][n1].
    Returns (dDc map [n3][n1], lambda_0 = (u_bar, v_bar, a_bar) of the initial
    state)."""
    fem = FEMOracle(mesh, cs, cp, rho)
    m = fem.mass
    A = mesh.h ** 2
    L1, L3 = mesh.n1 * mesh.h, mesh.n3 * mesh.h
    adj_top = SBIMAdjointOracle(mesh.n1, mesh.n3, L1, L3, cs, cp, rho, dt, n_cut, +1)
    adj_bot = SBIMAdjointOracle(mesh.n1, mesh.n3, L1, L3, cs, cp, rho, dt, n_cut, -1)
    # forward replay to recover the boundary tractions of every step
    rep = HybridOracle(mesh, cs, cp, rho, dt, n_cut=n_cut, fault=fault)
    rep.u, rep.v, rep.a = (x.copy() for x in xs[0])
    t_top, t_bot = [], []
    for _ in range(len(xs)):
        rep.step()
        t_top.append(rep.last_tau_top)
        t_bot.append(rep.last_tau_bot)
    p, q = mesh.f + 1, mesh.f
    fl = fault
    lu = np.zeros_like(xs[0][0]); lv = np.zeros_like(lu); la = np.zeros_like(lu)
    dDc = np.zeros((mesh.n3, mesh.n1))
    for n in range(len(xs) - 1, -1, -1):
        u, v, a = xs[n]
        # forward quantities of step n
        v_pred = v + dt * a
        u_new = u + dt * v + 0.5 * dt * dt * a
        f = np.zeros_like(u)
        f[mesh.top] += A * t_top[n]
        f[0] -= A * t_bot[n]
        a_free = (-fem.internal_force(u_new) + f) / m
        vfree = v_pred - 0.5 * dt * a + dt * a_free
        imp = dt * A * (1.0 / m[p] + 1.0 / m[q])
        stick = (vfree[p] - vfree[q]) / imp
        du = u_new[p] - u_new[q]
        slip = np.hypot(du[0], du[2])
        sig = fl.sigma0 - stick[1]
        fric = fl.friction(slip)
        S = sig * fric
        t1, t3 = fl.tau0 + stick[0], stick[2]
        mag = np.hypot(t1, t3)
        over = mag > S
        # corrector transpose: v' = v_pred + dt/2 (an - a), a' = an
        l_vp = lv.copy()
        l_an = 0.5 * dt * lv + la
        l_a = -0.5 * dt * lv
        l_un = lu.copy()
        # fault forces: an[p] -= A tau / m[p], an[q] += A tau / m[q]
        l_af = l_an.copy()
        tb = -A / m[p] * l_an[p] + A / m[q] * l_an[q] + tau_bar[n]
        # fault traction
        l_stick = tb.copy()
        magc = np.where(mag > 0, mag, 1.0)
        th1, th3 = t1 / magc, t3 / magc
        proj = th1 * tb[0] + th3 * tb[2]
        l_t1 = S / magc * (tb[0] - th1 * proj)
        l_t3 = S / magc * (tb[2] - th3 * proj)
        l_S = proj
        weak = slip < fl.Dc
        dmu_dslip = np.where(weak, -(fl.mu_s - fl.mu_k) / fl.Dc, 0.0)
        dmu_dDc = np.where(weak, (fl.mu_s - fl.mu_k) * slip / fl.Dc ** 2, 0.0)
        l_stick[0] = np.where(over, l_t1, tb[0])
        l_stick[2] = np.where(over, l_t3, tb[2])
        l_stick[1] = tb[1] + np.where(over, -fric * l_S, 0.0)
        l_slip = np.where(over, l_S * sig * dmu_dslip, 0.0)
        dDc += np.where(over, l_S * sig * dmu_dDc, 0.0)
        sl = np.where(slip > 0, slip, 1.0)
        for c in (0, 2):
            g = np.where(slip > 0, l_slip * du[c] / sl, 0.0)
            l_un[p, c] += g
            l_un[q, c] -= g
        # stick = (vfree[p] - vfree[q]) / imp, vfree = v_pred - dt/2 a + dt a_free
        for lay, sgn in ((p, 1.0), (q, -1.0)):
            lvf = sgn * l_stick / imp
            l_vp[lay] += lvf
            l_a[lay] += -0.5 * dt * lvf
            l_af[lay] += dt * lvf
        # a_free = (-K u_new + f) / m
        l_F = l_af / m
        l_un += -fem.internal_force(l_F)
        ub, vb = adj_top.step(A * l_F[mesh.top])
        l_un[mesh.top] += ub
        l_vp[mesh.top] += vb
        ub, vb = adj_bot.step(-A * l_F[0])
        l_un[0] += ub
        l_vp[0] += vb
        # predictor transpose: v_pred = v + dt a, u_new = u + dt v + dt^2/2 a
        lu = l_un
        lv = l_vp + dt * l_un
        la = l_a + dt * l_vp + 0.5 * dt * dt * l_un
    return dDc, (lu, lv, la)
