"""The dual-splitting time step of Sec. 2.2 with the V3c spatial variant
(oracle; test infrastructure).

One step from t^n to t^(n+1) = t^n + dt with the order-J BDF / extrapolation
constants of Karniadakis, Israeli and Orszag (1991) (gamma0, alpha_i, beta_i;
``BDF_EX`` below), for J = 1, 2, 3:

(i)   explicit convective step, Eq. (convstepspat):
        M u_hat = ( M sum_i alpha_i u^(n-i) + dt sum_i beta_i C(u^(n-i)) + dt M f ) / gamma0
      with C the weak convective term (``convective.ConvectiveOp``).
(ii)  pressure Poisson equation, Eq. (poissonspat) with a(q, u_hat) of
      Eq. (av3) and the flux Pi* of Eq. (ipflux) on the velocity-Dirichlet
      boundary (the walls, where the pressure has Neumann data):
        L_N p = (gamma0/dt) D u_hat + (q, h)_(walls),
        h = -( sum_i beta_i ( div F^c(u^(n-i)) + nu curl omega^(n-i) ) - f ) . n,
      omega the cell-wise L2 projection of curl u (Sec. 3.2 (ii)); dg/dt = 0
      (no-slip walls at rest).  L_N is the SIPG Laplacian with Neumann walls;
      the problem is singular and solved for the zero-mean p (Sec. 5.1).
(iii) projection with the div-div penalty, Eq. (div-div) with b of Eq. (bv3):
        (M + tau_D B) u_hathat = M u_hat + (dt/gamma0) G p,
      tau_D of Eq. (tauD) from u^n.
(iv)  implicit viscous step, Eq. (visc) in the divergence form of Sec. 3.2 (iii):
        ((gamma0/dt) M + A_nu) u^(n+1) = (gamma0/dt) M u_hathat.

The first steps raise the order one by one (Sec. 2.2) unless the caller
provides older time levels.  The linear systems are solved by CG to a tight
tolerance (the pressure for its zero-mean solution) on assembled matrices,
from the previous pressure and from u_hathat.

Velocity boundaries: periodic and no-slip (Dirichlet, g_u = 0) walls; outflow
(Neumann) velocity boundaries are not modelled.  Layout: u[d, cell, i].
"""
import dataclasses

import numpy as np
import scipy.sparse as sp

from .convective import ConvectiveOp
from .mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec
from .projection import ProjectionOps
from .sipg import SIPG
from .solvers import cg
from .viscous import ViscousOp

# (gamma0, alpha_0..J-1, beta_0..J-1) of the order-J BDF / extrapolation pair
BDF_EX = {
    1: (1.0, (1.0,), (1.0,)),
    2: (1.5, (2.0, -0.5), (2.0, -1.0)),
    3: (11.0 / 6.0, (3.0, -1.5, 1.0 / 3.0), (3.0, -3.0, 1.0)),
}


def pressure_spec(spec):
    """The same mesh with the velocity-Dirichlet walls as pressure-Neumann faces."""
    swap = {DIRICHLET: NEUMANN, PERIODIC: PERIODIC}
    for bc in spec.bc_lo + spec.bc_hi:
        if bc not in swap:
            raise ValueError("velocity boundaries must be periodic or no-slip walls")
    return dataclasses.replace(spec, bc_lo=tuple(swap[b] for b in spec.bc_lo),
                               bc_hi=tuple(swap[b] for b in spec.bc_hi))


class DualSplitting:
    def __init__(self, spec, k, nu, dt, order=3, zeta=1.0, penalty_factor=1.0, rtol=1e-13):
        if order not in BDF_EX:
            raise ValueError("order must be 1, 2 or 3")
        self.spec, self.k, self.nu, self.dt, self.order, self.zeta = spec, k, nu, dt, order, zeta
        self.rtol = rtol
        self.P = (k + 1) ** 3
        self.N = spec.ncell * self.P
        self.conv = ConvectiveOp(spec, k)
        self.proj = ProjectionOps(spec, k)
        self.visc = ViscousOp(spec, k, penalty_factor)
        self.lap = SIPG(pressure_spec(spec), k, penalty_factor).assemble()
        self.sipg = self.visc.sipg
        self.A_nu = self.visc.assemble(nu=nu, mass_coef=0.0)
        M = self.sipg.assemble(mass_coef=1.0, stiffness=False)
        self.M3 = sp.block_diag([M, M, M]).tocsr()
        # wall faces: (cell, d, side)
        self.walls = [(e, d, side) for e in range(spec.ncell) for d in range(3) for side in (0, 1)
                      if not self.sipg.interior[d, side, e] and self.sipg.bkind[(d, side)] == DIRICHLET]
        self.u_hist, self.c_hist, self.h_hist = [], [], []
        self.p_last = None  # initial guess of the next pressure solve

    # ------------------------------------------------------------ pieces
    def vorticity(self, u):
        """omega = cell-wise L2 projection of curl u: M_e omega_e = (v, curl u)_e."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        w = np.zeros_like(u)
        for e in range(self.spec.ncell):
            cq = self.proj._cq(e)
            # (phi_i, d u_c / d x_d)_e = sum_j (d phi_j / d x_d, phi_i)_e u_c,j = C[d]^T u_c
            g = [[cq.C[d].T @ u[c, e] for d in range(3)] for c in range(3)]  # g[c][d]
            r = np.stack([g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]])
            w[:, e, :] = np.linalg.solve(cq.M, r.T).T
        return w.ravel()

    def wall_values(self, u):
        """(div F^c(u) + nu curl omega) . n at the Gauss points of every wall face
        (k+1 per direction), from the own cell: a list of arrays, one per face."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        w = self.vorticity(u).reshape(3, self.spec.ncell, self.P)
        out = []
        for e, d, side in self.walls:
            n, wA, phif, gradf = self.visc._cq(e).face[(d, side)]
            uq = phif @ u[:, e, :].T                               # (q, c)
            G = np.einsum("qbk,cb->qck", gradf, u[:, e, :])        # d u_c / d x_k
            Gw = np.einsum("qbk,cb->qck", gradf, w[:, e, :])
            div = np.einsum("qcc->q", G)
            divF = np.einsum("qj,qij->qi", uq, G) + uq * div[:, None]   # d_j (u_i u_j)
            curl = np.stack([Gw[:, 2, 1] - Gw[:, 1, 2], Gw[:, 0, 2] - Gw[:, 2, 0], Gw[:, 1, 0] - Gw[:, 0, 1]],
                            axis=1)
            out.append(np.einsum("qi,qi->q", divF + self.nu * curl, n))
        return out

    def wall_rhs(self, hvals):
        """(q, h)_F on the wall faces for values h at their Gauss points."""
        y = np.zeros((self.spec.ncell, self.P))
        for (e, d, side), h in zip(self.walls, hvals):
            _, wA, phif, _ = self.visc._cq(e).face[(d, side)]
            y[e] += phif.T @ (wA * h)
        return y.ravel()

    def wall_normals_dot(self, f):
        """f . n at the Gauss points of every wall face."""
        return [self.visc._cq(e).face[(d, side)][0] @ np.asarray(f, dtype=np.float64)
                for e, d, side in self.walls]

    # ------------------------------------------------------------ state
    def reset(self, dt):
        """Change the time step and forget the history."""
        self.dt = dt
        self.u_hist, self.c_hist, self.h_hist = [], [], []
        self.p_last = None

    def set_history(self, levels):
        """levels = [u^n, u^(n-1), ...] (most recent first, at most ``order``)."""
        self.u_hist = [np.asarray(v, dtype=np.float64).copy() for v in levels[: self.order]]
        self.c_hist = [self.conv.apply(v) for v in self.u_hist]
        self.h_hist = [self.wall_values(v) for v in self.u_hist]

    def step(self, f=(0.0, 0.0, 0.0)):
        """Advance one step with the constant body force f at t^(n+1); returns
        (u^(n+1), p^(n+1), details)."""
        J = min(self.order, len(self.u_hist))
        g0, alpha, beta = BDF_EX[J]
        dt, N = self.dt, self.N
        fv = np.repeat(np.asarray(f, dtype=np.float64), N)
        # (i) convective step
        ext = sum(a * v for a, v in zip(alpha, self.u_hist))
        csum = sum(b * c for b, c in zip(beta, self.c_hist))
        uhat = (ext + dt * self.sipg.inverse_mass_apply(csum) + dt * fv) / g0
        # (ii) pressure
        fn = self.wall_normals_dot(f)
        h = [-(sum(b * hh[i] for b, hh in zip(beta, self.h_hist)) - fn[i]) for i in range(len(self.walls))]
        rhs_p = (g0 / dt) * self.proj.divergence(uhat) + self.wall_rhs(h)
        p, p_its, _ = cg(lambda v: self.lap @ v, rhs_p, x0=self.p_last, rtol=self.rtol, zero_mean=True)
        self.p_last = p
        # (iii) projection
        tau = self.proj.tau_div(self.u_hist[0], self.zeta, dt)
        rhs_proj = self.proj.mass(uhat) + (dt / g0) * self.proj.gradient(p)
        uhh = self.proj.project(rhs_proj, tau)
        # (iv) viscous step
        A = (g0 / dt) * self.M3 + self.A_nu
        u_new, v_its, _ = cg(lambda v: A @ v, (g0 / dt) * self.proj.mass(uhh), x0=uhh, rtol=self.rtol)
        self.u_hist = [u_new] + self.u_hist[: self.order - 1]
        self.c_hist = [self.conv.apply(u_new)] + self.c_hist[: self.order - 1]
        self.h_hist = [self.wall_values(u_new)] + self.h_hist[: self.order - 1]
        return u_new, p, dict(order=J, uhat=uhat, uhathat=uhh, tau=tau, p_iters=p_its, v_iters=v_its, rhs_p=rhs_p)
