"""Velocity-pressure coupling operators of the pressure-projection step, by
dense quadrature (oracle; test infrastructure).

* Divergence, Eq. (av3) (variant V3c): for a pressure test function q and a
  velocity u,
      a(q, u) = (grad q, u)_e - (q, {{u}}^ND . n)_{de},
  summed over the cells; {{u}}^ND is the average on interior (and periodic)
  faces and the own trace u^- on boundary faces (Sec. 3.1).  The factor
  gamma0/dt of the paper is left to the caller.
* Gradient, Eq. (bv3): for a velocity test function v and a pressure p,
      b(v, p) = (div v, p)_e - (v, {{p}}^ND n)_{de},
  again without the factor dt/gamma0.
* Div-div penalised local projection, Eq. (div-div): per cell
      (v, w)_e + tau_D (div v, div w)_e = rhs_e(v),
  with tau_D = zeta_D ||ubar_e|| h dt, Eq. (tauD): ubar_e the volume average
  of the velocity over the cell, h = V_e^(1/3).

Everything is evaluated by dense quadrature with the full Jacobian of the
iso-parametric map at every Gauss point (k+1 per direction, Sec. 5), as in
``sipg.SIPG``, whose geometry keys and face tables are reused.

Layouts: velocity u[d, cell, i] (d = x, y, z component), pressure p[cell, i],
i = (c p + b) p + a with a along x.
"""
import numpy as np

from .sipg import SIPG


class CellQuadrature:
    """Per-geometry-key quadrature data of one mapped cell."""

    def __init__(self, op, xn):
        J = np.einsum("ik,dqi->qkd", xn, op.dphi_vol)  # dx_k / dxi_d
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        grad = np.einsum("qdk,dqi->qik", Jinv, op.dphi_vol)  # grad[q, i, k] = d phi_i / d x_k
        wdet = op.w_vol * det
        phi = op.phi_vol
        self.volume = wdet.sum()
        self.mvec = wdet @ phi  # integral of each basis function
        self.M = np.einsum("q,qi,qj->ij", wdet, phi, phi)
        # C[d][i, j] = (d phi_i / d x_d, phi_j)_e
        self.C = np.stack([np.einsum("q,qi,qj->ij", wdet, grad[:, :, d], phi) for d in range(3)])
        # B[d, e][i, j] = (d phi_i / d x_d, d phi_j / d x_e)_e
        self.B = np.einsum("q,qid,qje->deij", wdet, grad, grad)
        self.face = {}
        for d in range(3):
            for side in (0, 1):
                phif, dphif, wref = op.face_tables[(d, side)]
                Jf = np.einsum("ik,dqi->qkd", xn, dphif)
                detf = np.linalg.det(Jf)
                Jinvf = np.linalg.inv(Jf)
                a = detf[:, None] * Jinvf[:, d, :]  # Nanson: det(J) J^-T e_d
                norm = np.linalg.norm(a, axis=1)
                n = (1.0 if side == 1 else -1.0) * a / norm[:, None]
                self.face[(d, side)] = (n, wref * norm, phif)


class ProjectionOps:
    """Divergence, gradient and div-div projection on a structured mesh."""

    def __init__(self, spec, k):
        self.sipg = SIPG(spec, k)
        self.spec, self.k, self.p, self.P = spec, k, k + 1, (k + 1) ** 3
        from .mesh import cell_node_coords
        first = {}
        for c, key in enumerate(self.sipg.cell_key):
            first.setdefault(int(key), c)
        self.q = [CellQuadrature(self.sipg, cell_node_coords(spec, self.p, [first[kk]])[0])
                  for kk in range(len(first))]

    def _cq(self, e):
        return self.q[self.sipg.cell_key[e]]

    def divergence(self, u):
        """y_i = (grad phi_i, u)_e - (phi_i, {{u}}^ND . n)_{de}, Eq. (av3)."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        y = np.zeros((self.spec.ncell, self.P))
        for e in range(self.spec.ncell):
            cq = self._cq(e)
            y[e] = sum(cq.C[d] @ u[d, e] for d in range(3))
            for d in range(3):
                for side in (0, 1):
                    n, wA, phif = cq.face[(d, side)]
                    um = phif @ u[:, e, :].T  # (nq, 3) own trace
                    if self.sipg.interior[d, side, e]:
                        nb = self.sipg.nb[d, side, e]
                        _, _, phin = self._cq(nb).face[(d, 1 - side)]
                        avg = 0.5 * (um + phin @ u[:, nb, :].T)
                    else:
                        avg = um
                    flux = np.einsum("qk,qk->q", avg, n)
                    y[e] -= phif.T @ (wA * flux)
        return y.ravel()

    def gradient(self, p):
        """y_(d, i) = (d phi_i / d x_d, p)_e - (phi_i, {{p}}^ND n_d)_{de}, Eq. (bv3)."""
        p = np.asarray(p, dtype=np.float64).reshape(self.spec.ncell, self.P)
        y = np.zeros((3, self.spec.ncell, self.P))
        for e in range(self.spec.ncell):
            cq = self._cq(e)
            for d in range(3):
                y[d, e] = cq.C[d] @ p[e]
            for fd in range(3):
                for side in (0, 1):
                    n, wA, phif = cq.face[(fd, side)]
                    pm = phif @ p[e]
                    if self.sipg.interior[fd, side, e]:
                        nb = self.sipg.nb[fd, side, e]
                        _, _, phin = self._cq(nb).face[(fd, 1 - side)]
                        avg = 0.5 * (pm + phin @ p[nb])
                    else:
                        avg = pm
                    for d in range(3):
                        y[d, e] -= phif.T @ (wA * avg * n[:, d])
        return y.ravel()

    def mass(self, u, ncomp=3):
        u = np.asarray(u, dtype=np.float64).reshape(ncomp, self.spec.ncell, self.P)
        y = np.zeros_like(u)
        for e in range(self.spec.ncell):
            M = self._cq(e).M
            for c in range(ncomp):
                y[c, e] = M @ u[c, e]
        return y.ravel()

    def tau_div(self, u, zeta, dt):
        """tau_D per cell, Eq. (tauD): zeta ||ubar_e|| V_e^(1/3) dt with ubar_e the
        volume average of the velocity over the cell."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        tau = np.zeros(self.spec.ncell)
        for e in range(self.spec.ncell):
            cq = self._cq(e)
            ubar = np.array([cq.mvec @ u[d, e] for d in range(3)]) / cq.volume
            tau[e] = zeta * np.linalg.norm(ubar) * cq.volume ** (1.0 / 3.0) * dt
        return tau

    def cell_matrix(self, e, tau_e):
        """The (3P x 3P) matrix of Eq. (div-div) on cell e: blockdiag(M) + tau_e B."""
        cq = self._cq(e)
        P = self.P
        A = np.zeros((3 * P, 3 * P))
        for d in range(3):
            A[d * P:(d + 1) * P, d * P:(d + 1) * P] += cq.M
            for f in range(3):
                A[d * P:(d + 1) * P, f * P:(f + 1) * P] += tau_e * cq.B[d, f]
        return A

    def projection_apply(self, u, tau):
        """y = (blockdiag(M) + tau_e B) u cell by cell."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        y = np.zeros_like(u)
        for e in range(self.spec.ncell):
            ye = self.cell_matrix(e, tau[e]) @ u[:, e, :].ravel()
            y[:, e, :] = ye.reshape(3, self.P)
        return y.ravel()

    def project(self, rhs, tau):
        """Solve the local problems of Eq. (div-div) cell by cell (dense solve)."""
        rhs = np.asarray(rhs, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        x = np.zeros_like(rhs)
        for e in range(self.spec.ncell):
            xe = np.linalg.solve(self.cell_matrix(e, tau[e]), rhs[:, e, :].ravel())
            x[:, e, :] = xe.reshape(3, self.P)
        return x.ravel()

    def divergence_l2(self, u):
        """sum over cells of ||div u||^2_e (the divergence error measure)."""
        u = np.asarray(u, dtype=np.float64).reshape(3, self.spec.ncell, self.P)
        s = 0.0
        for e in range(self.spec.ncell):
            cq = self._cq(e)
            ue = u[:, e, :].ravel()
            Bfull = np.block([[cq.B[d, f] for f in range(3)] for d in range(3)])
            s += ue @ Bfull @ ue
        return s
