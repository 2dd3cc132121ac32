"""Viscous operator in divergence form (oracle; test infrastructure).

Sec. 3.2 (iii): the implicit viscous step with the symmetric interior penalty
(s = 1), the numerical fluxes U* and F^nu* and homogeneous boundary data.
With F^nu(u) = 2 nu eps(u), eps(u) = (grad u + grad u^T) / 2 and the fluxes
  U*        = {{u}} on interior faces, 0 on Dirichlet faces, u on Neumann faces,
  F^nu*.n   = {{2 nu eps(u)}} n - tau nu [u]  (interior),
              2 nu eps(u) n - 2 tau nu u      (Dirichlet), 0 (Neumann),
the element-wise form summed over both sides of every face reads
  a(v, u) = sum_e (eps(v), 2 nu eps(u))_e
          - sum_F int_F ( {{2 nu eps(u)}} n . [v] + {{2 nu eps(v)}} n . [u] - tau_F nu [u] . [v] )
          - sum_{F Dirichlet} int_F ( 2 nu eps(u) n . v + 2 nu eps(v) n . u - 2 tau_e nu u . v ),
with [w] = w^- - w^+, n = n^- and tau of Eq. (taue) / Eq. (tau).  The viscous
Helmholtz operator of the step is (gamma0/dt) M + a (Eq. (viscous) with the
paper's F^nu).

Dense quadrature with the full Jacobian at every Gauss point, as in
``sipg.SIPG`` (whose geometry keys, neighbours and penalties are reused); the
operator is assembled as a sparse matrix (small meshes only).

Layout: u[d, cell, i] (d = x, y, z component), i = (c p + b) p + a.
"""
import numpy as np
import scipy.sparse as sp

from .mesh import DIRICHLET, NEUMANN, PERIODIC, cell_node_coords
from .sipg import SIPG


class _Quad:
    """Values, full gradients, normals and weights of one mapped cell."""

    def __init__(self, op, xn):
        J = np.einsum("ik,dqi->qkd", xn, op.dphi_vol)
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        self.grad = np.einsum("qdk,dqi->qik", Jinv, op.dphi_vol)  # (q, basis, k)
        self.wdet = op.w_vol * det
        self.face = {}
        for d in range(3):
            for side in (0, 1):
                phif, dphif, wref = op.face_tables[(d, side)]
                Jf = np.einsum("ik,dqi->qkd", xn, dphif)
                detf = np.linalg.det(Jf)
                Jinvf = np.linalg.inv(Jf)
                a = detf[:, None] * Jinvf[:, d, :]
                norm = np.linalg.norm(a, axis=1)
                n = (1.0 if side == 1 else -1.0) * a / norm[:, None]
                gradf = np.einsum("qdk,dqi->qik", Jinvf, dphif)
                self.face[(d, side)] = (n, wref * norm, phif, gradf)


def _traction(grad, n):
    """T[q, (j, b), m] = (2 eps(phi_b e_j) n)_m = delta_mj grad phi_b . n + n_j d_m phi_b."""
    nq, P, _ = grad.shape
    gn = np.einsum("qbk,qk->qb", grad, n)
    T = np.zeros((nq, 3, P, 3))
    for j in range(3):
        T[:, j, :, j] += gn
        T[:, j, :, :] += n[:, j][:, None, None] * grad
    return T.reshape(nq, 3 * P, 3)


def _values(phi):
    """V[q, (j, b), m] = (phi_b e_j)_m."""
    nq, P = phi.shape
    V = np.zeros((nq, 3, P, 3))
    for j in range(3):
        V[:, j, :, j] = phi
    return V.reshape(nq, 3 * P, 3)


class ViscousOp:
    """(mass_coef) M + a(., .) of the divergence-form viscous operator."""

    def __init__(self, spec, k, penalty_factor=1.0):
        self.sipg = SIPG(spec, k, penalty_factor)
        self.spec, self.k, self.P = spec, k, (k + 1) ** 3
        first = {}
        for c, key in enumerate(self.sipg.cell_key):
            first.setdefault(int(key), c)
        self.q = [_Quad(self.sipg, cell_node_coords(spec, k + 1, [first[kk]])[0]) for kk in range(len(first))]

    def _cq(self, e):
        return self.q[self.sipg.cell_key[e]]

    def _gidx(self, e):
        """Global indices of the 3P unknowns of cell e, ordered (component, basis)."""
        N = self.spec.ncell * self.P
        return (np.arange(3)[:, None] * N + e * self.P + np.arange(self.P)[None, :]).ravel()

    def assemble(self, nu=1.0, mass_coef=0.0):
        spec, P = self.spec, self.P
        nd = 3 * spec.ncell * P
        rows, cols, vals = [], [], []

        def add(ri, ci, B):
            rr, cc = np.meshgrid(ri, ci, indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(B.ravel())

        tau = self.sipg.tau
        for e in range(spec.ncell):
            cq = self._cq(e)
            g = cq.grad
            # cell: nu (grad v : grad u + grad v : grad u^T) and the mass
            lap = np.einsum("q,qak,qbk->ab", cq.wdet, g, g, optimize=True)
            B = np.zeros((3, P, 3, P))
            for i in range(3):
                B[i, :, i, :] += nu * lap
                for j in range(3):
                    B[i, :, j, :] += nu * np.einsum("q,qa,qb->ab", cq.wdet, g[:, :, j], g[:, :, i], optimize=True)
            if mass_coef:
                phi = self.sipg.phi_vol
                Mloc = np.einsum("q,qa,qb->ab", cq.wdet, phi, phi, optimize=True)
                for i in range(3):
                    B[i, :, i, :] += mass_coef * Mloc
            add(self._gidx(e), self._gidx(e), B.reshape(3 * P, 3 * P))
            # faces
            for d in range(3):
                for side in (0, 1):
                    n, wA, phif, gradf = cq.face[(d, side)]
                    if self.sipg.interior[d, side, e]:
                        if side == 0:
                            continue  # each interior face once, from its low (e^-) cell... see below
                        nb = self.sipg.nb[d, 1, e]
                        _, _, phip, gradp = self._cq(nb).face[(d, 0)]
                        tauF = max(tau[e], tau[nb])
                        Vs = (_values(phif), _values(phip))
                        Ts = (_traction(gradf, n), _traction(gradp, n))  # both along n = n^-
                        sig = (1.0, -1.0)
                        idx = (self._gidx(e), self._gidx(nb))
                        for t in (0, 1):
                            for s in (0, 1):
                                # - {{2 eps(u)}} n . [v] - {{2 eps(v)}} n . [u] + tau [u].[v]
                                Bf = -0.5 * sig[t] * np.einsum("q,qam,qbm->ab", wA, Vs[t], Ts[s], optimize=True)
                                Bf += -0.5 * sig[s] * np.einsum("q,qam,qbm->ab", wA, Ts[t], Vs[s], optimize=True)
                                Bf *= nu
                                Bf += tauF * nu * sig[t] * sig[s] * np.einsum("q,qam,qbm->ab", wA, Vs[t], Vs[s], optimize=True)
                                add(idx[t], idx[s], Bf)
                    elif self.sipg.bkind[(d, side)] == DIRICHLET:
                        V = _values(phif)
                        T = _traction(gradf, n)
                        Bf = -nu * (np.einsum("q,qam,qbm->ab", wA, V, T, optimize=True) + np.einsum("q,qam,qbm->ab", wA, T, V, optimize=True))
                        Bf += 2.0 * tau[e] * nu * np.einsum("q,qam,qbm->ab", wA, V, V, optimize=True)
                        add(self._gidx(e), self._gidx(e), Bf)
                    elif self.sipg.bkind[(d, side)] not in (NEUMANN, PERIODIC):
                        raise ValueError("unknown boundary condition")
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(nd, nd)).tocsr()
