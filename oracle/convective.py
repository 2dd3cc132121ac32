"""Convective term of the explicit convective step with the local
Lax-Friedrichs flux (oracle; test infrastructure).

Eq. (convstepspat): for a velocity test function v,
    c(v, u) = (grad v, u (x) u)_e - (v, F^c*(u) n)_de,
with F^c(u) = u (x) u and
    F^c* n = {{u (x) u}} n + Lambda/2 (u^- - u^+)          on interior faces,
           = (u^- (x) u^-) n                               on Neumann faces,
           = 1/2 (F(2 g - u^-) + F(u^-)) n + Lambda (u^- - g) on Dirichlet faces,
Lambda = max(lambda^-, lambda^+), lambda = 2 |u . n| at every quadrature point
(on a Dirichlet face lambda^+ = 2 |(2 g - u^-) . n|).  Homogeneous wall data
g = 0 here (no-slip walls of the channel).  Cell and face integrals use Gauss
quadrature with floor(3k/2) + 1 points per direction (Sec. 5: exact on
affine cells, no aliasing).

Dense quadrature with the full Jacobian, as in ``sipg.SIPG`` (constructed
with the over-integration rule so that its tables, geometry keys and
neighbours are reused).  Layout: u[d, cell, i], i = (c p + b) p + a.
"""
import numpy as np

from .mesh import DIRICHLET, NEUMANN, PERIODIC, cell_node_coords
from .sipg import SIPG
from .viscous import _Quad


def over_integration_points(k):
    """floor(3k/2) + 1 Gauss points per direction (Sec. 5)."""
    return (3 * k) // 2 + 1


class ConvectiveOp:
    def __init__(self, spec, k, nq=None):
        self.nq = nq if nq is not None else over_integration_points(k)
        self.sipg = SIPG(spec, k, nq=self.nq)
        self.spec, self.k, self.P = spec, k, (k + 1) ** 3
        first = {}
        for c, key in enumerate(self.sipg.cell_key):
            first.setdefault(int(key), c)
        self.q = [_Quad(self.sipg, cell_node_coords(spec, k + 1, [first[kk]])[0]) for kk in range(len(first))]

    def _cq(self, e):
        return self.q[self.sipg.cell_key[e]]

    def apply(self, u, cells=None):
        """y[i, e, a] = c(phi_a e_i, u) for every cell e (or only the cells
        listed in ``cells``; the other entries stay zero)."""
        spec, P = self.spec, self.P
        u = np.asarray(u, dtype=np.float64).reshape(3, spec.ncell, P)
        y = np.zeros_like(u)
        phi = self.sipg.phi_vol
        for e in (range(spec.ncell) if cells is None else cells):
            cq = self._cq(e)
            uq = phi @ u[:, e, :].T  # (q, 3)
            F = uq[:, :, None] * uq[:, None, :]  # F[q, i, k] = u_i u_k
            # (grad phi_a, u_i u) = sum_q wdet sum_k d_k phi_a u_i u_k
            y[:, e, :] += np.einsum("q,qak,qik->ia", cq.wdet, cq.grad, F)
            for d in range(3):
                for side in (0, 1):
                    n, wA, phif, _ = cq.face[(d, side)]
                    um = phif @ u[:, e, :].T  # (q, 3)
                    unm = np.einsum("qk,qk->q", um, n)
                    interior = self.sipg.interior[d, side, e]
                    if interior:
                        nb = self.sipg.nb[d, side, e]
                        _, _, phin, _ = self._cq(nb).face[(d, 1 - side)]
                        up = phin @ u[:, nb, :].T
                        unp = np.einsum("qk,qk->q", up, n)
                        lam = np.maximum(2 * np.abs(unm), 2 * np.abs(unp))
                        flux = 0.5 * (um * unm[:, None] + up * unp[:, None]) + 0.5 * lam[:, None] * (um - up)
                    else:
                        bc = self.sipg.bkind[(d, side)]
                        if bc == NEUMANN:
                            flux = um * unm[:, None]
                        elif bc == DIRICHLET:
                            lam = 2 * np.abs(unm)  # lambda^+ = 2 |(2g - u^-) . n| = lambda^- for g = 0
                            flux = um * unm[:, None] + lam[:, None] * um
                        else:
                            raise ValueError("unknown boundary condition")
                    y[:, e, :] -= np.einsum("q,qa,qi->ia", wA, phif, flux)
        return y.ravel()
