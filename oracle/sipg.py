"""SIPG Laplacian / Helmholtz operator by dense quadrature (oracle; test infrastructure).

The bilinear form is the element-wise weak form of the pressure Poisson
equation (Sec. 3.2 (ii): the fluxes P* and Pi*, the penalty of Eq. (taue) and
the max rule of Eq. (tau)), summed over both sides of every face:

  a(u, v) = sum_K nu_K (grad u, grad v)_K
          - sum_{F interior} ( {{nu grad u}}.n [v] + {{nu grad v}}.n [u] - tau_F nu_F [u][v] )_F
          - sum_{F Dirichlet} nu_K ( grad u.n v + grad v.n u - 2 tau_K u v )_F
          + 0 on Neumann faces,

with [w] = w^- - w^+, {{w}} = (w^- + w^+)/2 and n = n^- (Sec. 3.1), tau_F =
max(tau^-, tau^+) on interior faces (Eq. (tau)).  "Dirichlet" is the face
where the unknown itself is prescribed (the pressure's partial Omega^N, the
velocity's partial Omega^D, Sec. 3.2 (ii)/(iii)); "Neumann" faces carry no
operator term.  For a constant viscosity nu this is nu times the SIPG
Laplacian; a per-cell nu_K uses the arithmetic average of nu grad u in the
consistency terms and nu_F = max(nu^-, nu^+) in the penalty (the paper has
only constant nu; this reading is stated in the design notes).

The viscous Helmholtz operator in Laplace form is (gamma0/dt) M + nu L
(Sec. 3.2 (iii), Sec. 4.4 Eq. (viscous)), with M the Gauss-quadrature mass
matrix.

Everything is built by DENSE quadrature: each basis function is evaluated at
each quadrature point (tensor product of 1D Lagrange values, the expansion of
Sec. 5), the full 3x3 Jacobian of the iso-parametric map is formed at every
point, normals and surface measures come from Nanson's formula
n dA = det(J) J^{-T} N dA_ref, and matrices are sums over points.  No sum
factorisation and no separability of the mapping is assumed.

Vector layout: x[comp, cell, i] with i = (c p + b) p + a, a along x.
"""
import numpy as np
import scipy.sparse as sp
from scipy.linalg import cho_factor, cho_solve

from .basis import gauss_rule, gll_rule, lagrange_derivatives, lagrange_values
from .mesh import DIRICHLET, NEUMANN, PERIODIC, cell_node_coords, neighbor

MINUS, PLUS = 0, 1
SIGMA = (1.0, -1.0)  # sign of each side inside the jump [w] = w^- - w^+


def _tensor_tables(zn, px, py, pz):
    """Values and reference gradients of all p^3 nodal basis functions at the
    tensor points px x py x pz (x fastest).  Returns phi (npts, p^3) and
    dphi (3, npts, p^3)."""
    vx, vy, vz = (lagrange_values(zn, t) for t in (px, py, pz))
    dx, dy, dz = (lagrange_derivatives(zn, t) for t in (px, py, pz))

    def prod(ax, ay, az):
        # T[qz, qy, qx, c, b, a] = az[qz, c] * ay[qy, b] * ax[qx, a]
        t = np.einsum("zc,yb,xa->zyxcba", az, ay, ax)
        n = t.shape[0] * t.shape[1] * t.shape[2]
        return t.reshape(n, -1)

    phi = prod(vx, vy, vz)
    dphi = np.stack([prod(dx, vy, vz), prod(vx, dy, vz), prod(vx, vy, dz)])
    return phi, dphi


class CellGeometry:
    """Everything the operator needs from one mapped cell (one geometry key)."""

    def __init__(self, op, xn):
        p, nq = op.p, op.nq
        # volume quadrature
        J = np.einsum("ik,dqi->qkd", xn, op.dphi_vol)  # J[q, k, d] = dx_k / dxi_d
        det = np.linalg.det(J)
        if np.any(det <= 0):
            raise ValueError("inverted or degenerate cell")
        Jinv = np.linalg.inv(J)  # Jinv[q, d, k] = dxi_d / dx_k
        grad = np.einsum("qdk,dqi->qik", Jinv, op.dphi_vol)
        wdet = op.w_vol * det
        self.volume = wdet.sum()
        self.K = np.einsum("q,qik,qjk->ij", wdet, grad, grad)
        self.M = np.einsum("q,qi,qj->ij", wdet, op.phi_vol, op.phi_vol)
        # faces (d, side): outward normal, surface weights, outward normal gradients
        self.face = {}
        self.area = np.zeros((3, 2))
        for d in range(3):
            for side in (0, 1):
                phi, dphi, wref = op.face_tables[(d, side)]
                Jf = np.einsum("ik,dqi->qkd", xn, dphi)
                detf = np.linalg.det(Jf)
                Jinvf = np.linalg.inv(Jf)
                a = detf[:, None] * Jinvf[:, d, :]  # det(J) J^{-T} e_d
                norm = np.linalg.norm(a, axis=1)
                n = (1.0 if side == 1 else -1.0) * a / norm[:, None]
                wA = wref * norm
                gradf = np.einsum("qdk,dqi->qik", Jinvf, dphi)
                G = np.einsum("qik,qk->qi", gradf, n)
                self.face[(d, side)] = (n, wA, phi, G)
                self.area[d, side] = wA.sum()


class SIPG:
    """Dense-quadrature SIPG operator on a structured mesh (oracle).

    ``penalty_factor`` multiplies tau of Eq. (taue); ``nq`` overrides the
    number of Gauss points per direction (default k+1, Sec. 5)."""

    def __init__(self, spec, k, penalty_factor=1.0, nq=None):
        if k < 1:
            raise ValueError("k >= 1")
        self.spec, self.k, self.p = spec, k, k + 1
        self.P = self.p ** 3
        self.nq = nq if nq is not None else k + 1
        self.penalty_factor = penalty_factor
        self.zn, _ = gll_rule(self.p)
        zq, wq = gauss_rule(self.nq)
        self.phi_vol, self.dphi_vol = _tensor_tables(self.zn, zq, zq, zq)
        self.w_vol = np.einsum("z,y,x->zyx", wq, wq, wq).ravel()
        self.face_tables = {}
        for d in range(3):
            for side in (0, 1):
                pts = [zq, zq, zq]
                pts[d] = np.array([float(side)])
                phi, dphi = _tensor_tables(self.zn, *pts)
                ws = [wq, wq, wq]
                ws[d] = np.array([1.0])
                wref = np.einsum("z,y,x->zyx", ws[2], ws[1], ws[0]).ravel()
                self.face_tables[(d, side)] = (phi, dphi, wref)
        self._prepare()

    # ------------------------------------------------------------------ mesh
    def _prepare(self):
        spec, p = self.spec, self.p
        ncell = spec.ncell
        lmax = max(h - l for h, l in zip(spec.hi, spec.lo))
        key_rows = []
        chunk = 8192
        for c0 in range(0, ncell, chunk):
            cells = np.arange(c0, min(ncell, c0 + chunk))
            xn = cell_node_coords(spec, p, cells)
            rel = (xn - xn[:, :1, :]) / lmax
            key_rows.append(np.round(rel * 1e10).astype(np.int64).reshape(len(cells), -1))
        keys = np.concatenate(key_rows)
        ukeys, first, inv = np.unique(keys, axis=0, return_index=True, return_inverse=True)
        self.cell_key = inv.ravel()
        self.geom = [CellGeometry(self, cell_node_coords(spec, p, [c])[0]) for c in first]
        cells = np.arange(ncell)
        # face classification and penalty (Eq. (taue) and Eq. (tau))
        self.nb = np.zeros((3, 2, ncell), dtype=np.int64)
        self.bkind = {}
        interior = np.zeros((3, 2, ncell), dtype=bool)
        for d in range(3):
            for side in (0, 1):
                nb, on_b, bc = neighbor(spec, cells, d, side)
                self.nb[d, side] = nb
                interior[d, side] = ~on_b
                self.bkind[(d, side)] = bc
        areas = np.stack([g.area for g in self.geom])[self.cell_key]  # (ncell, 3, 2)
        vol = np.array([g.volume for g in self.geom])[self.cell_key]
        a_int = np.where(interior.transpose(2, 0, 1), areas, 0.0).sum(axis=(1, 2))
        a_bdy = np.where(~interior.transpose(2, 0, 1), areas, 0.0).sum(axis=(1, 2))
        self.tau = self.penalty_factor * (self.k + 1) ** 2 * (0.5 * a_int + a_bdy) / vol
        self.interior = interior
        # interior faces per direction: (e^-, e^+) = (cell, its +side neighbour)
        self.faces = []
        self._face_pieces = {}
        for d in range(3):
            em = cells[interior[d, 1]]
            ep = self.nb[d, 1][interior[d, 1]]
            pair = np.stack([self.cell_key[em], self.cell_key[ep]], axis=1)
            if len(pair):
                up, finv = np.unique(pair, axis=0, return_inverse=True)
            else:
                up, finv = np.zeros((0, 2), dtype=np.int64), np.zeros(0, dtype=np.int64)
            finv = finv.ravel()
            for gi, (km, kp) in enumerate(up):
                sel = finv == gi
                self.faces.append((d, int(km), int(kp), em[sel], ep[sel]))
        # boundary faces with an operator term (Dirichlet only)
        self.bfaces = []
        for d in range(3):
            for side in (0, 1):
                bc = self.bkind[(d, side)]
                if bc == PERIODIC:
                    continue
                bcells = cells[~interior[d, side]]
                if bc == DIRICHLET:
                    self.bfaces.append((d, side, bcells))
                elif bc != NEUMANN:
                    raise ValueError("unknown boundary condition " + bc)

    def face_pieces(self, d, km, kp):
        """Geometric pieces of an interior face between e^- (key km, its +d face)
        and e^+ (key kp, its -d face).  For sides t (test) and s (trial):
          cu[t][s][i, j] = -1/2 sum_q wA G^s_j sigma_t phi^t_i    (scaled by nu_s)
          cv[t][s]       = cu[s][t]^T                               (scaled by nu_t)
          pen[t][s][i,j] = sigma_s sigma_t sum_q wA phi^s_j phi^t_i (scaled by tau_F nu_F)
        G^s is the gradient of side s along n = n^-."""
        key = (d, km, kp)
        if key in self._face_pieces:
            return self._face_pieces[key]
        nm, wAm, phim, Gm = self.geom[km].face[(d, 1)]
        np_, wAp, phip, Gp = self.geom[kp].face[(d, 0)]
        if not (np.allclose(nm, -np_, atol=1e-10) and np.allclose(wAm, wAp, rtol=1e-10)):
            raise ValueError("non-conforming face")
        wA = wAm
        phi = (phim, phip)
        G = (Gm, -Gp)  # both along n^-
        cu = [[None, None], [None, None]]
        pen = [[None, None], [None, None]]
        for t in (MINUS, PLUS):
            for s in (MINUS, PLUS):
                cu[t][s] = -0.5 * SIGMA[t] * np.einsum("q,qj,qi->ij", wA, G[s], phi[t])
                pen[t][s] = SIGMA[s] * SIGMA[t] * np.einsum("q,qj,qi->ij", wA, phi[s], phi[t])
        cv = [[cu[s][t].T for s in (MINUS, PLUS)] for t in (MINUS, PLUS)]
        out = (cu, cv, pen)
        self._face_pieces[key] = out
        return out

    def boundary_pieces(self, kc, d, side):
        """Dirichlet face of one cell: bcons[i, j] = -sum wA G_j phi_i, bpen = sum wA phi_j phi_i."""
        n, wA, phi, G = self.geom[kc].face[(d, side)]
        bcons = -np.einsum("q,qj,qi->ij", wA, G, phi)
        bpen = np.einsum("q,qj,qi->ij", wA, phi, phi)
        return bcons, bpen

    # ------------------------------------------------------------- operators
    def _nu(self, nu, nu_cell):
        if nu_cell is not None:
            nu_cell = np.asarray(nu_cell, dtype=np.float64)
            if nu_cell.shape != (self.spec.ncell,):
                raise ValueError("nu_cell must have one value per cell")
            return nu_cell
        return np.full(self.spec.ncell, float(nu))

    def blocks(self, mass_coef=0.0, nu=1.0, nu_cell=None, stiffness=True, targets=None):
        """Yield (tgt_cells, src_cells, B) with B (n, P, P): y[tgt] += B @ x[src].

        This is the operator as a list of element-coupling blocks; ``apply`` and
        ``assemble`` both consume it.  ``targets`` (bool mask over cells) keeps
        only the blocks whose rows belong to those cells."""
        nue = self._nu(nu, nu_cell)
        keep = (lambda c: targets[c]) if targets is not None else (lambda c: np.ones(len(c), dtype=bool))
        for kc in range(len(self.geom)):
            cells = np.nonzero(self.cell_key == kc)[0]
            cells = cells[keep(cells)]
            if len(cells) == 0:
                continue
            g = self.geom[kc]
            B = mass_coef * g.M[None] + (nue[cells, None, None] * g.K[None] if stiffness else 0.0)
            yield cells, cells, np.broadcast_to(B, (len(cells), self.P, self.P))
        if not stiffness:
            return
        for d, km, kp, em, ep in self.faces:
            cu, cv, pen = self.face_pieces(d, km, kp)
            tauF = np.maximum(self.tau[em], self.tau[ep])
            nuF = np.maximum(nue[em], nue[ep])
            side_cells = (em, ep)
            for t in (MINUS, PLUS):
                sel = keep(side_cells[t])
                if not sel.any():
                    continue
                for s in (MINUS, PLUS):
                    tgt, src = side_cells[t][sel], side_cells[s][sel]
                    B = (nue[src, None, None] * cu[t][s][None] + nue[tgt, None, None] * cv[t][s][None]
                         + (tauF[sel] * nuF[sel])[:, None, None] * pen[t][s][None])
                    yield tgt, src, B
        for d, side, bcells in self.bfaces:
            bcells = bcells[keep(bcells)]
            for kc in np.unique(self.cell_key[bcells]):
                cells = bcells[self.cell_key[bcells] == kc]
                bcons, bpen = self.boundary_pieces(kc, d, side)
                B = nue[cells, None, None] * ((bcons + bcons.T)[None]
                                              + 2.0 * self.tau[cells, None, None] * bpen[None])
                yield cells, cells, B

    def apply(self, x, mass_coef=0.0, nu=1.0, nu_cell=None, stiffness=True, targets=None):
        """y = A x element by element; x has shape (ncomp, N) or (N,).

        ``targets`` (bool mask over cells) restricts the output to those cells
        (other rows are returned as zero)."""
        x = np.asarray(x, dtype=np.float64)
        flat = x.ndim == 1
        X = x.reshape(-1, self.spec.ncell, self.P)
        Y = np.zeros_like(X)
        for tgt, src, B in self.blocks(mass_coef, nu, nu_cell, stiffness, targets):
            Y[:, tgt] += np.einsum("nij,cnj->cni", B, X[:, src])
        return Y.reshape(x.shape) if not flat else Y.ravel()

    def assemble(self, mass_coef=0.0, nu=1.0, nu_cell=None, stiffness=True):
        """Global sparse matrix (CSR) of the operator (small meshes)."""
        P = self.P
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
        for tgt, src, B in self.blocks(mass_coef, nu, nu_cell, stiffness):
            rows.append((tgt[:, None, None] * P + ii[None]).ravel())
            cols.append((src[:, None, None] * P + jj[None]).ravel())
            vals.append(np.asarray(B).ravel())
        n = self.spec.ncell * P
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
        return A.tocsr()

    def diagonal(self, mass_coef=0.0, nu=1.0, nu_cell=None):
        """diag(A) from the self-coupling blocks (Sec. 5.1: the matrix diagonal used by
        Jacobi and Chebyshev)."""
        D = np.zeros((self.spec.ncell, self.P))
        for tgt, src, B in self.blocks(mass_coef, nu, nu_cell):
            self_mask = tgt == src
            if self_mask.any():
                D[tgt[self_mask]] += np.einsum("nii->ni", B[self_mask])
        return D.ravel()

    def norm_inf(self, mass_coef=0.0, nu=1.0, nu_cell=None, stiffness=True, targets=None):
        """max_i sum_j |A_ij| (over the rows of ``targets`` when given)."""
        rows = np.zeros((self.spec.ncell, self.P))
        for tgt, src, B in self.blocks(mass_coef, nu, nu_cell, stiffness, targets):
            rows[tgt] += np.abs(B).sum(axis=2)
        return float(rows.max())

    def mass_apply(self, x):
        return self.apply(x, mass_coef=1.0, stiffness=False)

    def inverse_mass_apply(self, x):
        """M^-1 x by a dense Cholesky factorisation of every element mass matrix.

        Sec. 5 inverts the block-diagonal mass matrix cell by cell; with n_q = k+1
        the tensorial form used by the fast kernels is the same matrix."""
        x = np.asarray(x, dtype=np.float64)
        X = x.reshape(-1, self.spec.ncell, self.P)
        Y = np.empty_like(X)
        for kc, g in enumerate(self.geom):
            cells = np.nonzero(self.cell_key == kc)[0]
            if len(cells) == 0:
                continue
            f = cho_factor(g.M)
            rhs = X[:, cells].reshape(-1, self.P).T
            Y[:, cells] = cho_solve(f, rhs).T.reshape(X.shape[0], len(cells), self.P)
        return Y.reshape(x.shape)

    # ---------------------------------------------------------- geometry out
    def node_coordinates(self):
        """Physical coordinates (ncell, p^3, 3) of the nodal (GLL) points."""
        return cell_node_coords(self.spec, self.p, np.arange(self.spec.ncell))

    def quadrature_points(self, nq):
        """Mapped Gauss points and weights det(J) w of an nq-point rule, per cell,
        through the iso-parametric map (for error norms and load vectors)."""
        zq, wq = gauss_rule(nq)
        phi, dphi = _tensor_tables(self.zn, zq, zq, zq)
        w = np.einsum("z,y,x->zyx", wq, wq, wq).ravel()
        xn = self.node_coordinates()
        xq = np.einsum("qi,eik->eqk", phi, xn)
        J = np.einsum("eik,dqi->eqkd", xn, dphi)
        return xq, w[None, :] * np.linalg.det(J), phi

    def load_vector(self, f, nq=None):
        """b_i = int f phi_i by an nq-point Gauss rule (default k+3) on the mapped cells."""
        nq = nq or self.k + 3
        xq, wdet, phi = self.quadrature_points(nq)
        fq = f(xq[..., 0], xq[..., 1], xq[..., 2])
        return np.einsum("eq,qi->ei", wdet * fq, phi).ravel()

    def l2_error(self, u, exact, nq=None):
        """|| u_h - u ||_L2 with an nq-point rule (default k+3)."""
        nq = nq or self.k + 3
        xq, wdet, phi = self.quadrature_points(nq)
        uh = np.einsum("qi,ei->eq", phi, np.asarray(u).reshape(self.spec.ncell, self.P))
        e = uh - exact(xq[..., 0], xq[..., 1], xq[..., 2])
        return float(np.sqrt(np.sum(wdet * e * e)))
