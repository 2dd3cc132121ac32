"""Pins of the oracle's convective term (Eq. (convstepspat), local
Lax-Friedrichs flux, over-integration with floor(3k/2)+1 Gauss points)."""
import numpy as np
import pytest

from oracle.basis import gll_rule
from oracle.convective import ConvectiveOp, over_integration_points
from oracle.mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec

P_, D_, N_ = PERIODIC, DIRICHLET, NEUMANN


def test_over_integration_rule():
    assert [over_integration_points(k) for k in (1, 2, 3, 4, 5)] == [2, 4, 5, 7, 8]


def test_constant_field_on_periodic_mesh():
    """div(c (x) c) = 0 and no jumps: the term vanishes."""
    spec = MeshSpec(2, 3, 2, hi=(1.0, 1.5, 0.8), mapping="affine")
    op = ConvectiveOp(spec, 2)
    N = spec.ncell * op.P
    u = np.concatenate([np.full(N, 0.7), np.full(N, -1.3), np.full(N, 0.4)])
    y = op.apply(u)
    assert np.abs(y).max() <= 1e-13


@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_consistency_neumann(k):
    """Continuous u in Q_k, Neumann faces everywhere (own-trace flux): the
    form equals -(v, div(u (x) u)) exactly; the right side is evaluated here by
    an independent 2k+2-point Gauss rule of the analytic divergence."""
    spec = MeshSpec(2, 2, 2, lo=(0.0, -1.0, 0.0), hi=(1.5, 1.0, 1.2), bc_lo=(N_,) * 3, bc_hi=(N_,) * 3)
    op = ConvectiveOp(spec, k)
    X = op.sipg.node_coordinates().reshape(-1, 3)

    def vel(x, y, z):
        return np.stack([x * y + z ** k, y ** 2 - x * z, x ** 2 * z + y])

    def div_uu(x, y, z):
        u = vel(x, y, z)
        # d/dx_j (u_i u_j) = u_j d_j u_i + u_i div u
        gu = np.zeros((3, 3) + x.shape)  # gu[i, j] = d_j u_i
        gu[0, 0], gu[0, 1], gu[0, 2] = y, x, k * z ** (k - 1)
        gu[1, 0], gu[1, 1], gu[1, 2] = -z, 2 * y, -x
        gu[2, 0], gu[2, 1], gu[2, 2] = 2 * x * z, 1.0 + 0 * x, x ** 2
        div = gu[0, 0] + gu[1, 1] + gu[2, 2]
        return np.einsum("j...,ij...->i...", u, gu) + u * div

    u = vel(X[:, 0], X[:, 1], X[:, 2])
    y = op.apply(u.ravel())
    from oracle.sipg import SIPG
    ref = SIPG(spec, k)
    nq = 2 * k + 2
    want = -np.concatenate([ref.load_vector(lambda x, yy, z, i=i: div_uu(x, yy, z)[i], nq=nq) for i in range(3)])
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_piecewise_constant_llf_flux_closed_form():
    """Piecewise-constant velocities on an affine periodic row of cells: the
    cell term equals the own-trace face flux, so each face leaves
    -int_F phi (s {{u_i u_d}} + Lambda/2 (u_i - u_nb,i) - s u_i u_d); the face
    integral of the nodal basis is the product of GLL weights times the face
    extents (exact: degree k per direction)."""
    k = 2
    spec = MeshSpec(3, 1, 1, hi=(3.0, 0.5, 0.8))
    op = ConvectiveOp(spec, k)
    P = op.P
    c = np.array([[1.0, 0.2, -0.3], [-0.5, 0.4, 0.1], [0.3, -0.7, 0.6]])  # cell velocities
    u = np.concatenate([np.repeat(c[:, i], P) for i in range(3)])
    y = op.apply(u).reshape(3, 3, P)
    _, wg = gll_rule(k + 1)  # weights on [0, 1]
    hx, hy, hz = 1.0, 0.5, 0.8
    want = np.zeros((3, 3, P))
    for e in range(3):
        for side, s in ((0, -1.0), (1, 1.0)):
            nb = (e + (1 if side else -1)) % 3
            un, unb = s * c[e, 0], s * c[nb, 0]
            lam = max(2 * abs(un), 2 * abs(unb))
            a_end = k if side else 0
            for i in range(3):
                flux = 0.5 * (c[e, i] * un + c[nb, i] * unb) + 0.5 * lam * (c[e, i] - c[nb, i])
                own = c[e, i] * un  # the cell term, integrated by parts
                for cc in range(k + 1):
                    for bb in range(k + 1):
                        idx = (cc * (k + 1) + bb) * (k + 1) + a_end
                        want[i, e, idx] += (own - flux) * wg[bb] * hy * wg[cc] * hz
        # y- and z-faces: periodic with the same cell on both sides: own flux only, cancels
    assert np.abs(y - want).max() <= 1e-13 * np.abs(want).max()


def test_dirichlet_wall_flux():
    """On a no-slip wall with u . n != 0 the flux adds Lambda u^- (Lambda = 2|u.n|)
    to the own-trace flux: a constant field in a closed box then gives
    -int_F phi (Lambda u_i) on every wall face."""
    k = 1
    spec = MeshSpec(1, 1, 1, hi=(1.0, 1.0, 1.0), bc_lo=(D_,) * 3, bc_hi=(D_,) * 3)
    op = ConvectiveOp(spec, k)
    cvec = np.array([0.5, -1.0, 0.25])
    u = np.concatenate([np.full(op.P, cvec[i]) for i in range(3)])
    y = op.apply(u).reshape(3, op.P)
    _, wg = gll_rule(k + 1)
    want = np.zeros((3, op.P))
    for d in range(3):
        for side, s in ((0, -1.0), (1, 1.0)):
            lam = 2 * abs(s * cvec[d])
            for node in range(op.P):
                a = [node % 2, (node // 2) % 2, node // 4]
                if a[d] != (1 if side else 0):
                    continue
                t = [a[j] for j in range(3) if j != d]
                want[:, node] -= lam * cvec * wg[t[0]] * wg[t[1]]
    assert np.abs(y - want).max() <= 1e-13 * np.abs(want).max()
