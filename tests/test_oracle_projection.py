"""Pins of the oracle's pressure-projection operators (variant V3c): the
divergence of Eq. (av3), the gradient of Eq. (bv3) and the div-div penalised
local projection of Eq. (div-div) with tau_D of Eq. (tauD).

Each pin is fixed by the mathematics: integration by parts on continuous
polynomial fields (where jumps vanish and Gauss quadrature is exact), the
discrete adjointness of the two central-flux forms on a periodic mesh, the
closed form of tau_D for a uniform velocity, and invariants of the local
projection (identity without penalty, divergence-free fields untouched,
monotone decrease of the divergence)."""
import math

import numpy as np
import pytest

from oracle.mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec
from oracle.projection import ProjectionOps

P_, D_, N_ = PERIODIC, DIRICHLET, NEUMANN


def box(n, bc=D_, mapping="affine"):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(1.5, 1.0, 1.0), bc_lo=(bc,) * 3, bc_hi=(bc,) * 3,
                    mapping=mapping)


def channel(n):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi), bc_lo=(P_, D_, P_),
                    bc_hi=(P_, D_, P_), mapping="channel", gamma=1.8)


@pytest.mark.parametrize("k", [2, 3])
def test_divergence_of_polynomial_field(k):
    """Continuous u of degree k per direction: the jumps vanish, the boundary
    flux is the own trace, and integrating by parts cell by cell gives
    a(q, u) = -(q, div u) exactly (Gauss k+1 is exact on affine cells)."""
    ops = ProjectionOps(box((2, 2, 3)), k)
    x, y, z = ops.sipg.node_coordinates().reshape(-1, 3).T
    if k == 2:
        u = np.stack([x * x * y + z, y * y - x * z, x * y * z * z])
        div = 2 * x * y + 2 * y + 2 * x * y * z
    else:
        u = np.stack([x ** 2 * y + z ** 3, y ** 3 - x * z, x * y * z ** 2])
        div = 2 * x * y + 3 * y ** 2 + 2 * x * y * z
    got = ops.divergence(u.ravel())
    want = -ops.mass(div, 1)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("k", [2, 3])
def test_gradient_of_polynomial_field(k):
    """Continuous p: b(v, p) = -(v, grad p) exactly."""
    ops = ProjectionOps(box((3, 2, 2)), k)
    x, y, z = ops.sipg.node_coordinates().reshape(-1, 3).T
    p = x ** k * y - y ** 2 * z + z ** k
    grad = np.stack([k * x ** (k - 1) * y, x ** k - 2 * y * z, -y ** 2 + k * z ** (k - 1)])
    got = ops.gradient(p)
    want = -ops.mass(grad.ravel(), 3)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("spec", [box((2, 3, 2), bc=P_), channel((2, 4, 2))], ids=["periodic_box", "channel"])
def test_divergence_gradient_adjoint_on_periodic_faces(spec):
    """With central fluxes on every interior/periodic face the two forms are
    discrete negative adjoints: sum_e a(phi_i, phi_j e_d) = -sum_e b(phi_j e_d, phi_i).
    On the channel (walls with the own-trace flux) the relation holds for
    every pair not touching a wall face."""
    ops = ProjectionOps(spec, 2)
    nu, npp = 3 * spec.ncell * ops.P, spec.ncell * ops.P
    D = np.stack([ops.divergence(e) for e in np.eye(nu)], axis=1)
    G = np.stack([ops.gradient(e) for e in np.eye(npp)], axis=1)
    S = D + G.T
    if spec.bc_lo[1] == P_:
        assert np.abs(S).max() <= 1e-13 * np.abs(D).max()
    else:
        # only entries coupling nodes on a wall face may differ
        y = ops.sipg.node_coordinates().reshape(-1, 3)[:, 1]
        wall = np.isclose(np.abs(y), 1.0)
        rows = np.nonzero(np.abs(S).max(axis=1) > 1e-13 * np.abs(D).max())[0]
        assert rows.size and wall[rows].all()
        assert np.abs(S[~wall]).max() <= 1e-13 * np.abs(D).max()


def test_tau_div_closed_form():
    """Uniform velocity U on affine cells: tau_D = zeta |U| V^(1/3) dt."""
    spec = box((2, 2, 2))
    ops = ProjectionOps(spec, 2)
    U = np.array([0.3, -1.2, 0.4])
    u = np.repeat(U[:, None], spec.ncell * ops.P, axis=1)
    tau = ops.tau_div(u.ravel(), zeta=2.0, dt=1e-3)
    vol = (1.5 / 2) * (2.0 / 2) * (1.0 / 2)
    assert np.allclose(tau, 2.0 * np.linalg.norm(U) * vol ** (1 / 3) * 1e-3, rtol=1e-13)


def test_projection_invariants():
    ops = ProjectionOps(channel((2, 4, 2)), 3)
    ncell, P = ops.spec.ncell, ops.P
    rng = np.random.default_rng(4)
    uh = rng.standard_normal(3 * ncell * P)
    rhs = ops.mass(uh, 3)
    # no penalty: the L2 projection of u onto itself
    assert np.allclose(ops.project(rhs, np.zeros(ncell)), uh, rtol=0, atol=1e-11)
    # the local matrices are symmetric positive definite
    A = ops.cell_matrix(3, 0.7)
    assert np.allclose(A, A.T, atol=1e-14 * np.abs(A).max()) and np.linalg.eigvalsh(A).min() > 0
    # divergence error decreases monotonically with the penalty
    errs = [ops.divergence_l2(ops.project(rhs, np.full(ncell, t))) for t in (0.0, 0.1, 1.0, 10.0)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_projection_keeps_divergence_free_field():
    """A divergence-free polynomial field solves the penalised problem for any
    tau_D: its div-div term vanishes cell by cell."""
    ops = ProjectionOps(box((2, 2, 2)), 3)
    x, y, z = ops.sipg.node_coordinates().reshape(-1, 3).T
    u = np.stack([y * z * z, x * z + z ** 3, x * x * y]).ravel()  # div u = 0
    tau = np.linspace(0.5, 5.0, ops.spec.ncell)
    assert np.allclose(ops.project(ops.mass(u, 3), tau), u, rtol=0, atol=1e-11)
    assert abs(ops.divergence_l2(u)) <= 1e-12  # rounding of a sum of O(1) terms
