"""Pins of the oracle on the perturbed (general, non-separable) map: the map
itself (zero displacement on the box boundary, non-separability, the affine
limit), and the SIPG form on it (symmetry, constant null space with periodic
sides, positive definiteness with Dirichlet sides, optimal L2 convergence of a
manufactured solution: a wrong metric term fails the rate)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.mesh import DIRICHLET, PERIODIC, MeshSpec, analytic_map, perturbation_coefficients
from oracle.sipg import SIPG

P_, D_ = PERIODIC, DIRICHLET


def _spec(n, bc=P_, amp=0.06, seed=0x1234_5678_9ABC):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5), bc_lo=(bc,) * 3, bc_hi=(bc,) * 3,
                    mapping="perturbed", amplitude=amp, seed=seed)


def test_perturbed_map():
    spec = _spec((2, 2, 2))
    c = perturbation_coefficients(spec.seed)
    assert np.all(np.abs(c) <= 1) and np.abs(c).min() > 0.05
    rng = np.random.default_rng(0)
    s = rng.uniform(0, 1, (50, 3))
    aff = MeshSpec(2, 2, 2, lo=spec.lo, hi=spec.hi)
    # boundary of the box: the displacement vanishes
    for d in range(3):
        for v in (0.0, 1.0):
            sb = s.copy()
            sb[:, d] = v
            assert np.abs(analytic_map(spec, sb) - analytic_map(aff, sb)).max() <= 1e-15
    # interior: displaced, and x depends on s_y and s_z (not separable)
    assert np.abs(analytic_map(spec, s) - analytic_map(aff, s)).max() > 1e-3
    s2 = s.copy()
    s2[:, 1] += 0.01
    assert np.abs(analytic_map(spec, s2)[:, 0] - analytic_map(spec, s)[:, 0]).max() > 1e-5
    # zero amplitude: the affine map
    assert np.abs(analytic_map(_spec((2, 2, 2), amp=0.0), s) - analytic_map(aff, s)).max() == 0.0


def test_sipg_on_perturbed_periodic_mesh():
    op = SIPG(_spec((3, 2, 2)), 2)
    A = op.assemble()
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    one = np.ones(A.shape[0])
    assert np.abs(A @ one).max() <= 1e-11 * abs(A).max()
    w = np.linalg.eigvalsh(A.toarray())
    assert w[0] > -1e-10 * w[-1] and w[1] > 1e-6 * w[-1]  # one zero eigenvalue, the rest positive


def test_sipg_on_perturbed_dirichlet_mesh_is_spd():
    op = SIPG(_spec((2, 2, 2), bc=D_), 3)
    w = np.linalg.eigvalsh(op.assemble().toarray())
    assert w[0] > 0


def test_convergence_on_perturbed_mesh():
    """k = 2, u = sin(pi x / 2) cos(pi y / 2) sin(2 pi z / 1.5) with Dirichlet data
    zero on the box (x = 0, 2; y = -1, 1; z = 0, 1.5): L2 rate >= 2.7 from 4^3
    to 8^3 cells."""
    ue = lambda x, y, z: np.sin(np.pi * x / 2) * np.cos(np.pi * y / 2) * np.sin(2 * np.pi * z / 1.5)
    lam = (np.pi / 2) ** 2 + (np.pi / 2) ** 2 + (2 * np.pi / 1.5) ** 2
    fe = lambda x, y, z: lam * ue(x, y, z)
    errs = []
    for n in (4, 8):
        op = SIPG(_spec((n, n, n), bc=D_, amp=0.04), 2)
        A = op.assemble()
        d = A.diagonal()
        u, info = spla.cg(A, op.load_vector(fe), rtol=1e-12, maxiter=20000,
                          M=spla.LinearOperator(A.shape, matvec=lambda r: r / d))
        assert info == 0
        errs.append(op.l2_error(u, ue))
    assert math.log2(errs[0] / errs[1]) >= 2.7, errs
