"""Pins of the oracle's geometric multigrid V-cycle (Sec. 5.1): level
transfer by tensorial embedding, the Chebyshev smoother, symmetry of the
V-cycle as a preconditioner, and mesh-independent iteration counts.

Each test checks a property the mathematics fixes (polynomial exactness of
the embedding, nestedness of the spaces, symmetry, the shift identity of a
polynomial iteration) or the paper's claim that the iteration count does not
grow with the mesh size."""
import math

import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import solvers
from oracle.mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec
from oracle.sipg import SIPG

P_, D_, N_ = PERIODIC, DIRICHLET, NEUMANN


def box(n, bc=D_, mapping="affine"):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5), bc_lo=(bc,) * 3, bc_hi=(bc,) * 3,
                    mapping=mapping)


def channel(n, wall=D_):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi), bc_lo=(P_, wall, P_),
                    bc_hi=(P_, wall, P_), mapping="channel", gamma=1.8)


def poly(x, k, seed):
    """A random polynomial of total degree <= k in each coordinate (tensor degree k)."""
    c = np.random.default_rng(seed).standard_normal((k + 1, k + 1, k + 1))
    out = np.zeros(x.shape[0])
    for i in range(k + 1):
        for j in range(k + 1):
            for m in range(k + 1):
                out += c[i, j, m] * x[:, 0] ** i * x[:, 1] ** j * x[:, 2] ** m
    return out


def test_coarsening_hierarchy():
    mg = omg.Multigrid(channel((4, 2, 1)), 1)
    assert [s.n for s in mg.specs] == [(4, 2, 1), (2, 1, 1), (1, 1, 1)]
    assert [s.mapping for s in mg.specs] == ["channel", "channel_linear", "channel_linear"]
    c, f = omg.coarsen_spec(MeshSpec(3, 5, 1))
    assert c is None and f == [1, 1, 1]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_reproduces_polynomials(k):
    """On an affine mesh the coarse space is nested in the fine one: the
    embedding of the coarse interpolant of a tensor polynomial of degree k is
    the fine interpolant of the same polynomial (Sec. 5.1 tensorial
    embedding).  A transposed or mis-indexed 1D embedding fails this."""
    fine = box((4, 2, 3))            # z has an odd count: not coarsened
    c, f = omg.coarsen_spec(fine)
    assert f == [2, 2, 1]
    opf, opc = SIPG(fine, k), SIPG(c, k)
    P = omg.prolongation(fine, c, f, opf.zn)
    xf, xc = opf.node_coordinates().reshape(-1, 3), opc.node_coordinates().reshape(-1, 3)
    for seed in range(3):
        assert np.allclose(P @ poly(xc, k, seed), poly(xf, k, seed), rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [1, 3])
def test_prolongation_preserves_mass(k):
    """Nested spaces and exact Gauss quadrature on affine cells: the fine mass
    matrix restricted to the coarse space is the coarse mass matrix,
    P^T M_f P = M_c (each fine cell is one half of its parent per direction)."""
    fine = box((2, 4, 2))
    c, f = omg.coarsen_spec(fine)
    opf, opc = SIPG(fine, k), SIPG(c, k)
    P = omg.prolongation(fine, c, f, opf.zn).toarray()
    nc = P.shape[1]
    Mc = np.stack([opc.mass_apply(e) for e in np.eye(nc)], axis=1)
    MfP = np.stack([opf.mass_apply(P[:, j]) for j in range(nc)], axis=1)
    assert np.allclose(P.T @ MfP, Mc, rtol=0, atol=1e-13 * np.abs(Mc).max())


def test_chebyshev_from_shift_identity():
    """A polynomial iteration started from x0 equals x0 plus the same
    iteration from zero applied to the residual b - A x0."""
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    d = A.diagonal().copy()
    b, x0 = rng.standard_normal(30), rng.standard_normal(30)
    for deg in (1, 2, 5):
        got = solvers.chebyshev_from(lambda v: A @ v, d, b, x0, deg, 0.3, 4.0)
        want = x0 + solvers.chebyshev(lambda v: A @ v, d, b - A @ x0, deg, 0.3, 4.0)
        assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
        assert np.array_equal(solvers.chebyshev_from(lambda v: A @ v, d, b, None, deg, 0.3, 4.0),
                              solvers.chebyshev(lambda v: A @ v, d, b, deg, 0.3, 4.0))


def _levels_lmax(mg):
    return [1.1 * solvers.lanczos_max_eig(lambda v, A=A: A @ v, D, np.ones(A.shape[0]), steps=30)
            for A, D in zip(mg.A, mg.D)]


@pytest.mark.parametrize("wall", [D_, N_])
def test_vcycle_symmetric_positive(wall):
    """With the same Chebyshev polynomial before and after the coarse
    correction, the V-cycle is a symmetric linear operator, positive definite
    on the range of A: a valid CG preconditioner (Sec. 5.1)."""
    mg = omg.Multigrid(channel((2, 4, 2), wall), 2)
    lmax = _levels_lmax(mg)
    n = mg.A[0].shape[0]
    V = np.stack([mg.vcycle(e, lmax, coarse_degree=8) for e in np.eye(n)], axis=1)
    assert np.abs(V - V.T).max() <= 1e-12 * np.abs(V).max()
    ev = np.linalg.eigvalsh(0.5 * (V + V.T))
    if wall == D_:
        assert ev.min() > 0
    else:
        # one (near-)null direction from the constant null space of A
        Z = np.linalg.qr(np.ones((n, 1)), mode="complete")[0][:, 1:]
        assert np.linalg.eigvalsh(Z.T @ V @ Z).min() > 0


def test_vcycle_mesh_independent_iterations():
    """One V-cycle as CG preconditioner: the iteration count stays flat under
    refinement while Jacobi-PCG grows (Sec. 5.1, h-independent iterations)."""
    its, jac = [], []
    for n in (4, 8):
        mg = omg.Multigrid(channel((n, n, n)), 2)
        lmax = _levels_lmax(mg)
        b = np.random.default_rng(0).standard_normal(mg.A[0].shape[0])
        _, it, rel = solvers.cg(lambda v: mg.A[0] @ v, b, rtol=1e-10,
                                precond=lambda r: mg.vcycle(r, lmax, coarse_degree=10))
        _, itj, _ = solvers.cg(lambda v: mg.A[0] @ v, b, rtol=1e-10, precond=lambda r: r / mg.D[0])
        assert rel <= 1e-10
        its.append(it)
        jac.append(itj)
    assert its[1] <= its[0] + 5 and its[1] * 5 < jac[1], (its, jac)


def test_mutation_embedding_child_caught(monkeypatch):
    """Planting a swapped child half in the 1D embedding breaks polynomial
    reproduction (the pin above would catch it)."""
    good = omg.embedding_1d
    monkeypatch.setattr(omg, "embedding_1d", lambda zn, child, factor: good(zn, 1 - child, factor))
    fine = box((4, 2, 1))
    c, f = omg.coarsen_spec(fine)
    opf, opc = SIPG(fine, 2), SIPG(c, 2)
    P = omg.prolongation(fine, c, f, opf.zn)
    xf, xc = opf.node_coordinates().reshape(-1, 3), opc.node_coordinates().reshape(-1, 3)
    assert not np.allclose(P @ poly(xc, 2, 0), poly(xf, 2, 0), rtol=0, atol=1e-6)
