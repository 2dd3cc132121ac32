"""GPU conjugate-gradient solves against the oracle's solutions and error paths.

Solves are compared by (i) the GPU's own recursive residual <= rtol, (ii) the
true residual of the GPU solution under the ORACLE's operator, and (iii) the
distance to the oracle's solution of the same system, within
kappa * rtol-level bounds (the solutions of a system solved to 1e-10 agree to
about cond(A) * 1e-10)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import case, channel, gpu_mesh, oracle_spec, uniform
from oracle.sipg import SIPG
from paper_1607_01323_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def distance_bound(A, b, x_a, x_b):
    """||x_a - x_b|| <= (||b - A x_a|| + ||b - A x_b||) / lambda_min(A) for SPD A."""
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    return 1.01 * (np.linalg.norm(b - A @ x_a) + np.linalg.norm(b - A @ x_b)) / lmin


def manufactured_rhs(m, op):
    """b = M f_I, f = (5 + pi^2/4) sin x cos(pi y/2) sin 2z at the nodes; each side
    evaluates f at its own node coordinates and applies its own mass matrix."""
    from paper_1607_01323_gb300 import apply_mass_f64
    f = lambda X: (5 + math.pi ** 2 / 4) * np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    b_gpu = apply_mass_f64(m, _cuda(f(m.node_coordinates())))
    b_orc = op.mass_apply(f(op.node_coordinates().reshape(-1, 3)))
    return b_gpu, b_orc


@pytest.mark.parametrize("use_graph", [0, 1])
def test_poisson_jacobi_cg_channel(use_graph):
    from paper_1607_01323_gb300 import cg_solve
    c = channel((6, 6, 6))
    k = 3
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    b_gpu, b_orc = manufactured_rhs(m, op)
    assert np.max(np.abs(b_gpu.cpu().numpy() - b_orc)) <= 1e-13 * np.max(np.abs(b_orc))
    x, res = cg_solve(m, b_gpu, precond="jacobi", rtol=1e-10, use_graph=use_graph, check_every=8)
    assert res.converged and res.relres <= 1e-10
    A = op.assemble()
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b_orc - A @ xg) / np.linalg.norm(b_orc)
    assert true_rel <= 1e-9
    x_orc = spla.spsolve(A.tocsc(), b_orc)
    assert np.linalg.norm(xg - x_orc) <= distance_bound(A, b_orc, xg, x_orc)
    assert np.linalg.norm(xg - x_orc) <= 1e-6 * np.linalg.norm(x_orc)


def test_poisson_double_float_operator():
    """CG with the double-float FP64 operator reaches 1e-10 and agrees with the
    native FP64 solve within the residual bound."""
    from paper_1607_01323_gb300 import cg_solve
    c = channel((6, 6, 6))
    k = 4
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    b_gpu, b_orc = manufactured_rhs(m, op)
    xn, rn = cg_solve(m, b_gpu, precond="jacobi", rtol=1e-10)
    m.set_f64_arithmetic("double_float")
    xd, rd = cg_solve(m, b_gpu, precond="jacobi", rtol=1e-10)
    assert rn.converged and rd.converged
    A = op.assemble()
    xg = xd.cpu().numpy()
    assert np.linalg.norm(b_orc - A @ xg) <= 1e-9 * np.linalg.norm(b_orc)
    assert np.linalg.norm(xg - xn.cpu().numpy()) <= distance_bound(A, b_orc, xg, xn.cpu().numpy())


def test_graph_and_loop_bitwise_equal():
    from paper_1607_01323_gb300 import cg_solve
    c = channel((4, 4, 4))
    m = gpu_mesh(c, 4)
    b = _cuda(uniform(m.n_dofs, "b"))
    x1, r1 = cg_solve(m, b, use_graph=0, check_every=5)
    x2, r2 = cg_solve(m, b, use_graph=1, check_every=5)
    x3, r3 = cg_solve(m, b, use_graph=1, check_every=16)
    assert r1.iters == r2.iters == r3.iters
    assert torch.equal(x1, x2) and torch.equal(x1, x3)


@pytest.mark.parametrize("precond", ["invmass", "jacobi", "none"])
def test_helmholtz_three_components(precond):
    from paper_1607_01323_gb300 import apply_mass_f64, cg_solve
    c = channel((4, 4, 3))
    k = 3
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    N = m.n_dofs
    cm, nu = 1500.0, 1.0 / 180.0
    X = m.node_coordinates()
    u_in = np.concatenate([(1 - X[:, 1] ** 2) + 0.1 * inputs.normal(0, "ux", N), 0.1 * inputs.normal(0, "uy", N),
                           0.1 * inputs.normal(0, "uz", N)])
    rhs = cm * apply_mass_f64(m, _cuda(u_in))
    x, res = cg_solve(m, rhs, op="helmholtz", mass_coef=cm, nu=nu, precond=precond, rtol=1e-10)
    assert res.converged
    A = op.assemble(mass_coef=cm, nu=nu)
    xg = x.cpu().numpy().reshape(3, N)
    r = rhs.cpu().numpy().reshape(3, N)
    true_rel = np.sqrt(sum(np.linalg.norm(r[i] - A @ xg[i]) ** 2 for i in range(3))) / np.linalg.norm(r)
    assert true_rel <= 1e-9
    for i in range(3):
        xo = spla.spsolve(A.tocsc(), r[i])
        assert np.linalg.norm(xg[i] - xo) <= distance_bound(A, r[i], xg[i], xo)


def test_neumann_zero_mean_chebyshev_f32():
    """Singular Poisson problem (Neumann walls): zero-mean rhs, FP32 Chebyshev(4)
    preconditioner under flexible FP64 CG, versus plain FP64 Jacobi CG and the
    oracle solution (all compared after projection onto zero mean)."""
    from paper_1607_01323_gb300 import cg_solve
    c = channel((4, 6, 4), wall="neumann")
    k = 3
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    b = uniform(m.n_dofs, "b")
    b = b - b.mean()
    xc, rc = cg_solve(m, _cuda(b), precond="cheb_f32", cheb_degree=4, zero_mean=1, rtol=1e-10)
    xj, rj = cg_solve(m, _cuda(b), precond="jacobi", zero_mean=1, rtol=1e-10)
    assert rc.converged and rj.converged
    assert rc.iters < rj.iters
    A = op.assemble()
    for x in (xc, xj):
        xg = x.cpu().numpy()
        xg = xg - xg.mean()
        assert np.linalg.norm(b - A @ xg) <= 1e-9 * np.linalg.norm(b)
    xo, _, _ = __import__("oracle.solvers", fromlist=["cg"]).cg(lambda v: A @ v, b, rtol=1e-12, zero_mean=True,
                                                                precond=lambda r: r / A.diagonal())
    xo = xo - xo.mean()
    for x in (xc, xj):
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xg.mean() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_status_codes_without_faults():
    """Failures come back as status codes (no trap, no hang): an indefinite
    operator breaks down, a NaN right-hand side is non-finite, maxit stops."""
    from paper_1607_01323_gb300 import SipgError, cg_solve
    from paper_1607_01323_gb300 import _lib as L
    m = gpu_mesh(channel((2, 3, 2)), 2)  # the 3-layer tanh channel at k=2 is indefinite
    b = _cuda(uniform(m.n_dofs, "b"))
    _, r = cg_solve(m, b, precond="none", rtol=1e-14, maxit=5000, raise_on_fail=False)
    assert r.status == L.BREAKDOWN
    m = gpu_mesh(channel((3, 4, 2)), 2)
    bn = _cuda(uniform(m.n_dofs, "b"))
    bn[7] = float("nan")
    _, r = cg_solve(m, bn, raise_on_fail=False)
    assert r.status == L.NONFINITE
    _, r = cg_solve(m, _cuda(uniform(m.n_dofs, "b")), maxit=1, raise_on_fail=False)
    assert r.status == L.MAXITER and r.iters == 1
    with pytest.raises(SipgError):
        cg_solve(m, _cuda(uniform(m.n_dofs, "b")), maxit=0)
    # the context is still usable afterwards
    x, r = cg_solve(m, _cuda(uniform(m.n_dofs, "b")))
    assert r.converged
