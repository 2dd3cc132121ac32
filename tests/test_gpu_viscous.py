"""GPU parity of the divergence-form viscous operator (Sec. 3.2 (iii))
against the oracle's assembled matrix: within 1e-12 of ||A||_inf ||u||_inf,
with the Laplace part in native FP64 and in double-float arithmetic; symmetry
at a size the oracle cannot assemble."""
import math

import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, oracle_spec, uniform
from oracle.viscous import ViscousOp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


CASES = [
    ("channel_k2", channel((2, 8, 2)), 2, 1.0),
    ("channel_4_layers_k4_penalty2", channel((2, 4, 2)), 4, 2.0),
    ("affine_neumann_walls_k3", case((2, 3, 2), lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5),
                                     bc_lo=("periodic", "neumann", "periodic"),
                                     bc_hi=("periodic", "neumann", "periodic")), 3, 1.0),
    ("box_mixed_k4", case((3, 2, 2), hi=(1.0, 0.7, 1.3), bc_lo=("dirichlet", "neumann", "periodic"),
                          bc_hi=("dirichlet", "dirichlet", "periodic")), 4, 1.0),
    ("single_periodic_cell_k3", case((1, 1, 1)), 3, 1.0),
    ("channel_k1", channel((3, 4, 2)), 1, 1.0),
]


@pytest.mark.parametrize("arith", ["native", "double_float"])
@pytest.mark.parametrize("name,c,k,pen", CASES, ids=[x[0] for x in CASES])
def test_viscous_parity(name, c, k, pen, arith):
    from paper_1607_01323_gb300 import apply_viscous_f64
    op = ViscousOp(oracle_spec(c), k, pen)
    m = gpu_mesh(c, k, penalty=pen)
    m.set_f64_arithmetic(arith)
    N = m.n_dofs
    u = uniform(3 * N, "u", seed=11)
    for cm, nu in ((0.0, 1.0), (1500.0, 1.0 / 180.0)):
        A = op.assemble(nu=nu, mass_coef=cm)
        y_ref = A @ u
        y = apply_viscous_f64(m, _cuda(u), cm, nu).cpu().numpy()
        scale = abs(A).sum(axis=1).max() * np.abs(u).max()
        assert np.abs(y - y_ref).max() <= 1e-12 * scale, (cm, nu, np.abs(y - y_ref).max() / scale)


def test_viscous_symmetry_at_size():
    """v^T A u = u^T A v on the 32^3 k = 3 channel (2.1M DoF per component)."""
    from paper_1607_01323_gb300 import apply_viscous_f64
    c = channel((32, 32, 32))
    m = gpu_mesh(c, 3)
    N = m.n_dofs
    u = _cuda(uniform(3 * N, "u", seed=12))
    v = _cuda(uniform(3 * N, "v", seed=13))
    a = torch.dot(v, apply_viscous_f64(m, u, 1500.0, 1 / 180.0)).item()
    b = torch.dot(u, apply_viscous_f64(m, v, 1500.0, 1 / 180.0)).item()
    scale = torch.dot(v.abs(), apply_viscous_f64(m, u, 1500.0, 1 / 180.0).abs()).item()
    assert abs(a - b) <= 1e-12 * scale


def test_viscous_errors():
    from paper_1607_01323_gb300 import SipgError, apply_viscous_f64
    m = gpu_mesh(channel((2, 4, 2)), 2)
    u = _cuda(uniform(3 * m.n_dofs, "u"))
    with pytest.raises(SipgError):
        apply_viscous_f64(m, u, 1.0, 0.0)
    with pytest.raises(SipgError):
        apply_viscous_f64(m, u, -1.0, 1.0)
    assert torch.isfinite(apply_viscous_f64(m, u, 1.0, 1.0)).all()


def test_viscous_cg_solve_matches_oracle():
    """(gamma0/dt) M + A_nu solved by CG with the inverse-mass preconditioner
    (the paper's viscous-step solver) against a sparse direct solve of the
    oracle's assembled operator."""
    import scipy.sparse.linalg as spla
    from paper_1607_01323_gb300 import cg_solve
    c = channel((2, 8, 2))
    k = 2
    op = ViscousOp(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    A = op.assemble(nu=1 / 180.0, mass_coef=1500.0)
    b = A @ uniform(3 * m.n_dofs, "x", seed=21)
    x_ref = spla.spsolve(A.tocsc(), b)
    # ||x - x_ref|| <= (||b - A x|| + ||b - A x_ref||) / lambda_min(A) for SPD A
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    for pc in ("invmass", "none"):
        x, res = cg_solve(m, _cuda(b), op="viscous", mass_coef=1500.0, nu=1 / 180.0, precond=pc, rtol=1e-10)
        assert res.converged and res.relres <= 1e-10
        xg = x.cpu().numpy()
        rg = np.linalg.norm(b - A @ xg)
        assert rg <= 2e-10 * np.linalg.norm(b)
        bound = 1.01 * (rg + np.linalg.norm(b - A @ x_ref)) / lmin
        assert np.linalg.norm(xg - x_ref) <= bound


def test_viscous_cg_rejects_unsupported_options():
    from paper_1607_01323_gb300 import SipgError, cg_solve
    m = gpu_mesh(channel((2, 4, 2)), 2)
    b = _cuda(uniform(3 * m.n_dofs, "b"))
    for kw in (dict(precond="jacobi"), dict(precond="gmg_f32"), dict(precond="invmass", zero_mean=1)):
        with pytest.raises(SipgError):
            cg_solve(m, b, op="viscous", mass_coef=1.0, nu=1.0, **kw)
    with pytest.raises(SipgError):
        cg_solve(m, b[: 2 * m.n_dofs].contiguous(), op="viscous", mass_coef=1.0, nu=1.0, precond="invmass")
