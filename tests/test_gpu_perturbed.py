"""GPU parity of the general-metric path (SIPG_MAP_PERTURBED: a box plus a
smooth displacement, metric stored per quadrature point) against the oracle's
dense-quadrature SIPG matrix: Laplace, Helmholtz and mass applies within
1e-12 of ||A||_inf ||x||_inf, node coordinates and penalties, CG solves, and
at a size the oracle cannot assemble, symmetry and the constant null space;
the diagonal and Jacobi-preconditioned CG; entry points that need a separable
map reject the mesh."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import case, gpu_mesh, oracle_spec, uniform
from oracle.sipg import SIPG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 0x1234_5678_9ABC


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def pert(n, bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3, amp=0.06, seed=SEED):
    return case(n, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5), bc_lo=bc_lo, bc_hi=bc_hi, mapping="perturbed",
                amplitude=amp, seed=seed)


CASES = [
    ("periodic_k2", pert((3, 2, 2)), 2),
    ("dirichlet_box_k3", pert((2, 2, 2), ("dirichlet",) * 3, ("dirichlet",) * 3), 3),
    ("mixed_k4", pert((2, 3, 2), ("dirichlet", "neumann", "periodic"), ("neumann", "dirichlet", "periodic")), 4),
    ("channel_walls_k3", pert((3, 3, 2), ("periodic", "dirichlet", "periodic"), ("periodic", "dirichlet", "periodic"),
                              amp=0.1, seed=0xFFFF_0000_8001), 3),
    ("single_periodic_cell_k3", pert((1, 1, 1)), 3),
]


@pytest.mark.parametrize("arith", ["native", "double_float"])
@pytest.mark.parametrize("name,c,k", CASES, ids=[x[0] for x in CASES])
def test_perturbed_apply_parity(name, c, k, arith):
    from paper_1607_01323_gb300 import apply_helmholtz_f64, apply_laplace_f64, apply_mass_f64
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic(arith)
    assert np.abs(m.node_coordinates() - op.node_coordinates().reshape(-1, 3)).max() <= 1e-14
    assert np.allclose(m.penalty_values(), op.tau, rtol=1e-12, atol=0)
    x = uniform(m.n_dofs, "x", seed=31)
    A = op.assemble()
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    scale = abs(A).sum(axis=1).max() * np.abs(x).max()
    assert np.abs(y - A @ x).max() <= 1e-12 * scale
    H = op.assemble(mass_coef=1500.0, nu=1 / 180)
    x2 = np.concatenate([x, uniform(m.n_dofs, "x2", seed=32)])
    yh = apply_helmholtz_f64(m, _cuda(x2), 1500.0, 1 / 180).cpu().numpy().reshape(2, -1)
    sh = abs(H).sum(axis=1).max() * np.abs(x2).max()
    assert np.abs(yh[0] - H @ x).max() <= 1e-12 * sh
    assert np.abs(yh[1] - H @ x2[m.n_dofs:]).max() <= 1e-12 * sh
    Mx = op.mass_apply(x)
    ym = apply_mass_f64(m, _cuda(x)).cpu().numpy()
    assert np.abs(ym - Mx).max() <= 1e-13 * np.abs(Mx).max()
    # the diagonal (Jacobi), including self-coupling when a periodic
    # direction has one cell
    from paper_1607_01323_gb300 import diagonal_f64
    dA = diagonal_f64(m).cpu().numpy()
    assert np.abs(dA - A.diagonal()).max() <= 1e-12 * np.abs(A.diagonal()).max()
    dH = diagonal_f64(m, op="helmholtz", mass_coef=1500.0, nu=1 / 180).cpu().numpy()
    assert np.abs(dH - H.diagonal()).max() <= 1e-12 * np.abs(H.diagonal()).max()


def test_perturbed_cg_solves():
    from paper_1607_01323_gb300 import cg_solve
    c = pert((2, 2, 2), ("dirichlet",) * 3, ("dirichlet",) * 3)
    op = SIPG(oracle_spec(c), 3)
    m = gpu_mesh(c, 3)
    b = uniform(m.n_dofs, "b", seed=33)
    x, res = cg_solve(m, _cuda(b), precond="none", rtol=1e-12)
    assert res.converged
    x_ref = spla.spsolve(op.assemble().tocsc(), b)
    assert np.abs(x.cpu().numpy() - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
    xj, rj = cg_solve(m, _cuda(b), precond="jacobi", rtol=1e-12)
    assert rj.converged and rj.iters <= res.iters + 2
    assert np.abs(xj.cpu().numpy() - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
    # singular periodic problem: zero-mean right-hand side and solve
    cp = pert((2, 2, 2))
    mp = gpu_mesh(cp, 2)
    bp = uniform(mp.n_dofs, "bp", seed=34)
    bp -= bp.mean()
    xp, rp = cg_solve(mp, _cuda(bp), precond="none", zero_mean=True, rtol=1e-11)
    assert rp.converged
    Ap = SIPG(oracle_spec(cp), 2).assemble()
    r = bp - Ap @ xp.cpu().numpy()
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(bp)


def test_perturbed_properties_at_size():
    """16^3 cells at k = 3 (262,144 DoF): v.Au = u.Av and A 1 = 0 (periodic)."""
    from paper_1607_01323_gb300 import apply_laplace_f64
    m = gpu_mesh(pert((16, 16, 16), amp=0.04), 3)
    m.set_f64_arithmetic("double_float")
    u = _cuda(uniform(m.n_dofs, "u", seed=35))
    v = _cuda(uniform(m.n_dofs, "v", seed=36))
    Au, Av = apply_laplace_f64(m, u), apply_laplace_f64(m, v)
    a, b = torch.dot(v, Au).item(), torch.dot(u, Av).item()
    assert abs(a - b) <= 1e-12 * torch.dot(v.abs(), Au.abs()).item()
    one = torch.ones(m.n_dofs, dtype=torch.float64, device="cuda")
    A1 = apply_laplace_f64(m, one)
    assert A1.abs().max().item() <= 1e-11 * Au.abs().max().item()


def test_perturbed_rejections():
    from paper_1607_01323_gb300 import SipgError, apply_inverse_mass_f64, apply_laplace_f32, cg_solve
    c = pert((2, 2, 2), ("dirichlet",) * 3, ("dirichlet",) * 3)
    m = gpu_mesh(c, 2)
    x = _cuda(uniform(m.n_dofs, "x"))
    with pytest.raises(SipgError):
        apply_inverse_mass_f64(m, x)
    with pytest.raises(SipgError):
        apply_laplace_f32(m, x.float())
    with pytest.raises(SipgError):
        cg_solve(m, x, precond="invmass")
    with pytest.raises(SipgError):
        cg_solve(m, x, precond="gmg_f32")
