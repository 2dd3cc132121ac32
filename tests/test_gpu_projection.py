"""GPU parity of the V3c pressure-projection operators against the oracle:
divergence (Eq. (av3)), gradient (Eq. (bv3)), tau_D (Eq. (tauD)), the div-div
operator and its per-cell solve (Eq. (div-div)).

Bars: operators within 1e-12 of ||A||_inf ||x||_inf (FP64, the operator bar)
on meshes small enough to assemble the oracle's matrix, 1e-11 of max|y_ref|
on larger ones; the local solve within 1e-10 relative of the oracle's dense
solve.  At sizes the oracle cannot run, properties that hold at any size:
the discrete adjointness D = -G^T on periodic meshes and exact integration
by parts for polynomial fields on affine meshes."""
import math

import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, oracle_spec, uniform
from oracle.projection import ProjectionOps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


CASES = [
    ("channel_k3", channel((2, 4, 2)), 3),
    ("channel_neumann_k2", channel((3, 4, 2), wall="neumann"), 2),
    ("box_mixed_k4", case((3, 2, 2), hi=(1.0, 0.7, 1.3), bc_lo=("dirichlet", "neumann", "periodic"),
                          bc_hi=("dirichlet", "dirichlet", "periodic")), 4),
    ("single_periodic_cell_k3", case((1, 1, 1)), 3),
    ("periodic_k1", case((3, 3, 2)), 1),
    ("channel_k6", channel((2, 4, 1)), 6),
]


@pytest.mark.parametrize("name,c,k", CASES, ids=[x[0] for x in CASES])
def test_divergence_gradient_parity(name, c, k):
    from paper_1607_01323_gb300 import apply_divergence_f64, apply_gradient_f64
    ops = ProjectionOps(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    N = m.n_dofs
    u = uniform(3 * N, "u", seed=1)
    p = uniform(N, "p", seed=2)
    yd_ref = ops.divergence(u)
    yg_ref = ops.gradient(p)
    yd = apply_divergence_f64(m, _cuda(u)).cpu().numpy()
    yg = apply_gradient_f64(m, _cuda(p)).cpu().numpy()
    if 3 * N <= 1600:  # assemble the oracle matrices for the scaled bar
        D = np.stack([ops.divergence(e) for e in np.eye(3 * N)], axis=1)
        G = np.stack([ops.gradient(e) for e in np.eye(N)], axis=1)
        sd = np.abs(D).sum(axis=1).max() * np.abs(u).max()
        sg = np.abs(G).sum(axis=1).max() * np.abs(p).max()
        tol = 1e-12
    else:
        sd, sg, tol = np.abs(yd_ref).max(), np.abs(yg_ref).max(), 1e-11
    assert np.abs(yd - yd_ref).max() <= tol * sd
    assert np.abs(yg - yg_ref).max() <= tol * sg


@pytest.mark.parametrize("name,c,k", CASES[:3], ids=[x[0] for x in CASES[:3]])
def test_tau_divdiv_apply_and_solve(name, c, k):
    from paper_1607_01323_gb300 import apply_divdiv_f64, project_divdiv_f64, tau_div_f64
    ops = ProjectionOps(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    N = m.n_dofs
    u = uniform(3 * N, "u", seed=3)
    tau_ref = ops.tau_div(u, zeta=5.0, dt=0.02)
    tau = tau_div_f64(m, _cuda(u), 5.0, 0.02).cpu().numpy()
    assert np.allclose(tau, tau_ref, rtol=1e-13, atol=0)
    y_ref = ops.projection_apply(u, tau_ref)
    y = apply_divdiv_f64(m, _cuda(tau_ref), _cuda(u)).cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    rhs = ops.mass(u, 3) + 0.1 * ops.gradient(uniform(N, "p", seed=4))
    x_ref = ops.project(rhs, tau_ref)
    x, iters = project_divdiv_f64(m, _cuda(tau_ref), _cuda(rhs), rtol=1e-13, maxit=500)
    x = x.cpu().numpy()
    assert np.abs(x - x_ref).max() <= 1e-10 * np.abs(x_ref).max()
    assert 1 <= iters <= 3 * (k + 1) ** 3
    # the local solve in double-float arithmetic: same solution to the tolerance
    m.set_f64_arithmetic("double_float")
    x2, iters2 = project_divdiv_f64(m, _cuda(tau_ref), _cuda(rhs), rtol=1e-12, maxit=500)
    assert np.abs(x2.cpu().numpy() - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
    assert abs(iters2 - iters) <= 3 + iters // 4


def test_projection_reduces_divergence_and_keeps_free_fields():
    """Larger penalties give smaller divergence (the oracle's measure of the
    GPU results); tau = 0 returns M^-1 rhs."""
    from paper_1607_01323_gb300 import apply_inverse_mass_f64, project_divdiv_f64
    c = channel((4, 4, 4))
    k = 3
    ops = ProjectionOps(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    N = m.n_dofs
    u = uniform(3 * N, "u", seed=6)
    rhs = _cuda(ops.mass(u, 3))
    errs = []
    for t in (0.0, 0.05, 0.5, 5.0):
        x, _ = project_divdiv_f64(m, torch.full((m.ncell,), t, dtype=torch.float64, device="cuda"), rhs,
                                  rtol=1e-13, maxit=500)
        errs.append(ops.divergence_l2(x.cpu().numpy()))
        if t == 0.0:
            xm = apply_inverse_mass_f64(m, rhs).cpu().numpy()
            assert np.abs(x.cpu().numpy() - xm).max() <= 1e-11 * np.abs(xm).max()
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_adjointness_and_polynomial_exactness_at_size():
    """Properties at sizes the oracle cannot run: p^T D u = -(G p)^T u on a
    periodic affine box (48 x 16 x 16 cells, k = 4), and D u = -M (div u)
    for a polynomial field on an affine box with walls."""
    from paper_1607_01323_gb300 import Mesh, apply_divergence_f64, apply_gradient_f64, apply_mass_f64
    m = Mesh((48, 16, 16), (0.0, 0.0, 0.0), (3.0, 1.0, 1.0), k=4)
    N = m.n_dofs
    u = _cuda(uniform(3 * N, "u", seed=7))
    p = _cuda(uniform(N, "p", seed=8))
    a = torch.dot(p, apply_divergence_f64(m, u)).item()
    b = torch.dot(apply_gradient_f64(m, p), u).item()
    scale = torch.dot(p.abs(), apply_divergence_f64(m, u).abs()).item()
    assert abs(a + b) <= 1e-12 * scale * math.sqrt(N)
    w = Mesh((16, 12, 10), (0.0, -1.0, 0.0), (2.0, 1.0, 1.0), ("dirichlet",) * 3, ("neumann",) * 3, k=3)
    X = w.node_coordinates()
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    uu = np.stack([x ** 2 * y + z ** 3, y ** 3 - x * z, x * y * z ** 2]).ravel()
    div = 2 * x * y + 3 * y ** 2 + 2 * x * y * z
    lhs = apply_divergence_f64(w, _cuda(uu))
    rhs = -apply_mass_f64(w, _cuda(div))
    assert (lhs - rhs).abs().max().item() <= 1e-12 * rhs.abs().max().item() * 10


def test_projection_errors():
    from paper_1607_01323_gb300 import SipgError, project_divdiv_f64
    c = channel((2, 4, 2))
    m = gpu_mesh(c, 2)
    N = m.n_dofs
    rhs = _cuda(uniform(3 * N, "r"))
    tau = torch.full((m.ncell,), 1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(SipgError) as e:
        project_divdiv_f64(m, tau, rhs, rtol=1e-30, maxit=1)
    assert e.value.status == 1  # SIPG_MAXITER
    with pytest.raises(SipgError) as e:
        project_divdiv_f64(m, tau, rhs, maxit=0)
    assert e.value.status == -1
    # the context stays usable
    x, it = project_divdiv_f64(m, tau, rhs, rtol=1e-12, maxit=500)
    assert it >= 1
