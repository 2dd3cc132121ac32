"""Adjoint gradient dJ/dnu_e against the oracle's assembled-derivative gradient
and against central finite differences of J."""
import math

import numpy as np
import pytest

from helpers import channel, gpu_mesh, oracle_spec, uniform
from oracle import adjoint as oadj
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


@pytest.mark.parametrize("k,ties", [(2, False), (3, False), (3, True), (5, False)])
def test_grad_formula_matches_oracle(k, ties):
    from paper_1607_01323_gb300 import adjoint_grad_nu
    c = channel((3, 4, 2))
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    nu = np.full(m.ncell, 1 / 180.0) if ties else np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0
    u, lam = uniform(m.n_dofs, "u"), uniform(m.n_dofs, "lam")
    g = adjoint_grad_nu(m, _cuda(nu), _cuda(u), _cuda(lam)).cpu().numpy()
    g_ref = oadj.grad_nu(op, nu, u, lam)
    assert np.max(np.abs(g - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))


def test_autograd_end_to_end_small():
    """J(nu, f) through HelmholtzSolve/MassApply: gradients equal the oracle's
    adjoint (assembled dA/dnu_e) and lambda for dJ/df."""
    import scipy.sparse.linalg as spla
    from paper_1607_01323_gb300.autograd import helmholtz_solve, mass_norm_loss
    c = channel((3, 4, 3))
    k = 3
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    cm = 1500.0
    nu = np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0
    X = m.node_coordinates()
    fc = np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    ut = np.cos(math.pi * X[:, 1] / 2) * (1 + 0.5 * np.sin(X[:, 0] + 1.0) * np.cos(X[:, 2] + 2.0))
    f = op.mass_apply(fc)
    nu_t = _cuda(nu).requires_grad_(True)
    f_t = _cuda(f).requires_grad_(True)
    u = helmholtz_solve(m, nu_t, f_t, cm, rtol=1e-13)
    J = mass_norm_loss(m, u, _cuda(ut))
    J.backward()
    A = op.assemble(mass_coef=cm, nu_cell=nu)
    uo = spla.spsolve(A.tocsc(), f)
    lo = spla.spsolve(A.tocsc(), op.mass_apply(uo - ut))
    g_ref = oadj.grad_nu(op, nu, uo, lo)
    assert abs(J.item() - oadj.loss(op, uo, ut)) <= 1e-10 * abs(J.item())
    assert np.max(np.abs(nu_t.grad.cpu().numpy() - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))
    assert np.max(np.abs(f_t.grad.cpu().numpy() - lo)) <= 1e-8 * np.max(np.abs(lo))
