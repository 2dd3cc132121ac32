"""GPU geometric multigrid (Sec. 5.1) against the oracle's V-cycle.

The hierarchy's eigenvalue estimates are checked against the exact extreme
eigenvalues of the oracle's assembled level operators; one V-cycle (FP32 on
the GPU) is compared element by element with the oracle's FP64 V-cycle run
with the same Chebyshev intervals and degrees; multigrid-preconditioned CG
solves are compared with the oracle's solution and checked for
mesh-independent iteration counts."""
import math

import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, oracle_spec, uniform
from oracle import multigrid as omg
from oracle.sipg import SIPG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 V-cycle against the FP64 oracle, relative to max|z|: single precision
# (unit roundoff 6e-8) through about 2 * 5 * levels chained FP32 operator
# products whose rounding the Chebyshev polynomials amplify at most by their
# maximum on the interval (about 1 / lambda_min-scale growth of the
# smallest-eigenvalue components of the coarse solve): a 2e-5 bound.
TOL_V = 2e-5


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _exact_extremes(A, D):
    """Extreme eigenvalues of D^-1 A (via the symmetric D^-1/2 A D^-1/2)."""
    s = 1.0 / np.sqrt(D)
    ev = np.linalg.eigvalsh((A.toarray() * s[:, None]) * s[None, :])
    return ev


VCASES = [
    ("channel_4_k3", channel((4, 4, 4)), 3, 0),
    ("channel_neumann_4x2x4_k2", channel((4, 2, 4), wall="neumann"), 2, 1),
    ("box_odd_x_k4", case((3, 4, 2), hi=(1.0, 1.5, 0.8), bc_lo=("dirichlet", "neumann", "periodic"),
                          bc_hi=("dirichlet", "dirichlet", "periodic")), 4, 0),
]


@pytest.mark.parametrize("name,c,k,zm", VCASES, ids=[v[0] for v in VCASES])
def test_hierarchy_and_eigenvalue_estimates(name, c, k, zm):
    from paper_1607_01323_gb300 import mg_setup
    m = gpu_mesh(c, k)
    info = mg_setup(m, precond="gmg_f32", zero_mean=zm)
    mg = omg.Multigrid(oracle_spec(c), k)
    assert info["nlevels"] == mg.nlevels
    assert info["n_cells"] == [s.n for s in mg.specs]
    for l in range(mg.nlevels):
        ev = _exact_extremes(mg.A[l], mg.D[l])
        lam_max = ev.max()
        est = info["lmax"][l] / 1.1
        # a Ritz value lies inside the spectrum; 20 Lanczos steps from a random
        # start come close to the top
        assert est <= lam_max * (1 + 1e-9) and est >= 0.9 * lam_max, (l, est, lam_max)
    ev = _exact_extremes(mg.A[-1], mg.D[-1])
    lam_min = ev[ev > 1e-10 * ev.max()].min()
    lo = info["coarse_lmin"] / 0.9
    if lo != info["lmax"][-1] / 20:  # not the fallback interval
        assert lo >= lam_min * (1 - 1e-9) and lo <= 1.25 * lam_min, (lo, lam_min)
    # degree: smallest with the Chebyshev error estimate <= 1e-3
    kap = info["lmax"][-1] / info["coarse_lmin"]
    s = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    est = lambda d: 2 * s ** d / (1 + s ** (2 * d))
    d = info["coarse_degree"]
    assert est(d) <= 1e-3 and (d == 1 or est(d - 1) > 1e-3)


@pytest.mark.parametrize("name,c,k,zm", VCASES, ids=[v[0] for v in VCASES])
def test_vcycle_matches_oracle(name, c, k, zm):
    from paper_1607_01323_gb300 import mg_setup, mg_vcycle
    m = gpu_mesh(c, k)
    info = mg_setup(m, precond="gmg_f32", zero_mean=zm)
    mg = omg.Multigrid(oracle_spec(c), k)
    r = uniform(m.n_dofs, "r", seed=3)
    if zm:
        r = r - r.mean()
    # the GPU rounds r to FP32 first; give the oracle the same input
    r = r.astype(np.float32).astype(np.float64)
    z = mg_vcycle(m, _cuda(r)).cpu().numpy()
    z_ref = mg.vcycle(r, info["lmax"], degree=5, smoothing_range=20.0, coarse_degree=info["coarse_degree"],
                      coarse_interval=(info["coarse_lmin"], info["lmax"][-1]))
    err = np.max(np.abs(z - z_ref)) / np.max(np.abs(z_ref))
    assert err <= TOL_V, err


def test_mg_pcg_matches_oracle_solution():
    from paper_1607_01323_gb300 import apply_mass_f64, cg_solve
    c = channel((8, 8, 8))
    k = 3
    m = gpu_mesh(c, k)
    op = SIPG(oracle_spec(c), k)
    X = m.node_coordinates()
    f = (5 + math.pi ** 2 / 4) * np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    b = apply_mass_f64(m, _cuda(f))
    x, res = cg_solve(m, b, precond="gmg_f32", rtol=1e-10)
    assert res.converged and res.relres <= 1e-10
    _, rj = cg_solve(m, b, precond="jacobi", rtol=1e-10)
    assert res.iters <= 30 and 4 * res.iters < rj.iters, (res.iters, rj.iters)
    A = op.assemble()
    bn = b.cpu().numpy()
    xg = x.cpu().numpy()
    assert np.linalg.norm(bn - A @ xg) <= 2e-10 * np.linalg.norm(bn)


def test_mg_pcg_singular_neumann():
    from paper_1607_01323_gb300 import cg_solve
    c = channel((4, 4, 4), wall="neumann")
    k = 3
    m = gpu_mesh(c, k)
    op = SIPG(oracle_spec(c), k)
    b = uniform(m.n_dofs, "b", seed=5)
    b = b - b.mean()
    x, res = cg_solve(m, _cuda(b), precond="gmg_f32", zero_mean=1, rtol=1e-10)
    assert res.converged and res.relres <= 1e-10
    r = b - op.apply(x.cpu().numpy())
    assert np.linalg.norm(r - r.mean()) <= 2e-10 * np.linalg.norm(b)


def test_mg_iterations_mesh_independent_and_deterministic():
    from paper_1607_01323_gb300 import apply_laplace_f64, cg_solve
    its = []
    for n in (8, 16, 32):
        c = channel((n, n, n))
        m = gpu_mesh(c, 4)
        b = _cuda(uniform(m.n_dofs, "b", seed=1))
        x, res = cg_solve(m, b, precond="gmg_f32", rtol=1e-10)
        assert res.converged
        r = b - apply_laplace_f64(m, x)
        assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() <= 2e-10
        its.append(res.iters)
        if n == 16:
            x2, res2 = cg_solve(m, b, precond="gmg_f32", rtol=1e-10, use_graph=0)
            assert res2.iters == res.iters and torch.equal(x, x2)
    # Jacobi-PCG doubles its count per refinement; the V-cycle's count grows far
    # slower on this graded channel (the wall-normal stretching, and with it the
    # cells' aspect ratio, grows under refinement)
    assert all(its[i + 1] <= 1.25 * its[i] + 2 for i in range(2)) and max(its) <= 50, its


def test_mg_errors_and_invalidation():
    from paper_1607_01323_gb300 import SipgError, cg_solve, mg_info, mg_setup, mg_vcycle
    c = channel((4, 4, 4))
    m = gpu_mesh(c, 2)
    b = _cuda(uniform(m.n_dofs, "b"))
    with pytest.raises(SipgError):
        mg_vcycle(m, b)  # no hierarchy yet
    with pytest.raises(SipgError):
        cg_solve(m, b, precond="gmg_f32", op="helmholtz", mass_coef=1.0, nu=1.0)
    with pytest.raises(SipgError):
        cg_solve(m, torch.cat([b, b]), precond="gmg_f32")
    with pytest.raises(SipgError):
        mg_setup(m, mg_degree=0)
    mg_setup(m)
    assert mg_info(m)["nlevels"] == 3
    m.set_degree(3)
    with pytest.raises(SipgError):
        mg_info(m)
