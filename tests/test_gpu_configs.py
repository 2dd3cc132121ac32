"""The five workload configurations at full size, in the launch configuration the
bench uses.  The oracle cannot assemble these operators, so parity is checked
on sampled cells (every output of a sampled cell, computed by the oracle's
element-by-element apply restricted to those rows), and the solves through
properties that hold at any size (recursive and true residuals, agreement of
two solvers, bounds from the residual).

Sampled cells always include the domain corners, both walls and the periodic
seams, plus seeded random cells.
"""
import math

import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, oracle_spec, scaled_err
from oracle import adjoint as oadj
from oracle.sipg import SIPG
from paper_1607_01323_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def sample_cells(n, count=48, seed=0):
    nx, ny, nz = n
    idx = set()
    for ix in (0, nx - 1):
        for iy in (0, 1, ny // 2, ny - 2, ny - 1):
            for iz in (0, nz - 1):
                idx.add((iz * ny + iy) * nx + ix)
    u = inputs.u64(seed, "cells", 0, count)
    for v in u:
        idx.add(int(v % np.uint64(nx * ny * nz)))
    mask = np.zeros(nx * ny * nz, dtype=bool)
    mask[sorted(idx)] = True
    return mask


def sampled_parity(c, k, y_gpu, x, targets, tol, ncomp=1, **kw):
    op = SIPG(oracle_spec(c), k)
    y_ref = op.apply(x.reshape(ncomp, -1), targets=targets, **kw).ravel()
    P = (k + 1) ** 3
    rows = np.repeat(targets, P)
    rows = np.tile(rows, ncomp)
    norm_a = op.norm_inf(targets=targets, **kw)
    err = scaled_err(y_gpu[rows], y_ref[rows], norm_a, x)
    assert err <= tol, err
    return op


C2 = channel((32, 32, 32))
# rounding-error constant of the C5 gradient comparison, in units of the unit
# roundoff times the summed term magnitudes
C_ROUND = 16
C3 = channel((64, 64, 64))
C4 = channel((48, 48, 48), wall="neumann")
C5 = channel((32, 32, 32))


def test_c1_periodic_cube_full():
    """4^3 periodic affine cube, k = 3, tau of Eq. (taue) (=192) and (k+1)^2/h (=64)."""
    from paper_1607_01323_gb300 import apply_laplace_f64
    c = case((4, 4, 4))
    for pen, tau in ((1.0, 192.0), (1 / 3, 64.0)):
        op = SIPG(oracle_spec(c), 3, penalty_factor=pen)
        m = gpu_mesh(c, 3, penalty=pen)
        assert np.allclose(m.penalty_values(), tau, rtol=1e-14)
        x = inputs.uniform(0, "x", m.n_dofs)
        A = op.assemble()
        y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
        assert scaled_err(y, A @ x, abs(A).sum(axis=1).max(), x) <= 1e-12


def test_c2_poisson_channel_32_k4():
    """Apply parity on sampled cells; Jacobi-PCG to 1e-10 with graph chunks of 16;
    the solution's true residual (GPU apply) and its L2 distance to the exact
    manufactured solution (discretisation error)."""
    from paper_1607_01323_gb300 import apply_laplace_f64, apply_mass_f64, cg_solve
    k = 4
    m = gpu_mesh(C2, k)
    x = inputs.uniform(0, "x", m.n_dofs)
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    tg = sample_cells(C2["n"])
    op = sampled_parity(C2, k, y, x, tg, 1e-12)
    X = m.node_coordinates()
    ue = np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    b = apply_mass_f64(m, _cuda((5 + math.pi ** 2 / 4) * ue))
    u, res = cg_solve(m, b, precond="jacobi", rtol=1e-10, use_graph=1, check_every=16)
    assert res.converged and res.relres <= 1e-10
    r = b - apply_laplace_f64(m, u)
    assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() <= 1e-9
    # nodal error against the exact solution: small (k = 4 on 32^3)
    assert np.max(np.abs(u.cpu().numpy() - ue)) <= 1e-5
    # the oracle's operator on sampled rows agrees with the GPU residual there
    ug = u.cpu().numpy()
    Au = op.apply(ug, targets=tg)
    rows = np.repeat(tg, (k + 1) ** 3)
    assert np.max(np.abs(Au[rows] - (b - r).cpu().numpy()[rows])) <= 1e-12 * op.norm_inf(targets=tg) * np.max(
        np.abs(ug))


def test_c2_poisson_channel_32_k4_double_float():
    """The bench's double-float variant at full size: sampled-cell apply parity
    at 1e-12 (also with the input scaled by 1e-250 and 1e250), the
    graph-captured Jacobi-PCG to 1e-10, and its solution's true residual taken
    with the native-FP64 operator; the solution agrees with the native solve's."""
    from paper_1607_01323_gb300 import apply_laplace_f64, apply_mass_f64, cg_solve
    k = 4
    m = gpu_mesh(C2, k)
    m.set_f64_arithmetic("double_float")
    m64 = gpu_mesh(C2, k)
    x = inputs.uniform(0, "x", m.n_dofs)
    tg = sample_cells(C2["n"])
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    op = sampled_parity(C2, k, y, x, tg, 1e-12)
    for s in (1e-250, 1e250):
        ys = apply_laplace_f64(m, _cuda(s * x)).cpu().numpy()
        sampled_parity(C2, k, ys, s * x, tg, 1e-12)
    del op
    X = m.node_coordinates()
    ue = np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    b = apply_mass_f64(m64, _cuda((5 + math.pi ** 2 / 4) * ue))
    u, res = cg_solve(m, b, precond="jacobi", rtol=1e-10, use_graph=1, check_every=16)
    assert res.converged and res.relres <= 1e-10
    r = b - apply_laplace_f64(m64, u)
    assert (torch.linalg.norm(r) / torch.linalg.norm(b)).item() <= 1e-9
    u64, res64 = cg_solve(m64, b, precond="jacobi", rtol=1e-10, use_graph=1, check_every=16)
    assert res64.converged
    assert (torch.linalg.norm(u - u64) / torch.linalg.norm(u64)).item() <= 1e-8
    assert np.max(np.abs(u.cpu().numpy() - ue)) <= 1e-5


def test_c3_helmholtz_three_components_64_k3():
    """(gamma0/dt) M + nu L with gamma0 = 1.5, dt = 1e-3, nu = 1/180 on 3 components
    of 64^3 k = 3 cells: sampled apply parity; autotuned cells per block; graph
    captured CG with M^-1 and with Jacobi preconditioning."""
    from paper_1607_01323_gb300 import apply_helmholtz_f64, apply_mass_f64, autotune, cg_solve
    k = 3
    m = gpu_mesh(C3, k)
    N = m.n_dofs
    cm, nu = 1.5 / 1e-3, 1 / 180
    X = m.node_coordinates()
    u_in = np.concatenate([(1 - X[:, 1] ** 2) + 0.1 * inputs.normal(0, "ux", N), 0.1 * inputs.normal(0, "uy", N),
                           0.1 * inputs.normal(0, "uz", N)])
    del X
    cpb = autotune(m, 0)
    assert cpb >= 1
    y = apply_helmholtz_f64(m, _cuda(u_in), cm, nu).cpu().numpy()
    tg = sample_cells(C3["n"], count=24)
    sampled_parity(C3, k, y, u_in, tg, 1e-12, ncomp=3, mass_coef=cm, nu=nu)
    rhs = cm * apply_mass_f64(m, _cuda(u_in))
    sols = []
    for pc in ("invmass", "jacobi"):
        u, res = cg_solve(m, rhs, op="helmholtz", mass_coef=cm, nu=nu, precond=pc, rtol=1e-10, use_graph=1)
        assert res.converged
        r = rhs - apply_helmholtz_f64(m, u, cm, nu)
        assert (torch.linalg.norm(r) / torch.linalg.norm(rhs)).item() <= 1e-9
        sols.append(u)
    assert (torch.linalg.norm(sols[0] - sols[1]) / torch.linalg.norm(sols[1])).item() <= 1e-8


def test_c4_mixed_precision_neumann_48_k5():
    """FP32 Chebyshev(4) under FP64 flexible CG versus plain FP64 Jacobi CG on the
    singular Neumann channel (zero-mean rhs): both reach 1e-10, agree after the
    zero-mean projection, and the FP32 operator matches the oracle to 1e-5."""
    from paper_1607_01323_gb300 import apply_laplace_f32, apply_laplace_f64, cg_solve
    k = 5
    m = gpu_mesh(C4, k)
    N = m.n_dofs
    b = inputs.uniform(0, "b", N)
    b -= b.mean()
    tg = sample_cells(C4["n"], count=16)
    y32 = apply_laplace_f32(m, _cuda(b, torch.float32)).cpu().numpy().astype(np.float64)
    sampled_parity(C4, k, y32, b.astype(np.float32).astype(np.float64), tg, 1e-5)
    bt = _cuda(b)
    xc, rc = cg_solve(m, bt, precond="cheb_f32", cheb_degree=4, zero_mean=1, rtol=1e-10)
    xj, rj = cg_solve(m, bt, precond="jacobi", zero_mean=1, rtol=1e-10)
    assert rc.converged and rj.converged
    for x in (xc, xj):
        x = x - x.mean()
        r = bt - apply_laplace_f64(m, x)
        r = r - r.mean()
        assert (torch.linalg.norm(r) / torch.linalg.norm(bt)).item() <= 1e-9
    d = (xc - xc.mean()) - (xj - xj.mean())
    assert (torch.linalg.norm(d) / torch.linalg.norm(xj - xj.mean())).item() <= 1e-6


def test_c5_adjoint_32_k3():
    """Per-cell log-normal viscosity nu_e = exp(0.5 xi_e)/180, gamma0/dt = 1500:
    the gradient formula matches the oracle on all cells; dJ/dnu_e matches
    central finite differences on 20 seeded cells within 1e-6 relative.

    The finite difference J(nu + h e_e) - J(nu - h e_e) is evaluated without
    cancellation: with u_+- = u + d_+- and A(nu +- h e_e) d_+- =
    -(A(nu +- h e_e) - A(nu)) u (both operators applied on the GPU),
    J_+ - J_- = (d_+ - d_-)^T M (u - u_t) + 1/2 (d_+^T M d_+ - d_-^T M d_-),
    which is the same difference of the exact losses."""
    from paper_1607_01323_gb300 import adjoint_grad_nu, apply_helmholtz_f64, apply_mass_f64, cg_solve
    from paper_1607_01323_gb300.autograd import helmholtz_solve, mass_norm_loss
    k = 3
    m = gpu_mesh(C5, k)
    N, ne = m.n_dofs, m.ncell
    cm = 1500.0
    nu = np.exp(0.5 * inputs.normal(0, "xi", ne)) / 180.0
    X = m.node_coordinates()
    fc = np.sin(X[:, 0]) * np.cos(math.pi * X[:, 1] / 2) * np.sin(2 * X[:, 2])
    ph = 2 * math.pi * (0.5 * (inputs.uniform(0, "phase", 2) + 1))
    ut = _cuda(np.cos(math.pi * X[:, 1] / 2) * (1 + 0.5 * np.sin(X[:, 0] + ph[0]) * np.cos(X[:, 2] + ph[1])))
    f = apply_mass_f64(m, _cuda(fc))
    nu_t = _cuda(nu).requires_grad_(True)
    u = helmholtz_solve(m, nu_t, f, cm, rtol=1e-13)
    J = mass_norm_loss(m, u, ut)
    J.backward()
    g = nu_t.grad.cpu().numpy()
    # formula vs oracle on every cell (with the GPU's u and lambda)
    u_d = u.detach()
    lam, _ = cg_solve(m, apply_mass_f64(m, u_d - ut), op="helmholtz", mass_coef=cm, nu=0.0, nu_cell=_cuda(nu),
                      rtol=1e-13)
    g_gpu = adjoint_grad_nu(m, _cuda(nu), u_d, lam).cpu().numpy()
    assert np.max(np.abs(g - g_gpu)) <= 1e-10 * np.max(np.abs(g))
    op = SIPG(oracle_spec(C5), k)
    u_h, lam_h = u_d.cpu().numpy(), lam.cpu().numpy()
    g_orc = oadj.grad_nu(op, nu, u_h, lam_h)
    # dJ/dnu_e = -lambda^T (dA/dnu_e) u sums ~3e4 cell and face terms per cell
    # that largely cancel; any evaluation order is exact up to a small multiple
    # of the unit roundoff times the sum of the terms' absolute values
    # (|lambda|^T |dA/dnu_e| |u| from the oracle's blocks), so the two codes
    # must agree to C_ROUND eps of that sum, cell by cell
    mag = oadj.grad_nu_magnitude(op, nu, u_h, lam_h)
    ratio = np.abs(g_gpu - g_orc) / (np.finfo(np.float64).eps * mag)
    print("C5 gradient: max |g_gpu - g_orc| / (eps sum|terms|) = %.3g" % ratio.max())
    assert np.all(ratio <= C_ROUND), ratio.max()
    # central finite differences on 20 seeded cells
    cells = [int(v % np.uint64(ne)) for v in inputs.u64(0, "fd_cells", 0, 20)]
    e_t = u_d - ut
    Au = apply_helmholtz_f64(m, u_d, cm, 0.0, nu_cell=_cuda(nu))
    for e in cells:
        h = 1e-4 * nu[e]
        dJ = []
        for s in (+1, -1):
            nus = nu.copy()
            nus[e] += s * h
            nus_t = _cuda(nus)
            rhs = Au - apply_helmholtz_f64(m, u_d, cm, 0.0, nu_cell=nus_t)
            d, res = cg_solve(m, rhs, op="helmholtz", mass_coef=cm, nu=0.0, nu_cell=nus_t, rtol=1e-13)
            assert res.converged
            Md = apply_mass_f64(m, d)
            dJ.append((torch.dot(Md, e_t) + 0.5 * torch.dot(Md, d)).item())
        fd = (dJ[0] - dJ[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * abs(g[e]), (e, fd, g[e])
