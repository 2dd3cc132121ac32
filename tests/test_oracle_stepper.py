"""Pins of the oracle's dual-splitting step (Sec. 2.2, variant V3c): the
BDF / extrapolation constants by their exactness on polynomials, the pressure
Neumann data of Eq. (ipflux) against the analytic div(u (x) u) + nu curl curl u
on polynomial fields, two exact discrete steady states (Poiseuille flow driven
by a body force; a hydrostatic pressure balancing a body force, which
exercises the wall data and the pressure gradient), and the temporal orders on
the Taylor-Green vortex, an exact Navier-Stokes solution."""
import math

import numpy as np
import pytest

from oracle.mesh import DIRICHLET, PERIODIC, MeshSpec, cell_node_coords
from oracle.stepper import BDF_EX, DualSplitting, pressure_spec

P_, D_ = PERIODIC, DIRICHLET


@pytest.mark.parametrize("J", [1, 2, 3])
def test_bdf_ex_constants(J):
    """(gamma0 y(t_n+1) - sum alpha_i y(t_n-i)) / dt = y'(t_n+1) for polynomials
    of degree <= J, and sum beta_i y(t_n-i) = y(t_n+1) for degree <= J-1."""
    g0, a, b = BDF_EX[J]
    t = np.array([1.0 - i for i in range(J)])  # t_n, t_n-1, ...; t_n+1 = 2, dt = 1
    for m in range(J + 1):
        lhs = g0 * 2.0 ** m - sum(ai * ti ** m for ai, ti in zip(a, t))
        assert abs(lhs - (m * 2.0 ** (m - 1) if m else 0.0)) <= 1e-13
    for m in range(J):
        assert abs(sum(bi * ti ** m for bi, ti in zip(b, t)) - 2.0 ** m) <= 1e-13
    # one order more is not exact
    m = J + 1
    assert abs(g0 * 2.0 ** m - sum(ai * ti ** m for ai, ti in zip(a, t)) - m * 2.0 ** (m - 1)) > 1e-3


def _box(n=(2, 2, 2), k=3):
    return MeshSpec(*n, lo=(0.0, -1.0, 0.0), hi=(1.5, 1.0, 1.2), bc_lo=(P_, D_, P_), bc_hi=(P_, D_, P_))


def test_pressure_spec():
    ps = pressure_spec(_box())
    assert ps.bc_lo == (P_, "neumann", P_) and ps.bc_hi == (P_, "neumann", P_)
    with pytest.raises(ValueError):
        pressure_spec(MeshSpec(1, 1, 1, bc_lo=(P_, "neumann", P_), bc_hi=(P_, "neumann", P_)))


def test_wall_values_polynomial():
    """u in Q_3 on affine cells: the L2-projected vorticity is curl u exactly,
    so the wall data equal (div(u (x) u) + nu curl curl u) . n at the points."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    U = sympy.Matrix([x * y ** 2 + z ** 3, y ** 3 - x * z + x ** 2, x ** 2 * y + z ** 2 * y])
    X = [x, y, z]
    nu = 0.3
    divF = sympy.Matrix([sum(sympy.diff(U[i] * U[j], X[j]) for j in range(3)) for i in range(3)])

    def curl(V):
        return sympy.Matrix([sympy.diff(V[2], y) - sympy.diff(V[1], z), sympy.diff(V[0], z) - sympy.diff(V[2], x),
                             sympy.diff(V[1], x) - sympy.diff(V[0], y)])

    D = sympy.lambdify((x, y, z), divF + nu * curl(curl(U)), "numpy")
    Uf = sympy.lambdify((x, y, z), U, "numpy")
    k = 3
    spec = _box()
    ds = DualSplitting(spec, k, nu, 0.1, order=1)
    Xn = ds.sipg.node_coordinates()
    u = np.stack([np.broadcast_to(np.asarray(Uf(Xn[..., 0], Xn[..., 1], Xn[..., 2])[i][0], dtype=float),
                                  Xn.shape[:2]) for i in range(3)]).ravel()
    vals = ds.wall_values(u)
    assert len(vals) == 2 * spec.nx * spec.nz
    worst = 0.0
    for (e, d, side), v in zip(ds.walls, vals):
        n, wA, phif, _ = ds.visc._cq(e).face[(d, side)]
        xq = phif @ cell_node_coords(spec, k + 1, [e])[0]
        ref = np.einsum("iq,qi->q", np.array([np.broadcast_to(np.asarray(c[0], dtype=float), xq.shape[:1])
                                              for c in D(xq[:, 0], xq[:, 1], xq[:, 2])]), n)
        worst = max(worst, np.abs(v - ref).max() / max(1.0, np.abs(ref).max()))
    assert worst <= 1e-11


def _nodal(ds, fx, fy, fz):
    X = ds.sipg.node_coordinates()
    return np.concatenate([fx(X).ravel(), fy(X).ravel(), fz(X).ravel()])


def test_poiseuille_is_a_steady_state():
    """u = (1 - y^2, 0, 0) with f = (2 nu, 0, 0) between no-slip walls at
    y = -1, 1: zero convective term, zero divergence, zero wall data; the
    viscous step returns u (exact on affine cells, degree 2 <= k)."""
    nu, dt = 0.05, 0.1
    ds = DualSplitting(_box((2, 3, 2)), 3, nu, dt, order=3, zeta=1.0)
    u0 = _nodal(ds, lambda X: 1 - X[..., 1] ** 2, lambda X: 0 * X[..., 0], lambda X: 0 * X[..., 0])
    ds.set_history([u0])
    for s in range(4):
        u, p, info = ds.step(f=(2 * nu, 0.0, 0.0))
        assert info["order"] == min(s + 1, 3)
        assert np.abs(u - u0).max() <= 1e-10
        assert np.abs(p).max() <= 1e-9


def test_hydrostatic_pressure_is_a_steady_state():
    """u = 0 and f = (0, c, 0): the wall data f . n drive p = c y (up to the
    mean), whose gradient cancels f in the projection; u stays zero.  A sign
    error in the wall data or in the gradient leaves a velocity."""
    c = 0.7
    ds = DualSplitting(_box((2, 3, 2)), 3, 0.05, 0.1, order=2, zeta=1.0)
    N = ds.N
    ds.set_history([np.zeros(3 * N)])
    Y = ds.sipg.node_coordinates()[..., 1].ravel()
    pe = c * Y - np.mean(c * Y)
    for s in range(3):
        u, p, info = ds.step(f=(0.0, c, 0.0))
        assert np.abs(u).max() <= 1e-11
        assert np.abs(p - pe).max() <= 1e-10


def _tgv(X, t, nu):
    x, y = X[..., 0], X[..., 1]
    F = math.exp(-2 * nu * t)
    return np.concatenate([(np.sin(x) * np.cos(y) * F).ravel(), (-np.cos(x) * np.sin(y) * F).ravel(),
                           np.zeros(x.size)])


def _tgv_p(X, t, nu):
    x, y = X[..., 0], X[..., 1]
    p = ((np.cos(2 * x) + np.cos(2 * y)) / 4 * math.exp(-4 * nu * t)).ravel()
    return p - p.mean()


def test_taylor_green_temporal_orders():
    """Taylor-Green vortex on the periodic [0, 2 pi]^2 x [0, 1] (4 x 4 x 1 cells,
    k = 5, nu = 0.1, T = 1), older levels from the exact solution: BDF2 velocity
    error falls by ~2^1.8 per halving of dt, BDF3 pressure error by ~2^3."""
    nu, T = 0.1, 1.0
    spec = MeshSpec(4, 4, 1, hi=(2 * math.pi, 2 * math.pi, 1.0))
    ds = DualSplitting(spec, 5, nu, 0.5, order=2, zeta=0.0)
    X = ds.sipg.node_coordinates()
    ue, pe = _tgv(X, T, nu), _tgv_p(X, T, nu)
    err = {}
    for J in (2, 3):
        ds.order = J
        for Nst in (2, 4):
            dt = T / Nst
            ds.reset(dt)
            ds.set_history([_tgv(X, -i * dt, nu) for i in range(J)])
            for _ in range(Nst):
                u, p, info = ds.step()
            err[(J, Nst)] = (np.abs(u - ue).max(), np.abs(p - p.mean() - pe).max())
    assert math.log2(err[(2, 2)][0] / err[(2, 4)][0]) >= 1.6
    assert math.log2(err[(3, 2)][1] / err[(3, 4)][1]) >= 2.6
    assert err[(3, 4)][0] <= 2e-5 and err[(3, 4)][1] <= 1e-3


def test_shear_wave_between_walls_temporal_orders():
    """u = (cos(pi y / 2) exp(-nu pi^2 t / 4), 0, 0) between no-slip walls at
    y = -1, 1 is an exact solution with constant pressure: the split step is
    then the BDF-J scheme for the heat equation, of order J, walls included
    (1 x 4 x 1 affine cells, k = 5, nu = 0.5, T = 1, older levels exact)."""
    nu, T = 0.5, 1.0
    spec = MeshSpec(1, 4, 1, lo=(0.0, -1.0, 0.0), hi=(1.0, 1.0, 1.0), bc_lo=(P_, D_, P_), bc_hi=(P_, D_, P_))
    ds = DualSplitting(spec, 5, nu, 0.25, order=2, zeta=1.0)
    X = ds.sipg.node_coordinates().reshape(-1, 3)
    lam = nu * math.pi ** 2 / 4

    def ue(t):
        return np.concatenate([np.cos(math.pi * X[:, 1] / 2) * math.exp(-lam * t), 0 * X[:, 0], 0 * X[:, 0]])

    err = {}
    for J in (2, 3):
        ds.order = J
        for Nst in (4, 8):
            dt = T / Nst
            ds.reset(dt)
            ds.set_history([ue(-i * dt) for i in range(J)])
            for _ in range(Nst):
                u, p, _ = ds.step()
            err[(J, Nst)] = np.abs(u - ue(T)).max()
            assert np.abs(p - p.mean()).max() <= 1e-8  # constant pressure
    assert math.log2(err[(2, 4)] / err[(2, 8)]) >= 1.8
    assert math.log2(err[(3, 4)] / err[(3, 8)]) >= 2.8
    assert err[(3, 8)] <= 1e-3
