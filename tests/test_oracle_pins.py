"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
a printed value of the paper, an invariant, a special case that reduces to a
textbook result, or the exact answer on a tiny case.  The ``test_mutation_*``
tests plant a plausible mistake in a copy of the oracle (on the CPU) and show
that a pin catches it.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

from oracle import adjoint, solvers
from oracle import sipg as sipg_mod
from oracle.basis import gauss_rule, gll_rule, lagrange_derivatives, lagrange_values
from oracle.mesh import DIRICHLET, NEUMANN, PERIODIC, MeshSpec, analytic_map
from oracle.sipg import SIPG

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P_, D_, N_ = PERIODIC, DIRICHLET, NEUMANN


def channel(n, wall=D_, mapping="channel", gamma=1.8, L=(2 * math.pi, 2.0, math.pi)):
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    return MeshSpec(nx, ny, nz, lo=(0.0, -L[1] / 2, 0.0), hi=(L[0], L[1] / 2, L[2]),
                    bc_lo=(P_, wall, P_), bc_hi=(P_, wall, P_), mapping=mapping, gamma=gamma)


# ------------------------------------------------------------- 1D rules
def test_gll_closed_forms():
    z, w = gll_rule(2)
    assert np.allclose(z, [0, 1]) and np.allclose(w, [0.5, 0.5])
    z, w = gll_rule(3)  # {-1, 0, 1} with weights {1/3, 4/3, 1/3} on [-1, 1]
    assert np.allclose(z, [0, 0.5, 1], atol=1e-15) and np.allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    z, w = gll_rule(4)  # +-1/sqrt(5), weights 1/6, 5/6 on [-1, 1]
    s = 1 / math.sqrt(5)
    assert np.allclose(z, [0, (1 - s) / 2, (1 + s) / 2, 1], atol=1e-15)
    assert np.allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)
    z, w = gll_rule(5)  # 0, +-sqrt(3/7); weights 1/10, 49/90, 32/45
    s = math.sqrt(3 / 7)
    assert np.allclose(z, [0, (1 - s) / 2, 0.5, (1 + s) / 2, 1], atol=1e-15)
    assert np.allclose(w, np.array([1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]) / 2, atol=1e-15)


def test_gauss_closed_forms():
    z, w = gauss_rule(2)
    s = 1 / math.sqrt(3)
    assert np.allclose(z, [(1 - s) / 2, (1 + s) / 2]) and np.allclose(w, [0.5, 0.5])
    z, w = gauss_rule(3)
    s = math.sqrt(3 / 5)
    assert np.allclose(z, [(1 - s) / 2, 0.5, (1 + s) / 2]) and np.allclose(w, [5 / 18, 8 / 18, 5 / 18])


@pytest.mark.parametrize("n", range(2, 10))
def test_rules_exactness_degree(n):
    """Gauss with n points integrates x^m exactly for m <= 2n-1 and not for 2n;
    GLL with n points for m <= 2n-3 and not for 2n-2."""
    z, w = gauss_rule(n)
    for m in range(2 * n):
        assert abs(w @ z ** m - 1 / (m + 1)) < 1e-14
    assert abs(w @ z ** (2 * n) - 1 / (2 * n + 1)) > 1e-12
    z, w = gll_rule(n)
    for m in range(2 * n - 2):
        assert abs(w @ z ** m - 1 / (m + 1)) < 1e-14
    assert abs(w @ z ** (2 * n - 2) - 1 / (2 * n - 1)) > 1e-12


@pytest.mark.parametrize("p", range(2, 9))
def test_lagrange_interpolates_and_differentiates_polynomials(p):
    z, _ = gll_rule(p)
    assert np.allclose(lagrange_values(z, z), np.eye(p), atol=1e-14)
    x = np.linspace(-0.3, 1.2, 17)
    V, D = lagrange_values(z, x), lagrange_derivatives(z, x)
    for m in range(p):
        assert np.allclose(V @ z ** m, x ** m, atol=1e-12)
        assert np.allclose(D @ z ** m, m * x ** max(m - 1, 0) if m else 0 * x, atol=1e-11)


# ------------------------------------------------------ mesh / golden
def test_channel_grading_matches_paper_table():
    """Table ch_flows prints element resolutions of the tanh-graded channel and the
    DoF count; both follow from the mapping of Sec. 7.1."""
    with open(os.path.join(GOLDEN, "channel_table.json")) as f:
        table = json.load(f)["cases"]
    for c in table:
        nx, ny, nz = c["cells"]
        k, re = c["k"], c["re_tau"]
        spec = MeshSpec(nx, ny, nz, lo=(0, -1, 0), hi=(c["L"][0], 1, c["L"][2]), bc_lo=(P_, D_, P_),
                        bc_hi=(P_, D_, P_), mapping="channel", gamma=c["gamma"])
        ys = analytic_map(spec, np.stack([np.zeros(ny + 1), np.arange(ny + 1) / ny, np.zeros(ny + 1)], -1))[:, 1]
        assert abs(ys[0] + 1) < 1e-15 and abs(ys[-1] - 1) < 1e-15
        dy = np.diff(ys)
        plus = re / (k + 1)

        def close(val, printed):
            digits = len(str(printed).split(".")[1]) if "." in str(printed) else 0
            return abs(val - printed) <= 0.5 * 10 ** (-digits) + 1e-9

        assert close(c["L"][0] / nx * plus, c["dx"]), c["name"]
        assert close(c["L"][2] / nz * plus, c["dz"]), c["name"]
        assert close(dy[0] * plus, c["dy1"]), c["name"]
        assert close(dy[ny // 2] * plus, c["dyc"]), c["name"]
        dofs = 4 * nx * ny * nz * (k + 1) ** 3
        printed = c["dofs"]
        assert abs(dofs - printed) <= 0.05 * printed, c["name"]


# ------------------------------------------------------------ penalty
def test_penalty_closed_forms():
    """Eq. (taue): on a box cell with sides hx, hy, hz, tau = (k+1)^2 (1/hx+1/hy+1/hz)
    if all faces are interior; a boundary face of area A adds (k+1)^2 A/(2V)."""
    op = SIPG(MeshSpec(4, 4, 4), 3)
    assert np.allclose(op.tau, 192.0, rtol=1e-14)  # 16 * (4 + 4 + 4)
    op = SIPG(MeshSpec(4, 4, 4), 3, penalty_factor=1 / 3)
    assert np.allclose(op.tau, 64.0, rtol=1e-14)  # (k+1)^2 / h
    spec = channel((3, 4, 2))
    op = SIPG(spec, 2)
    hx, hz = 2 * math.pi / 3, math.pi / 2
    ys = analytic_map(spec, np.stack([np.zeros(5), np.arange(5) / 4, np.zeros(5)], -1))[:, 1]
    dy = np.diff(ys)
    for iy in range(4):
        extra = 1.5 if iy in (0, 3) else 1.0
        want = 9 * (1 / hx + 1 / hz + extra / dy[iy])
        cells = [(iz * 4 + iy) * 3 + ix for ix in range(3) for iz in range(2)]
        assert np.allclose(op.tau[cells], want, rtol=1e-13)


# ----------------------------------------------------- operator invariants
CASES = [
    ("periodic box", lambda: MeshSpec(3, 2, 2, hi=(1.0, 0.7, 1.3)), 2),
    ("dirichlet channel", lambda: channel((2, 4, 2)), 3),
    ("neumann channel", lambda: channel((2, 4, 2), wall=N_), 2),
    ("dirichlet box", lambda: MeshSpec(2, 2, 2, bc_lo=(D_,) * 3, bc_hi=(D_, N_, D_)), 1),
]


@pytest.mark.parametrize("name,make,k", CASES)
def test_symmetry(name, make, k):
    op = SIPG(make(), k)
    rng = np.random.default_rng(1)
    nu_cell = np.exp(0.5 * rng.standard_normal(op.spec.ncell))
    for kw in ({}, {"mass_coef": 3.0, "nu": 0.5}, {"mass_coef": 2.0, "nu_cell": nu_cell}):
        A = op.assemble(**kw)
        nrm = abs(A).sum(axis=1).max()
        assert abs(A - A.T).max() <= 1e-14 * nrm


@pytest.mark.parametrize("name,make,k", [CASES[0], CASES[2]])
def test_nullspace_constants(name, make, k):
    op = SIPG(make(), k)
    A = op.assemble()
    nrm = abs(A).sum(axis=1).max()
    assert abs(A @ np.ones(A.shape[0])).max() <= 1e-13 * nrm


@pytest.mark.parametrize("name,make,k", CASES)
def test_positive_definite(name, make, k):
    op = SIPG(make(), k)
    ev = np.linalg.eigvalsh(op.assemble().toarray())
    nrm = abs(ev).max()
    if name in ("periodic box", "neumann channel"):
        assert abs(ev[0]) <= 1e-12 * nrm and ev[1] > 1e-6 * nrm  # positive on 1^perp
    else:
        assert ev[0] > 1e-6 * nrm


def test_positive_definite_c1_penalty_readings():
    """The 4^3 periodic cube at k=3 with tau of Eq. (taue) and with the smaller
    (k+1)^2/h: both stay positive on 1^perp."""
    for f in (1.0, 1 / 3):
        ev = np.linalg.eigvalsh(SIPG(MeshSpec(4, 4, 4), 3, penalty_factor=f).assemble().toarray())
        assert abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_brute_force_quadrature(k):
    """On affine cells every integrand has degree <= 2k per direction, so the
    (k+1)-point Gauss rule of Sec. 5 and a (k+3)-point rule give the same matrix."""
    spec = MeshSpec(2, 2, 2, hi=(1.0, 0.6, 1.7), bc_lo=(P_, D_, N_), bc_hi=(P_, D_, D_))
    rng = np.random.default_rng(k)
    nu_cell = np.exp(rng.standard_normal(8))
    a = SIPG(spec, k)
    b = SIPG(spec, k, nq=k + 3)
    for kw in ({}, {"mass_coef": 5.0, "nu_cell": nu_cell}):
        A, B = a.assemble(**kw), b.assemble(**kw)
        assert abs(A - B).max() <= 1e-13 * abs(B).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_galerkin_consistency_parabola(k):
    """u = 1 - y^2 lies in the space on the affine channel and vanishes on the
    walls; -u'' = 2, so A u = M 2 to rounding (SIPG is consistent)."""
    spec = channel((3, 4, 2), mapping="affine")
    op = SIPG(spec, k)
    y = op.node_coordinates()[..., 1].ravel()
    u = 1 - y ** 2
    lhs, rhs = op.apply(u), op.mass_apply(2 * np.ones_like(u))
    assert abs(lhs - rhs).max() <= 1e-12 * abs(rhs).max()


def test_galerkin_consistency_box_polynomial():
    """u = x(1-x) y(1-y) z(1-z) on the unit cube with Dirichlet faces (k = 2):
    A u = M f with f = -Laplace(u)."""
    op = SIPG(MeshSpec(2, 3, 2, bc_lo=(D_,) * 3, bc_hi=(D_,) * 3), 2)
    X = op.node_coordinates()
    x, y, z = X[..., 0].ravel(), X[..., 1].ravel(), X[..., 2].ravel()
    u = x * (1 - x) * y * (1 - y) * z * (1 - z)
    f = 2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z) + x * (1 - x) * y * (1 - y))
    lhs, rhs = op.apply(u), op.mass_apply(f)
    assert abs(lhs - rhs).max() <= 1e-12 * abs(rhs).max()


def test_neumann_consistency():
    """Neumann walls carry no operator term.  For the harmonic u = y on the unit
    cube (periodic in x, z; Neumann in y), integration by parts leaves only the
    wall flux: a(u, v) = int_{y=1} v dA - int_{y=0} v dA.  So a(u, 1) = 0 and
    a(u, y) = area of the top face = 1."""
    spec = MeshSpec(2, 3, 2, bc_lo=(P_, N_, P_), bc_hi=(P_, N_, P_))
    op = SIPG(spec, 2)
    y = op.node_coordinates()[..., 1].ravel()
    Ay = op.apply(y)
    assert abs(np.ones_like(y) @ Ay) < 1e-13
    assert abs(y @ Ay - 1.0) < 1e-12


@pytest.mark.parametrize("k,levels,rate", [(1, (4, 8, 16), 1.8), (2, (4, 8), 2.8), (4, (4, 8), 4.8)])
def test_convergence_manufactured(k, levels, rate):
    """Optimal L2 rate k+1 (Sec. 3.2 (iii); Sec. 6) for u = sin x cos(pi y/2) sin 2z
    on the stretched 2 pi x 2 x pi channel with Dirichlet walls."""
    ue = lambda x, y, z: np.sin(x) * np.cos(np.pi * y / 2) * np.sin(2 * z)
    fe = lambda x, y, z: (1 + np.pi ** 2 / 4 + 4) * ue(x, y, z)
    errs = []
    for n in levels:
        op = SIPG(channel(n), k)
        A = op.assemble()
        d = A.diagonal()
        u, info = spla.cg(A, op.load_vector(fe), rtol=1e-12, maxiter=20000,
                          M=spla.LinearOperator(A.shape, matvec=lambda r: r / d))
        assert info == 0
        errs.append(op.l2_error(u, ue))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= rate, (errs, rates)


# ------------------------------------------------------- mass operators
def test_mass_volume_and_inverse():
    spec = channel((3, 4, 2))
    op = SIPG(spec, 3)
    one = np.ones(spec.ncell * op.P)
    assert abs(one @ op.mass_apply(one) - 2 * math.pi * 2 * math.pi) < 1e-12
    x = np.random.default_rng(0).uniform(-1, 1, (2, one.size))
    assert abs(op.mass_apply(op.inverse_mass_apply(x)) - x).max() < 1e-13
    # the mass matrix is the k+1-point Gauss rule: for k+1 points the 1D Gauss
    # mass of a GLL basis is not diagonal (Sec. 5)
    assert abs(op.geom[0].M - np.diag(np.diag(op.geom[0].M))).max() > 1e-3


def test_helmholtz_is_mass_plus_laplace():
    spec = channel((2, 4, 2))
    op = SIPG(spec, 2)
    x = np.random.default_rng(3).standard_normal(spec.ncell * op.P)
    assert np.allclose(op.apply(x, mass_coef=1500.0, nu=1 / 180),
                       1500.0 * op.mass_apply(x) + op.apply(x) / 180, rtol=1e-13, atol=1e-12)


def test_diagonal_matches_assembled():
    op = SIPG(channel((2, 4, 2)), 3)
    nu_cell = np.exp(np.random.default_rng(2).standard_normal(16))
    for kw in ({}, {"mass_coef": 7.0, "nu_cell": nu_cell}):
        assert np.allclose(op.diagonal(**kw), op.assemble(**kw).diagonal(), rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------- solvers
def test_chebyshev_residual_polynomial():
    """For A = diag(lambda), D = I and x0 = 0, Chebyshev with d steps leaves the
    error e_d(lambda) = x* T_d((theta - lambda)/delta) / T_d(theta/delta)."""
    lam = np.linspace(1.0, 10.0, 37)
    xs = np.random.default_rng(5).standard_normal(lam.size)
    lmin, lmax = 0.8, 11.0
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    for d in range(1, 7):
        x = solvers.chebyshev(lambda v: lam * v, np.ones_like(lam), lam * xs, d, lmin, lmax)
        Td = C.Chebyshev.basis(d)
        want = xs * Td((theta - lam) / delta) / Td(theta / delta)
        assert np.allclose(xs - x, want, atol=1e-13)


def test_cg_and_lanczos():
    op = SIPG(channel((2, 4, 2)), 2)
    A = op.assemble()
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    d = A.diagonal()
    x_direct = spla.spsolve(A.tocsc(), b)
    for flexible in (False, True):
        x, it, rel = solvers.cg(lambda v: A @ v, b, rtol=1e-12, precond=lambda r: r / d, flexible=flexible)
        assert rel <= 1e-12 and np.linalg.norm(x - x_direct) <= 1e-8 * np.linalg.norm(x_direct)
    dinv_a = (A.toarray() / d[:, None])
    lmax = np.max(np.linalg.eigvals(dinv_a).real)
    est = solvers.lanczos_max_eig(lambda v: A @ v, d, b, steps=40)
    assert est <= lmax * (1 + 1e-10) and est >= 0.98 * lmax


def test_zero_mean_singular_solve():
    op = SIPG(channel((2, 4, 2), wall=N_), 2)
    A = op.assemble()
    b = np.random.default_rng(6).uniform(-1, 1, A.shape[0])
    x, it, rel = solvers.cg(lambda v: A @ v, b, rtol=1e-10, zero_mean=True, precond=lambda r: r / A.diagonal())
    bp = b - b.mean()
    assert np.linalg.norm(A @ x - bp) <= 1e-9 * np.linalg.norm(bp)


# -------------------------------------------------------------- adjoint
def test_adjoint_gradient_finite_differences():
    spec = channel((2, 4, 2))
    op = SIPG(spec, 2)
    rng = np.random.default_rng(7)
    # mass coefficient 1 and nu = O(1): J depends strongly on nu, so central
    # differences with a relative step 1e-4 are accurate to ~1e-8
    nu = np.exp(0.5 * rng.standard_normal(spec.ncell))
    cm = 1.0
    X = op.node_coordinates()
    f = op.mass_apply(np.sin(X[..., 0]).ravel() * np.cos(np.pi * X[..., 1].ravel() / 2))
    ut = np.cos(np.pi * X[..., 1].ravel() / 2) * (1 + 0.5 * np.cos(X[..., 2].ravel()))

    def solve(nuc):
        A = op.assemble(mass_coef=cm, nu_cell=nuc)
        return spla.spsolve(A.tocsc(), f)

    u = solve(nu)
    A = op.assemble(mass_coef=cm, nu_cell=nu)
    lam = spla.spsolve(A.tocsc(), op.mass_apply(u - ut))
    g = adjoint.grad_nu(op, nu, u, lam)
    for e in range(spec.ncell):
        h = 1e-4 * nu[e]
        nup, num = nu.copy(), nu.copy()
        nup[e] += h
        num[e] -= h
        fd = (adjoint.loss(op, solve(nup), ut) - adjoint.loss(op, solve(num), ut)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * abs(g).max(), (e, fd, g[e])


def _dA_dnu(op, nu, e, cm=1.0):
    """dA/dnu_e of the assembled operator by a central difference (A is linear in
    nu_e while the max of each face stays on the same side: exact to rounding)."""
    h = 1e-3 * nu[e]
    nup, num = nu.copy(), nu.copy()
    nup[e] += h
    num[e] -= h
    return ((op.assemble(mass_coef=cm, nu_cell=nup) - op.assemble(mass_coef=cm, nu_cell=num)) / (2 * h)).toarray()


def test_adjoint_term_magnitude_bounds():
    """|lambda|^T |dA/dnu_e| |u| summed block by block bounds the gradient
    (|-lambda^T dA/dnu_e u| <= it) and the entrywise absolute value of the
    assembled derivative (|lambda|^T |dA/dnu_e| |u| <= it), both computed here
    from the assembled matrix; it is homogeneous in lambda and u."""
    spec = channel((2, 4, 2))
    op = SIPG(spec, 2)
    rng = np.random.default_rng(8)
    nu = np.exp(0.5 * rng.standard_normal(spec.ncell))
    u = rng.uniform(-1, 1, spec.ncell * op.P)
    lam = rng.uniform(-1, 1, spec.ncell * op.P)
    gm = adjoint.grad_nu_magnitude(op, nu, u, lam)
    assert np.all(gm > 0)
    assert np.allclose(adjoint.grad_nu_magnitude(op, nu, -3.0 * u, 0.5 * lam), 1.5 * gm, rtol=1e-14)
    for e in range(spec.ncell):
        dA = _dA_dnu(op, nu, e)
        assert abs(lam @ dA @ u) <= gm[e] * (1 + 1e-9)
        assert np.abs(lam) @ np.abs(dA) @ np.abs(u) <= gm[e] * (1 + 1e-9), e


def test_adjoint_term_magnitude_single_neumann_cell():
    """One cell with Neumann faces only: dA/dnu_e is the cell stiffness alone,
    and the magnitude equals |lambda|^T |dA/dnu_e| |u| exactly."""
    spec = MeshSpec(1, 1, 1, hi=(1.0, 0.8, 1.3), bc_lo=(N_,) * 3, bc_hi=(N_,) * 3)
    op = SIPG(spec, 3)
    rng = np.random.default_rng(9)
    nu = np.array([0.7])
    u, lam = rng.uniform(-1, 1, op.P), rng.uniform(-1, 1, op.P)
    dA = _dA_dnu(op, nu, 0)
    ref = np.abs(lam) @ np.abs(dA) @ np.abs(u)
    assert abs(adjoint.grad_nu_magnitude(op, nu, u, lam)[0] - ref) <= 1e-9 * ref


# ------------------------------------------------------------ mutations
def test_mutation_average_weight_caught(monkeypatch):
    """Dropping the 1/2 of the average {{grad u}} breaks Galerkin consistency."""
    orig = sipg_mod.SIPG.face_pieces

    def wrong(self, d, km, kp):
        cu, cv, pen = orig(self, d, km, kp)
        return [[2 * c for c in row] for row in cu], [[2 * c for c in row] for row in cv], pen

    monkeypatch.setattr(sipg_mod.SIPG, "face_pieces", wrong)
    op = SIPG(channel((3, 4, 2), mapping="affine"), 2)
    y = op.node_coordinates()[..., 1].ravel()
    assert abs(op.apply(1 - y ** 2) - op.mass_apply(2 + 0 * y)).max() > 1e-3


def test_mutation_jump_sign_caught(monkeypatch):
    """Using [u] = u^- + u^+ breaks the constant nullspace of the periodic operator."""
    monkeypatch.setattr(sipg_mod, "SIGMA", (1.0, 1.0))
    op = SIPG(MeshSpec(3, 2, 2), 2)
    A = op.assemble()
    assert abs(A @ np.ones(A.shape[0])).max() > 1e-3


def test_mutation_penalty_degree_caught():
    """A penalty with k^2 instead of (k+1)^2 differs from the closed form 192."""
    op = SIPG(MeshSpec(4, 4, 4), 3, penalty_factor=9 / 16)
    assert not np.allclose(op.tau, 192.0)
