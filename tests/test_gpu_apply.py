"""GPU parity of the operator kernels against the CPU oracle, element by element.

Bar (from the method's precision): FP64 applies within 1e-12 ||A||_inf ||x||_inf
in the max norm; FP32 applies within 1e-5 in the same scaled sense.  Meshes
span several cell tiles of a thread block and ragged tails, every degree
1..7, every boundary kind, periodic self-neighbours, and per-cell viscosity.
"""
import math

import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, ncell, oracle_spec, scaled_err, uniform
from oracle.sipg import SIPG
from paper_1607_01323_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5

CASES = [
    ("c1_periodic_cube_k3", case((4, 4, 4)), 3, 1.0),
    ("c1_penalty_third", case((4, 4, 4)), 3, 1.0 / 3.0),
    ("box_mixed_bc_k2", case((3, 2, 5), hi=(1.0, 0.7, 1.3), bc_lo=("dirichlet", "neumann", "periodic"),
                             bc_hi=("dirichlet", "dirichlet", "periodic")), 2, 1.0),
    ("channel_k1", channel((3, 4, 2)), 1, 1.0),
    ("channel_k2", channel((2, 4, 3)), 2, 1.0),
    ("channel_k4", channel((3, 5, 2)), 4, 1.0),
    ("channel_k5", channel((2, 4, 2)), 5, 1.0),
    ("channel_k6", channel((2, 4, 1)), 6, 1.0),
    ("channel_k7", channel((1, 4, 2)), 7, 1.0),
    ("neumann_channel_k3", channel((3, 4, 3), wall="neumann"), 3, 1.0),
    ("single_periodic_cell_k3", case((1, 1, 1)), 3, 1.0),
    ("all_dirichlet_k3", case((2, 3, 2), bc_lo=("dirichlet",) * 3, bc_hi=("dirichlet",) * 3), 3, 1.0),
    # straight cells on graded vertices (coarse multigrid levels), down to one cell
    ("channel_linear_k3", dict(channel((2, 4, 2)), mapping="channel_linear"), 3, 1.0),
    ("channel_linear_single_cell_k4", dict(channel((1, 1, 1)), mapping="channel_linear"), 4, 1.0),
    ("channel_linear_pair_k2", dict(channel((2, 2, 2), wall="neumann"), mapping="channel_linear"), 2, 1.0),
]


def _cuda(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,c,k,pen", CASES, ids=[x[0] for x in CASES])
def test_laplace_f64_parity(name, c, k, pen):
    from paper_1607_01323_gb300 import apply_laplace_f64
    op = SIPG(oracle_spec(c), k, penalty_factor=pen)
    m = gpu_mesh(c, k, penalty=pen)
    N = m.n_dofs
    assert N == ncell(c) * (k + 1) ** 3
    ncomp = 2
    x = uniform(ncomp * N, "x")
    A = op.assemble()
    y_ref = np.concatenate([A @ x[i * N:(i + 1) * N] for i in range(ncomp)])
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    norm_a = abs(A).sum(axis=1).max()
    assert scaled_err(y, y_ref, norm_a, x) <= TOL64


@pytest.mark.parametrize("name,c,k,pen", CASES, ids=[x[0] for x in CASES])
def test_laplace_f64_double_float_parity(name, c, k, pen):
    """The FP64 operator evaluated in double-float arithmetic (FP32 pairs) meets
    the same 1e-12 bar as native FP64."""
    from paper_1607_01323_gb300 import apply_helmholtz_f64, apply_laplace_f64
    op = SIPG(oracle_spec(c), k, penalty_factor=pen)
    m = gpu_mesh(c, k, penalty=pen)
    m.set_f64_arithmetic("double_float")
    N = m.n_dofs
    x = uniform(2 * N, "x")
    A = op.assemble()
    y_ref = np.concatenate([A @ x[:N], A @ x[N:]])
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    assert scaled_err(y, y_ref, abs(A).sum(axis=1).max(), x) <= TOL64
    cm, nu = 1500.0, 1.0 / 180.0
    H = op.assemble(mass_coef=cm, nu=nu)
    y = apply_helmholtz_f64(m, _cuda(x[:N]), cm, nu).cpu().numpy()
    assert scaled_err(y, H @ x[:N], abs(H).sum(axis=1).max(), x[:N]) <= TOL64


@pytest.mark.parametrize("k", [2, 3, 5])
def test_helmholtz_nu_cell_and_mass_double_float(k):
    """Per-cell viscosity and mass-only applies in double-float keep the 1e-12 bar."""
    from paper_1607_01323_gb300 import apply_helmholtz_f64, apply_mass_f64
    c = channel((3, 4, 2))
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic("double_float")
    N = m.n_dofs
    x = uniform(N, "x")
    nu_cell = np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0
    A = op.assemble(mass_coef=1500.0, nu_cell=nu_cell)
    y = apply_helmholtz_f64(m, _cuda(x), 1500.0, 0.0, nu_cell=_cuda(nu_cell)).cpu().numpy()
    assert scaled_err(y, A @ x, abs(A).sum(axis=1).max(), x) <= TOL64
    Mm = op.assemble(mass_coef=1.0, stiffness=False)
    ym = apply_mass_f64(m, _cuda(x)).cpu().numpy()
    assert scaled_err(ym, Mm @ x, abs(Mm).sum(axis=1).max(), x) <= TOL64


def test_double_float_dynamic_range():
    """Inputs spanning many orders of magnitude (and exact zeros) keep the
    1e-12 scaled bar in double-float."""
    from paper_1607_01323_gb300 import apply_laplace_f64
    c = channel((3, 4, 2))
    k = 4
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic("double_float")
    x = uniform(m.n_dofs, "x") * 10.0 ** (8 * uniform(m.n_dofs, "exp"))
    x[::7] = 0.0
    A = op.assemble()
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    assert scaled_err(y, A @ x, abs(A).sum(axis=1).max(), x) <= TOL64


# magnitudes across the FP64 range: subnormals, far below and far above the
# FP32 exponent range, and a vector mixing 1e-150 with 1e150
EXTREME = [("subnormal", 1e-310), ("1e-200", 1e-200), ("1e-30", 1e-30), ("1e30", 1e30), ("1e200", 1e200),
           ("mixed_1e-150_1e150", None)]


@pytest.mark.parametrize("name,scale", EXTREME, ids=[e[0] for e in EXTREME])
def test_double_float_extreme_magnitudes(name, scale):
    """The double-float evaluation scales each call's input by a power of two,
    so FP64 data anywhere in the FP64 range keep the 1e-12 bar (Laplace,
    Helmholtz, per-cell viscosity, inverse mass), like native FP64."""
    from paper_1607_01323_gb300 import apply_helmholtz_f64, apply_inverse_mass_f64, apply_laplace_f64
    c = channel((3, 4, 2))
    k = 4
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic("double_float")
    N = m.n_dofs
    x = uniform(N, "x")
    if scale is None:
        x[::2] *= 1e-150
        x[1::2] *= 1e150
    else:
        x = x * scale
    A = op.assemble()
    y = apply_laplace_f64(m, _cuda(x)).cpu().numpy()
    assert np.all(np.isfinite(y))
    assert scaled_err(y, A @ x, abs(A).sum(axis=1).max(), x) <= TOL64
    cm, nu = 1500.0, 1.0 / 180.0
    H = op.assemble(mass_coef=cm, nu=nu)
    yh = apply_helmholtz_f64(m, _cuda(x), cm, nu).cpu().numpy()
    assert scaled_err(yh, H @ x, abs(H).sum(axis=1).max(), x) <= TOL64
    nu_cell = np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0
    Hc = op.assemble(mass_coef=cm, nu_cell=nu_cell)
    yc = apply_helmholtz_f64(m, _cuda(x), cm, 0.0, nu_cell=_cuda(nu_cell)).cpu().numpy()
    assert scaled_err(yc, Hc @ x, abs(Hc).sum(axis=1).max(), x) <= TOL64
    yi = apply_inverse_mass_f64(m, _cuda(x)).cpu().numpy()
    yi_ref = op.inverse_mass_apply(x)
    assert np.max(np.abs(yi - yi_ref)) <= 1e-12 * np.max(np.abs(yi_ref))


def test_double_float_nonfinite_inputs_propagate():
    """NaN and +-inf in the input give non-finite outputs in double-float,
    exactly where native FP64 gives them (same data flow); the other outputs
    keep the 1e-12 bar."""
    from paper_1607_01323_gb300 import apply_inverse_mass_f64, apply_laplace_f64
    c = channel((3, 4, 2))
    k = 3
    op = SIPG(oracle_spec(c), k)
    m64 = gpu_mesh(c, k)
    mdf = gpu_mesh(c, k)
    mdf.set_f64_arithmetic("double_float")
    N = m64.n_dofs
    A = op.assemble()
    norm_a = abs(A).sum(axis=1).max()
    for bad in ([(5, np.nan)], [(200, np.inf)], [(7, -np.inf), (N - 3, np.nan)]):
        x = uniform(N, "x")
        for i, v in bad:
            x[i] = v
        for f in (apply_laplace_f64, apply_inverse_mass_f64):
            y64 = f(m64, _cuda(x)).cpu().numpy()
            ydf = f(mdf, _cuda(x)).cpu().numpy()
            assert not np.all(np.isfinite(ydf))
            np.testing.assert_array_equal(np.isfinite(ydf), np.isfinite(y64))
            fin = np.isfinite(y64)
            xf = np.where(np.isfinite(x), x, 0.0)
            assert np.max(np.abs(ydf[fin] - y64[fin])) <= TOL64 * norm_a * np.max(np.abs(xf)) * 2


def test_double_float_cg_nonfinite_initial_guess():
    """A NaN in the initial guess of a double-float CG solve reaches the
    residual (A x0 is NaN there) and the solve returns SIPG_NONFINITE."""
    from paper_1607_01323_gb300 import cg_solve
    from paper_1607_01323_gb300 import _lib as L
    m = gpu_mesh(channel((3, 4, 2)), 3)
    m.set_f64_arithmetic("double_float")
    b = _cuda(uniform(m.n_dofs, "b"))
    for bad in (float("nan"), float("inf")):
        x0 = torch.zeros_like(b)
        x0[11] = bad
        _, r = cg_solve(m, b, x0, raise_on_fail=False)
        assert r.status == L.NONFINITE
    x, r = cg_solve(m, b)  # the context is still usable afterwards
    assert r.converged


def test_double_float_rejects_out_of_range_coefficients():
    """Scalar coefficients outside [2^-100, 2^100] cannot be held in double-float
    (FP32 exponents): the call is refused instead of computing a wrong result."""
    from paper_1607_01323_gb300 import SipgError, apply_helmholtz_f64
    m = gpu_mesh(channel((2, 2, 2)), 2)
    m.set_f64_arithmetic("double_float")
    x = _cuda(uniform(m.n_dofs, "x"))
    for cm, nu in ((1e35, 1.0), (1.0, 1e-35), (1e-40, 1.0)):
        with pytest.raises(SipgError):
            apply_helmholtz_f64(m, x, cm, nu)
    m.set_f64_arithmetic("native")
    assert torch.all(torch.isfinite(apply_helmholtz_f64(m, x, 1e35, 1.0)))


@pytest.mark.parametrize("arith", ["native", "double_float"])
@pytest.mark.parametrize("cpb", [1, 3, 5, 7])
def test_laplace_ragged_tiles(cpb, arith):
    """Cells per block that do not divide the cell count leave a ragged last tile."""
    from paper_1607_01323_gb300 import apply_laplace_f32, apply_laplace_f64
    c = channel((3, 4, 3))
    k = 3
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic(arith)
    m.set_cells_per_block(0, cpb)
    m.set_cells_per_block(1, cpb)
    x = uniform(m.n_dofs, "x")
    A = op.assemble()
    norm_a = abs(A).sum(axis=1).max()
    assert scaled_err(apply_laplace_f64(m, _cuda(x)).cpu().numpy(), A @ x, norm_a, x) <= TOL64
    x32 = x.astype(np.float32)
    y32 = apply_laplace_f32(m, _cuda(x32, torch.float32)).cpu().numpy()
    assert scaled_err(y32, A @ x32.astype(np.float64), norm_a, x) <= TOL32


@pytest.mark.parametrize("mapping", ["plane", "line"])
@pytest.mark.parametrize("name,c,k,pen", CASES[:1] + CASES[2:10], ids=[x[0] for x in CASES[:1] + CASES[2:10]])
def test_laplace_f32_parity(name, c, k, pen, mapping):
    from paper_1607_01323_gb300 import apply_laplace_f32
    op = SIPG(oracle_spec(c), k, penalty_factor=pen)
    m = gpu_mesh(c, k, penalty=pen)
    m.set_f32_mapping(mapping)
    x = uniform(m.n_dofs, "x").astype(np.float32)
    A = op.assemble()
    y = apply_laplace_f32(m, _cuda(x, torch.float32)).cpu().numpy().astype(np.float64)
    assert scaled_err(y, A @ x.astype(np.float64), abs(A).sum(axis=1).max(), x) <= TOL32


@pytest.mark.parametrize("k", [2, 3, 5])
def test_helmholtz_f64_parity(k):
    from paper_1607_01323_gb300 import apply_helmholtz_f32, apply_helmholtz_f64
    c = channel((3, 4, 2))
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    N = m.n_dofs
    x = uniform(3 * N, "u")
    cm, nu = 1500.0, 1.0 / 180.0
    A = op.assemble(mass_coef=cm, nu=nu)
    y_ref = np.concatenate([A @ x[i * N:(i + 1) * N] for i in range(3)])
    y = apply_helmholtz_f64(m, _cuda(x), cm, nu).cpu().numpy()
    norm_a = abs(A).sum(axis=1).max()
    assert scaled_err(y, y_ref, norm_a, x) <= TOL64
    for mapping in ("plane", "line"):
        m.set_f32_mapping(mapping)
        y32 = apply_helmholtz_f32(m, _cuda(x, torch.float32), cm, nu).cpu().numpy()
        assert scaled_err(y32, y_ref, norm_a, x) <= TOL32
    # per-cell viscosity nu_e = exp(0.5 xi_e) / 180
    nu_cell = np.exp(0.5 * inputs.normal(0, "xi", m.ncell)) / 180.0
    A = op.assemble(mass_coef=cm, nu_cell=nu_cell)
    y = apply_helmholtz_f64(m, _cuda(x[:N]), cm, 0.0, nu_cell=_cuda(nu_cell)).cpu().numpy()
    assert scaled_err(y, A @ x[:N], abs(A).sum(axis=1).max(), x[:N]) <= TOL64


def test_mass_inverse_mass_diagonal():
    from paper_1607_01323_gb300 import apply_inverse_mass_f64, apply_mass_f64, diagonal_f64
    # the last three have one cell across periodic directions (self-coupled faces)
    for c, k in [(channel((3, 4, 2)), 3), (case((2, 3, 2), bc_lo=("dirichlet",) * 3, bc_hi=("neumann",) * 3), 5),
                 (case((1, 1, 1)), 3), (case((1, 2, 3), hi=(0.5, 1.0, 2.0)), 2),
                 (dict(channel((1, 1, 1)), mapping="channel_linear"), 4)]:
        op = SIPG(oracle_spec(c), k)
        m = gpu_mesh(c, k)
        N = m.n_dofs
        x = uniform(2 * N, "x")
        Mref = op.assemble(mass_coef=1.0, stiffness=False)
        nm = abs(Mref).sum(axis=1).max()
        ym = apply_mass_f64(m, _cuda(x)).cpu().numpy()
        assert scaled_err(ym, np.concatenate([Mref @ x[:N], Mref @ x[N:]]), nm, x) <= TOL64
        yi = apply_inverse_mass_f64(m, _cuda(x)).cpu().numpy()
        yi_ref = op.inverse_mass_apply(x)
        assert np.max(np.abs(yi - yi_ref)) <= 1e-12 * np.max(np.abs(yi_ref))
        d = diagonal_f64(m).cpu().numpy()
        assert np.allclose(d, op.diagonal(), rtol=1e-13, atol=0)
        nu_cell = np.exp(0.5 * inputs.normal(1, "xi", m.ncell)) / 180.0
        d = diagonal_f64(m, "helmholtz", 1500.0, 0.0, nu_cell=_cuda(nu_cell)).cpu().numpy()
        assert np.allclose(d, op.diagonal(mass_coef=1500.0, nu_cell=nu_cell), rtol=1e-13, atol=0)


@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_inverse_mass_double_float(k):
    """The tensorial inverse mass in double-float arithmetic matches the oracle's
    per-element Cholesky solve to 1e-12 (relative to the largest output)."""
    from paper_1607_01323_gb300 import apply_inverse_mass_f64
    c = channel((3, 4, 2))
    op = SIPG(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic("double_float")
    x = uniform(2 * m.n_dofs, "x")
    y = apply_inverse_mass_f64(m, _cuda(x)).cpu().numpy()
    y_ref = op.inverse_mass_apply(x)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))


def test_autotune_json_cache(tmp_path):
    """The autotuner's choice goes to a JSON cache keyed by degree, precision,
    map, mesh size and arithmetic; a second mesh reads it back (same cells per
    block and FP32 thread mapping) without re-timing; results stay at parity."""
    import json
    from paper_1607_01323_gb300 import apply_laplace_f32, apply_laplace_f64, autotune
    c = channel((6, 4, 3))
    k = 3
    cache = str(tmp_path / "tune.json")
    m = gpu_mesh(c, k)
    c0 = autotune(m, 0, cache)
    c1 = autotune(m, 1, cache)
    m.set_f64_arithmetic("double_float")
    c2 = autotune(m, 0, cache)
    data = json.load(open(cache))
    assert len(data) == 3 and all(set(v) == {"cpb", "mapping"} for v in data.values())
    assert {v["cpb"] for v in data.values()} >= {c0}
    m2 = gpu_mesh(c, k)
    assert autotune(m2, 0, cache) == c0 and autotune(m2, 1, cache) == c1
    assert m2.cells_per_block(1) == m.cells_per_block(1)
    m2.set_f64_arithmetic("double_float")
    assert autotune(m2, 0, cache) == c2
    op = SIPG(oracle_spec(c), k)
    A = op.assemble()
    x = uniform(m2.n_dofs, "x")
    norm_a = abs(A).sum(axis=1).max()
    assert scaled_err(apply_laplace_f64(m2, _cuda(x)).cpu().numpy(), A @ x, norm_a, x) <= TOL64
    x32 = x.astype(np.float32)
    y32 = apply_laplace_f32(m2, _cuda(x32, torch.float32)).cpu().numpy()
    assert scaled_err(y32, A @ x32.astype(np.float64), norm_a, x) <= TOL32


def test_geometry_matches_oracle():
    for c, k in [(channel((3, 6, 2), gamma=2.25), 4), (case((2, 2, 3), lo=(-1, 0, 2), hi=(1, 3, 5)), 2)]:
        op = SIPG(oracle_spec(c), k)
        m = gpu_mesh(c, k)
        xyz = m.node_coordinates()
        assert np.max(np.abs(xyz - op.node_coordinates().reshape(-1, 3))) <= 1e-14 * np.max(np.abs(xyz))
        assert np.allclose(m.penalty_values(), op.tau, rtol=1e-13, atol=0)


def test_deterministic_and_stream_ordered():
    """Two applies give bitwise equal results (no atomics) on a side stream."""
    from paper_1607_01323_gb300 import apply_laplace_f64
    c = channel((4, 4, 4))
    m = gpu_mesh(c, 4)
    x = _cuda(uniform(m.n_dofs, "x"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y1 = apply_laplace_f64(m, x)
        y2 = apply_laplace_f64(m, x)
    s.synchronize()
    assert torch.equal(y1, y2)
