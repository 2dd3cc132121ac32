"""GPU parity of the convective term (Eq. (convstepspat), local Lax-Friedrichs
flux, floor(3k/2)+1 Gauss points) against the oracle: element by element on
small meshes in native FP64 and double-float arithmetic, on sampled cells of
the 32^3 k = 3 channel, and by properties that hold at any size (a constant
field on a periodic mesh gives zero; C(2u) = 4 C(u) exactly)."""
import numpy as np
import pytest

from helpers import case, channel, gpu_mesh, oracle_spec, uniform
from oracle.convective import ConvectiveOp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative to max|y_ref|: a few hundred roundings of O(max|y|) terms per output
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


CASES = [
    ("channel_k2", channel((2, 6, 2)), 2),
    ("channel_k3", channel((3, 4, 2)), 3),
    ("channel_linear_k4", case((2, 4, 2), lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.0),
                               bc_lo=("periodic", "dirichlet", "periodic"),
                               bc_hi=("periodic", "dirichlet", "periodic"), mapping="channel_linear"), 4),
    ("affine_neumann_walls_k3", case((2, 3, 2), lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5),
                                     bc_lo=("periodic", "neumann", "periodic"),
                                     bc_hi=("periodic", "neumann", "periodic")), 3),
    ("box_mixed_k4", case((3, 2, 2), hi=(1.0, 0.7, 1.3), bc_lo=("dirichlet", "neumann", "periodic"),
                          bc_hi=("dirichlet", "dirichlet", "periodic")), 4),
    ("single_periodic_cell_k3", case((1, 1, 1)), 3),
    ("channel_k1", channel((3, 4, 2)), 1),
    ("channel_k5", channel((2, 2, 1)), 5),
    ("channel_k7", channel((1, 2, 1)), 7),
]


@pytest.mark.parametrize("arith", ["native", "double_float"])
@pytest.mark.parametrize("name,c,k", CASES, ids=[x[0] for x in CASES])
def test_convective_parity(name, c, k, arith):
    from paper_1607_01323_gb300 import apply_convective_f64
    op = ConvectiveOp(oracle_spec(c), k)
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic(arith)
    u = uniform(3 * m.n_dofs, "u", seed=21)
    y_ref = op.apply(u)
    y = apply_convective_f64(m, _cuda(u)).cpu().numpy()
    err = np.abs(y - y_ref).max() / np.abs(y_ref).max()
    assert err <= TOL, err


def _channel_velocity(m, seed):
    from paper_1607_01323_gb300 import inputs
    X = m.node_coordinates()
    N = m.n_dofs
    return np.concatenate([(1 - X[:, 1] ** 2) + 0.1 * inputs.normal(seed, "ux", N),
                           0.1 * inputs.normal(seed, "uy", N), 0.1 * inputs.normal(seed, "uz", N)])


@pytest.mark.parametrize("arith", ["native", "double_float"])
def test_convective_sampled_cells_at_size(arith):
    """32^3 k = 3 channel (2.1M DoF per component), laminar profile plus
    noise: 48 cells (walls, interior and periodic seams) against the oracle."""
    from paper_1607_01323_gb300 import apply_convective_f64
    c = channel((32, 32, 32))
    k = 3
    m = gpu_mesh(c, k)
    m.set_f64_arithmetic(arith)
    u = _channel_velocity(m, 3)
    y = apply_convective_f64(m, _cuda(u)).cpu().numpy()
    op = ConvectiveOp(oracle_spec(c), k)
    n0, n1, n2 = c["n"]
    rng = np.random.default_rng(5)
    ids = [(0, 0, 0), (n0 - 1, n1 - 1, n2 - 1), (n0 - 1, 0, 0), (0, n1 - 1, n2 - 1)]
    ids += [tuple(int(v) for v in rng.integers(0, (n0, n1, n2))) for _ in range(44)]
    cells = sorted({i + n0 * (j + n1 * kk) for i, j, kk in ids})
    y_ref = op.apply(u, cells=cells).reshape(3, -1, op.P)
    yc = y.reshape(3, -1, op.P)
    scale = np.abs(y_ref[:, cells]).max()
    assert np.abs(yc[:, cells] - y_ref[:, cells]).max() <= TOL * scale


@pytest.mark.parametrize("arith", ["native", "double_float"])
def test_convective_properties_at_size(arith):
    """A constant field on a periodic tanh-mapped mesh gives zero (no
    divergence, no jumps); the term is homogeneous of degree 2, and scaling
    by 2 is exact in both arithmetics, so C(2u) = 4 C(u) bit for bit."""
    from paper_1607_01323_gb300 import apply_convective_f64
    c = case((32, 32, 32), lo=(0.0, -1.0, 0.0), hi=(6.283185307179586, 1.0, 3.141592653589793),
             mapping="channel")
    m = gpu_mesh(c, 3)
    m.set_f64_arithmetic(arith)
    N = m.n_dofs
    const = torch.cat([torch.full((N,), 0.7), torch.full((N,), -1.3), torch.full((N,), 0.4)]).double().cuda()
    y0 = apply_convective_f64(m, const)
    assert y0.abs().max().item() <= 1e-13
    mc = gpu_mesh(channel((32, 32, 32)), 3)
    mc.set_f64_arithmetic(arith)
    u = _cuda(_channel_velocity(mc, 4))
    y1 = apply_convective_f64(mc, u)
    y2 = apply_convective_f64(mc, 2 * u)
    assert torch.equal(y2, 4 * y1)


def test_convective_errors():
    from paper_1607_01323_gb300 import SipgError, apply_convective_f64
    m = gpu_mesh(channel((2, 4, 2)), 2)
    u = _cuda(uniform(3 * m.n_dofs, "u"))
    with pytest.raises(SipgError):
        apply_convective_f64(m, u, y=u)
    with pytest.raises(ValueError):
        apply_convective_f64(m, u[: m.n_dofs])
    assert torch.isfinite(apply_convective_f64(m, u)).all()


def test_convective_cells_per_block():
    """Every feasible cells-per-block gives the same bits (the cells of a block
    do not interact), including a ragged last block."""
    from paper_1607_01323_gb300 import SipgError, apply_convective_f64
    c = channel((3, 5, 3))
    m = gpu_mesh(c, 3)
    u = _cuda(uniform(3 * m.n_dofs, "u", seed=7))
    ref = apply_convective_f64(m, u)
    cpb = 1
    while True:
        try:
            m.set_cells_per_block(2, cpb)
        except SipgError:
            break
        assert m.cells_per_block(2) == cpb
        assert torch.equal(apply_convective_f64(m, u), ref), cpb
        cpb += 1
    assert cpb > 2
