"""GPU parity of the dual-splitting step (Sec. 2.2, variant V3c) against the
oracle: the pressure wall data of Eq. (ipflux), then several whole steps
(velocity and pressure) on a tanh channel with no-slip walls, a body force,
the div-div penalty and the BDF order ramp, in native FP64 and double-float
operator arithmetic, and on a periodic Taylor-Green vortex; Poiseuille flow
stays a steady state on a 32^3 channel; invalid set-ups are rejected."""
import math

import numpy as np
import pytest

from helpers import case, channel, oracle_spec
from oracle.stepper import DualSplitting

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _ns(c, k, **kw):
    from paper_1607_01323_gb300 import NavierStokes
    return NavierStokes(c["n"], c["lo"], c["hi"], c["bc_lo"], c["bc_hi"], mapping=c["mapping"], gamma=c["gamma"],
                        k=k, **kw)


def _velocity(X, seed, amp=0.2):
    """Laminar profile in x plus smooth seeded perturbations (not solenoidal)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (3, 4))
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    w = 1 - y ** 2
    pert = [amp * w * (a[i, 0] * np.sin(x + a[i, 1]) + a[i, 2] * np.cos(2 * z + a[i, 3]) + 0.3 * y) for i in range(3)]
    return np.concatenate([w + pert[0], pert[1], pert[2]])


def test_wall_data_parity():
    c = channel((2, 3, 2))
    k = 3
    ns = _ns(c, k, nu=0.05, dt=0.05)
    X = ns.velocity_mesh.node_coordinates()
    u = _velocity(X, 1)
    ns.set_velocity(_cuda(u))
    h = ns.wall_data().cpu().numpy()
    ds = DualSplitting(oracle_spec(c), k, 0.05, 0.05)
    ref = np.concatenate(ds.wall_values(u))
    assert h.shape == ref.shape
    assert np.abs(h - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("arith", ["native", "double_float"])
def test_steps_parity_channel(arith):
    """Five steps (orders 1, 2, 3, 3, 3) on the 2 x 4 x 2 tanh channel, k = 3."""
    c = channel((2, 4, 2))
    k, nu, dt, zeta = 3, 0.05, 0.05, 1.0
    f = (0.3, 0.0, 0.1)
    tol = dict(rtol_pressure=1e-13, rtol_viscous=1e-13, rtol_projection=1e-13)
    ns = _ns(c, k, nu=nu, dt=dt, order=3, zeta=zeta, f64_arithmetic=arith, **tol)
    ds = DualSplitting(oracle_spec(c), k, nu, dt, order=3, zeta=zeta, rtol=1e-14)
    X = ns.velocity_mesh.node_coordinates()
    u0 = _velocity(X, 2)
    ns.set_velocity(_cuda(u0))
    ds.set_history([u0])
    for s in range(5):
        st = ns.step(f)
        u_ref, p_ref, info = ds.step(f)
        assert st["order"] == info["order"] == min(s + 1, 3)
        u = ns.velocity().cpu().numpy()
        p = ns.pressure().cpu().numpy()
        p, p_ref = p - p.mean(), p_ref - p_ref.mean()
        assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max(), (s, np.abs(u - u_ref).max())
        assert np.abs(p - p_ref).max() <= 1e-8 * np.abs(p_ref).max(), (s, np.abs(p - p_ref).max())


def test_steps_parity_taylor_green():
    """Periodic Taylor-Green vortex, 3 x 3 x 1 cells, k = 4, GMG pressure
    preconditioner, older levels given (BDF3 from the first step)."""
    c = case((3, 3, 1), hi=(2 * math.pi, 2 * math.pi, 1.0))
    k, nu, dt = 4, 0.1, 0.1
    ns = _ns(c, k, nu=nu, dt=dt, order=3, zeta=0.0, pressure_precond="gmg_f32", rtol_pressure=1e-13,
             rtol_viscous=1e-13, rtol_projection=1e-13)
    ds = DualSplitting(oracle_spec(c), k, nu, dt, order=3, zeta=0.0, rtol=1e-14)
    X = ns.velocity_mesh.node_coordinates()

    def tgv(t):
        F = math.exp(-2 * nu * t)
        x, y = X[:, 0], X[:, 1]
        return np.concatenate([np.sin(x) * np.cos(y) * F, -np.cos(x) * np.sin(y) * F, 0 * x])

    levels = [tgv(-i * dt) for i in range(3)]
    for i, v in enumerate(levels):
        ns.set_velocity(_cuda(v), level=i)
    ds.set_history(levels)
    for s in range(3):
        st = ns.step()
        u_ref, p_ref, _ = ds.step()
        assert st["order"] == 3
        u = ns.velocity().cpu().numpy()
        p = ns.pressure().cpu().numpy()
        p, p_ref = p - p.mean(), p_ref - p_ref.mean()
        assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
        assert np.abs(p - p_ref).max() <= 1e-8 * np.abs(p_ref).max()


def test_poiseuille_steady_at_size():
    """u = (1 - y^2, 0, 0), f = (2 nu, 0, 0) between walls at y = -1, 1 on an
    affine 32 x 16 x 16 channel at k = 3 (3 x 2.1M velocity DoF): a discrete
    steady state, so u^(n+1) = u^n to the solver tolerance."""
    c = case((32, 16, 16), lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, math.pi),
             bc_lo=("periodic", "dirichlet", "periodic"), bc_hi=("periodic", "dirichlet", "periodic"))
    nu = 1 / 180
    ns = _ns(c, 3, nu=nu, dt=2e-3, order=3, zeta=1.0, pressure_precond="gmg_f32", rtol_pressure=1e-12,
             rtol_viscous=1e-12, rtol_projection=1e-12)
    X = ns.velocity_mesh.node_coordinates()
    u0 = np.concatenate([1 - X[:, 1] ** 2, 0 * X[:, 0], 0 * X[:, 0]])
    ns.set_velocity(_cuda(u0))
    for s in range(4):
        ns.step((2 * nu, 0.0, 0.0))
    u = ns.velocity().cpu().numpy()
    assert np.abs(u - u0).max() <= 1e-9
    p = ns.pressure()
    assert (p - p.mean()).abs().max().item() <= 1e-7


def test_stepper_errors():
    from paper_1607_01323_gb300 import SipgError
    c = channel((2, 4, 2))
    with pytest.raises(SipgError):
        _ns(c, 1)
    with pytest.raises(SipgError):
        _ns(channel((2, 4, 2), wall="neumann"), 3)
    with pytest.raises(SipgError):
        _ns(c, 3, order=4)
    with pytest.raises(SipgError):
        _ns(c, 3, pressure_precond="invmass")
    ns = _ns(c, 3)
    with pytest.raises(SipgError):
        ns.step()  # no velocity yet
    u = torch.zeros(3 * ns.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(SipgError):
        ns.set_velocity(u, level=1)  # level 0 first
    ns.set_velocity(u)
    st = ns.step()
    assert st["order"] == 1 and ns.velocity().abs().max().item() == 0.0


def test_long_run_stability_and_divergence():
    """Stability and divergence over 200 steps (the metrics the paper checks
    for the splitting, Sec. 4): a noisy start on the 8^3 k = 3 tanh channel at
    low Reynolds number (nu = 0.2, f = 2 nu) relaxes towards Poiseuille flow,
    the perturbation energy decays, and the weak divergence D u stays small
    relative to the velocity's own scale."""
    from paper_1607_01323_gb300 import apply_divergence_f64, apply_mass_f64
    c = channel((8, 8, 8))
    nu, dt = 0.2, 0.01
    ns = _ns(c, 3, nu=nu, dt=dt, order=3, zeta=1.0, pressure_precond="gmg_f32", rtol_pressure=1e-8,
             rtol_viscous=1e-8, rtol_projection=1e-10)
    X = ns.velocity_mesh.node_coordinates()
    N = ns.n_dofs
    up = np.concatenate([1 - X[:, 1] ** 2, 0 * X[:, 0], 0 * X[:, 0]])
    u0 = _velocity(X, 7, amp=0.3)
    ns.set_velocity(_cuda(u0))
    m = ns.velocity_mesh

    def energy(v):
        d = _cuda(v - up)
        return torch.dot(d, apply_mass_f64(m, d)).item()

    e0 = energy(u0)
    div0 = apply_divergence_f64(m, _cuda(u0)).abs().max().item()
    for s in range(200):  # a solve that stops at its iteration bound raises
        st = ns.step((2 * nu, 0.0, 0.0))
    assert st["order"] == 3
    u = ns.velocity().cpu().numpy()
    assert np.isfinite(u).all()
    assert energy(u) <= 0.2 * e0  # the perturbation decays
    div = apply_divergence_f64(m, _cuda(u)).abs().max().item()
    assert div <= 0.05 * div0  # the projection keeps the velocity nearly solenoidal
