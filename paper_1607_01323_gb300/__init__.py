"""GB300-native matrix-free SIPG operators (arXiv:1607.01323): Python binding.

A thin layer over the C ABI of ``include/sipg.h`` (libsipg.so).  It only
marshals arguments: tensors become raw device pointers, the current torch
stream becomes the CUDA stream.  Every computation runs in the library's
kernels; there is no CPU fallback, and a missing library raises.

The functions keep the C names without the ``sipg_`` prefix
(``apply_laplace_f64``, ``cg_solve``, ...); ``Mesh`` wraps ``sipg_mesh``.
The library is loaded lazily, so ``paper_1607_01323_gb300.inputs`` imports
without it.
"""
import ctypes as C

from . import _lib as L

__all__ = ["Mesh", "create_mesh", "apply_laplace_f64", "apply_laplace_f32", "apply_helmholtz_f64",
           "apply_helmholtz_f32", "apply_mass_f64", "apply_inverse_mass_f64", "diagonal_f64", "cg_solve",
           "mg_setup", "mg_info", "mg_vcycle", "apply_divergence_f64", "apply_gradient_f64", "tau_div_f64",
           "apply_divdiv_f64", "project_divdiv_f64", "apply_viscous_f64", "apply_convective_f64", "NavierStokes", "adjoint_grad_nu", "autotune", "CgResult",
           "SipgError"]

SipgError = L.SipgError


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return C.c_void_p(t.data_ptr())


class Mesh:
    """A structured hexahedral mesh with its geometry tables on the current GPU.

    n: cells per direction; lo, hi: box; bc_lo / bc_hi: 'periodic',
    'dirichlet' or 'neumann' per direction; mapping: 'affine', 'channel'
    (tanh grading of y with parameter gamma) or 'channel_linear' (the graded
    cell vertices with straight cells); k: polynomial degree;
    penalty: factor on tau of Eq. (taue)."""

    def __init__(self, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3,
                 bc_hi=("periodic",) * 3, mapping="affine", gamma=1.8, k=3, penalty=1.0, amplitude=0.0, seed=0):
        lib = L.lib()
        d = L.MeshDesc()
        d.amplitude, d.seed = float(amplitude), int(seed)
        for i in range(3):
            d.n[i] = int(n[i])
            d.lo[i] = float(lo[i])
            d.hi[i] = float(hi[i])
            d.bc_lo[i] = L.BC[bc_lo[i]]
            d.bc_hi[i] = L.BC[bc_hi[i]]
        d.map = L.MAP[mapping]
        d.gamma = float(gamma)
        h = C.c_void_p()
        L.check(lib.sipg_create_mesh(C.byref(d), C.byref(h)))
        self._h = h
        self.n = tuple(int(v) for v in n)
        self.bc_lo, self.bc_hi = tuple(bc_lo), tuple(bc_hi)
        self.mapping, self.gamma = mapping, gamma
        self.set_degree(k)
        self.set_penalty(penalty)

    @classmethod
    def _view(cls, handle, owner, n, bc_lo, bc_hi, mapping, gamma, k, penalty):
        """A mesh owned by another library object (kept alive through `owner`)."""
        m = cls.__new__(cls)
        m._h, m._owner = handle, owner
        m.n, m.bc_lo, m.bc_hi = tuple(n), tuple(bc_lo), tuple(bc_hi)
        m.mapping, m.gamma, m.k, m.p, m.penalty = mapping, gamma, int(k), int(k) + 1, float(penalty)
        return m

    def __del__(self):
        h = getattr(self, "_h", None)
        if getattr(self, "_owner", None) is not None:
            return
        if h is not None and h.value and L._lib is not None:
            L._lib.sipg_destroy_mesh(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_degree(self, k):
        L.check(L.lib().sipg_set_degree(self._h, int(k)))
        self.k = int(k)
        self.p = self.k + 1

    def set_penalty(self, factor):
        L.check(L.lib().sipg_set_penalty(self._h, float(factor)))
        self.penalty = float(factor)

    @property
    def n_dofs(self):
        v = C.c_longlong()
        L.check(L.lib().sipg_n_dofs(self._h, C.byref(v)))
        return v.value

    @property
    def ncell(self):
        v = C.c_longlong()
        L.check(L.lib().sipg_n_cells(self._h, C.byref(v)))
        return v.value

    def node_coordinates(self):
        """(n_dofs, 3) float64 numpy array of nodal point coordinates."""
        import numpy as np
        out = np.empty((self.n_dofs, 3), dtype=np.float64)
        L.check(L.lib().sipg_node_coordinates(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def penalty_values(self):
        import numpy as np
        out = np.empty(self.ncell, dtype=np.float64)
        L.check(L.lib().sipg_penalty_values(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_f64_arithmetic(self, mode):
        """'native' (FP64) or 'double_float' (FP32 pairs) arithmetic for the FP64
        operator, mass and inverse-mass applies (FP64 data either way)."""
        L.check(L.lib().sipg_set_f64_arithmetic(self._h, {"native": 0, "double_float": 1}[mode]))
        self.f64_arithmetic = mode

    def set_f32_mapping(self, mapping):
        """'line' (p^2 threads per cell) or 'plane' (p threads per cell) for the
        FP32 operator with a uniform viscosity."""
        L.check(L.lib().sipg_set_f32_mapping(self._h, {"line": 0, "plane": 1}[mapping]))

    def cells_per_block(self, precision=0):
        v = C.c_int()
        L.check(L.lib().sipg_get_cells_per_block(self._h, int(precision), C.byref(v)))
        return v.value

    def set_cells_per_block(self, precision, cpb):
        L.check(L.lib().sipg_set_cells_per_block(self._h, int(precision), int(cpb)))

    def profile_enable(self, on=True):
        L.check(L.lib().sipg_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        """(summed apply ms, timed applies, kernels launched) since the last reset."""
        ms, n, launches = C.c_double(), C.c_longlong(), C.c_longlong()
        L.check(L.lib().sipg_profile_read(self._h, 1 if reset else 0, C.byref(ms), C.byref(n), C.byref(launches)))
        return ms.value, n.value, launches.value


def create_mesh(*args, **kw):
    return Mesh(*args, **kw)


def _ncomp(mesh, x):
    n = mesh.n_dofs
    if x.numel() % n != 0 or x.numel() == 0:
        raise ValueError("vector length %d is not a multiple of n_dofs %d" % (x.numel(), n))
    return x.numel() // n


def _out(x, y):
    torch = _torch()
    return torch.empty_like(x) if y is None else y


def apply_laplace_f64(mesh, x, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    L.check(L.lib().sipg_apply_laplace_f64(mesh.handle, _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"),
                                           _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def apply_laplace_f32(mesh, x, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    L.check(L.lib().sipg_apply_laplace_f32(mesh.handle, _dev(x, torch.float32, "x"), _dev(y, torch.float32, "y"),
                                           _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def apply_helmholtz_f64(mesh, x, mass_coef, nu, nu_cell=None, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    nuc = _dev(nu_cell, torch.float64, "nu_cell") if nu_cell is not None else None
    L.check(L.lib().sipg_apply_helmholtz_f64(mesh.handle, float(mass_coef), float(nu), nuc,
                                             _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"),
                                             _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def apply_helmholtz_f32(mesh, x, mass_coef, nu, nu_cell=None, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    nuc = _dev(nu_cell, torch.float32, "nu_cell") if nu_cell is not None else None
    L.check(L.lib().sipg_apply_helmholtz_f32(mesh.handle, float(mass_coef), float(nu), nuc,
                                             _dev(x, torch.float32, "x"), _dev(y, torch.float32, "y"),
                                             _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def apply_mass_f64(mesh, x, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    L.check(L.lib().sipg_apply_mass_f64(mesh.handle, _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"),
                                        _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def apply_inverse_mass_f64(mesh, x, y=None, stream=None):
    torch = _torch()
    y = _out(x, y)
    L.check(L.lib().sipg_apply_inverse_mass_f64(mesh.handle, _dev(x, torch.float64, "x"),
                                                _dev(y, torch.float64, "y"), _ncomp(mesh, x), _stream_ptr(stream)))
    return y


def diagonal_f64(mesh, op="laplace", mass_coef=0.0, nu=1.0, nu_cell=None, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty(mesh.n_dofs, dtype=torch.float64, device="cuda")
    nuc = _dev(nu_cell, torch.float64, "nu_cell") if nu_cell is not None else None
    L.check(L.lib().sipg_diagonal_f64(mesh.handle, L.OP[op], float(mass_coef), float(nu), nuc,
                                      _dev(out, torch.float64, "diag"), _stream_ptr(stream)))
    return out


class CgResult:
    def __init__(self, status, iters, relres):
        self.status, self.iters, self.relres = status, iters, relres
        self.converged = status == L.OK

    def __repr__(self):
        return "CgResult(status=%d, iters=%d, relres=%.3e)" % (self.status, self.iters, self.relres)


def cg_opts(**kw):
    o = L.CgOpts()
    L.check(L.lib().sipg_cg_default_opts(C.byref(o)))
    for key, v in kw.items():
        if key == "op":
            v = L.OP[v] if isinstance(v, str) else v
        elif key == "precond":
            v = L.PC[v] if isinstance(v, str) else v
        elif key == "nu_cell":
            v = v.data_ptr() if v is not None else None
        setattr(o, key, v)
    return o


def cg_solve(mesh, b, x=None, stream=None, raise_on_fail=True, **opts):
    """Solve A x = b (x holds the initial guess; zeros when None).  Keyword
    options are the fields of sipg_cg_opts (op, precond, rtol, maxit, ...)."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(b)
    if opts.get("nu_cell") is not None:
        _dev(opts["nu_cell"], torch.float64, "nu_cell")
    o = cg_opts(**opts)
    it, rel = C.c_int(), C.c_double()
    st = L.lib().sipg_cg_solve(mesh.handle, C.byref(o), _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"),
                               _ncomp(mesh, b), _stream_ptr(stream), C.byref(it), C.byref(rel))
    if raise_on_fail:
        L.check(st)
    return x, CgResult(st, it.value, rel.value)


def mg_setup(mesh, stream=None, **opts):
    """Build (or reuse) the multigrid hierarchy for the given sipg_cg_opts fields."""
    o = cg_opts(**opts)
    L.check(L.lib().sipg_mg_setup(mesh.handle, C.byref(o), _stream_ptr(stream)))
    return mg_info(mesh)


def mg_info(mesh, max_levels=32):
    """dict(nlevels, n_cells [list of (nx, ny, nz)], lmax [per level], coarse_lmin, coarse_degree)."""
    nl, cdeg, clmin = C.c_int(), C.c_int(), C.c_double()
    cells = (C.c_int * (3 * max_levels))()
    lmax = (C.c_double * max_levels)()
    L.check(L.lib().sipg_mg_info(mesh.handle, max_levels, C.byref(nl), cells, lmax, C.byref(clmin), C.byref(cdeg)))
    n = min(nl.value, max_levels)
    return dict(nlevels=nl.value, n_cells=[tuple(cells[3 * i:3 * i + 3]) for i in range(n)],
                lmax=[lmax[i] for i in range(n)], coarse_lmin=clmin.value, coarse_degree=cdeg.value)


def mg_vcycle(mesh, r, z=None, stream=None):
    """z = V(r), one FP32 V-cycle of the hierarchy set up by mg_setup."""
    torch = _torch()
    if z is None:
        z = torch.empty_like(r)
    L.check(L.lib().sipg_mg_vcycle(mesh.handle, _dev(r, torch.float64, "r"), _dev(z, torch.float64, "z"),
                                   _stream_ptr(stream)))
    return z


def _vel(mesh, u, name):
    torch = _torch()
    if u.numel() != 3 * mesh.n_dofs:
        raise ValueError("%s must hold 3 * n_dofs values (velocity components x, y, z)" % name)
    return _dev(u, torch.float64, name)


def apply_divergence_f64(mesh, u, y=None, stream=None):
    """y = D u, the divergence of Eq. (av3) (u: 3 components, y: 1)."""
    torch = _torch()
    if y is None:
        y = torch.empty(mesh.n_dofs, dtype=torch.float64, device=u.device)
    L.check(L.lib().sipg_apply_divergence_f64(mesh.handle, _vel(mesh, u, "u"), _dev(y, torch.float64, "y"),
                                              _stream_ptr(stream)))
    return y


def apply_gradient_f64(mesh, p, y=None, stream=None):
    """y = G p, the gradient of Eq. (bv3) (p: 1 component, y: 3)."""
    torch = _torch()
    if p.numel() != mesh.n_dofs:
        raise ValueError("p must hold n_dofs values")
    if y is None:
        y = torch.empty(3 * mesh.n_dofs, dtype=torch.float64, device=p.device)
    L.check(L.lib().sipg_apply_gradient_f64(mesh.handle, _dev(p, torch.float64, "p"), _vel(mesh, y, "y"),
                                            _stream_ptr(stream)))
    return y


def apply_viscous_f64(mesh, u, mass_coef, nu, y=None, stream=None):
    """y = mass_coef M u + A_nu u, the divergence-form viscous operator of the
    implicit viscous step (3 coupled velocity components)."""
    torch = _torch()
    if y is None:
        y = torch.empty_like(u)
    L.check(L.lib().sipg_apply_viscous_f64(mesh.handle, float(mass_coef), float(nu), _vel(mesh, u, "u"),
                                           _vel(mesh, y, "y"), _stream_ptr(stream)))
    return y


def apply_convective_f64(mesh, u, y=None, stream=None):
    """y = the convective term of Eq. (convstepspat) with the local
    Lax-Friedrichs flux and floor(3k/2)+1 Gauss points (3 velocity components)."""
    torch = _torch()
    if y is None:
        y = torch.empty_like(u)
    L.check(L.lib().sipg_apply_convective_f64(mesh.handle, _vel(mesh, u, "u"), _vel(mesh, y, "y"),
                                              _stream_ptr(stream)))
    return y


def tau_div_f64(mesh, u, zeta, dt, out=None, stream=None):
    """Per-cell div-div penalty tau_D of Eq. (tauD)."""
    torch = _torch()
    if out is None:
        out = torch.empty(mesh.ncell, dtype=torch.float64, device=u.device)
    L.check(L.lib().sipg_tau_div_f64(mesh.handle, _vel(mesh, u, "u"), float(zeta), float(dt),
                                     _dev(out, torch.float64, "tau"), _stream_ptr(stream)))
    return out


def apply_divdiv_f64(mesh, tau, u, y=None, stream=None):
    """y = (M + tau_e B) u cell by cell, the operator of Eq. (div-div)."""
    torch = _torch()
    if y is None:
        y = torch.empty_like(u)
    L.check(L.lib().sipg_apply_divdiv_f64(mesh.handle, _dev(tau, torch.float64, "tau"), _vel(mesh, u, "u"),
                                          _vel(mesh, y, "y"), _stream_ptr(stream)))
    return y


def project_divdiv_f64(mesh, tau, rhs, x=None, rtol=1e-12, maxit=200, stream=None):
    """Solve the local projections (M + tau_e B) x = rhs (per-cell CG with the
    inverse-mass preconditioner).  Returns (x, largest iteration count)."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(rhs)
    it = C.c_int()
    L.check(L.lib().sipg_project_divdiv_f64(mesh.handle, _dev(tau, torch.float64, "tau"), _vel(mesh, rhs, "rhs"),
                                            _vel(mesh, x, "x"), float(rtol), int(maxit), _stream_ptr(stream),
                                            C.byref(it)))
    return x, it.value


def adjoint_grad_nu(mesh, nu_cell, u, lam, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty(mesh.ncell, dtype=torch.float64, device="cuda")
    L.check(L.lib().sipg_adjoint_grad_nu(mesh.handle, _dev(nu_cell, torch.float64, "nu_cell"),
                                         _dev(u, torch.float64, "u"), _dev(lam, torch.float64, "lambda"),
                                         _dev(out, torch.float64, "grad"), _stream_ptr(stream)))
    return out


def autotune(mesh, precision=0, cache_path=None):
    L.check(L.lib().sipg_autotune(mesh.handle, int(precision), cache_path.encode() if cache_path else None))
    return mesh.cells_per_block(precision)


class NavierStokes:
    """The dual-splitting time step (Sec. 2.2, variant V3c) on the device:
    explicit convective step, pressure Poisson equation with the wall data of
    Eq. (ipflux), div-div penalised projection, implicit viscous step, BDF
    order 1-3.  Velocity boundaries: periodic or no-slip walls ("dirichlet")."""

    def __init__(self, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3,
                 bc_hi=("periodic",) * 3, mapping="affine", gamma=1.8, k=3, nu=1.0 / 180.0, dt=1e-3, order=3,
                 zeta=1.0, pressure_precond="jacobi", rtol_pressure=1e-10, rtol_viscous=1e-10,
                 rtol_projection=1e-10, maxit=10000, maxit_projection=500, penalty=1.0, f64_arithmetic=None):
        lib = L.lib()
        d = L.MeshDesc()
        for i in range(3):
            d.n[i], d.lo[i], d.hi[i] = int(n[i]), float(lo[i]), float(hi[i])
            d.bc_lo[i], d.bc_hi[i] = L.BC[bc_lo[i]], L.BC[bc_hi[i]]
        d.map, d.gamma = L.MAP[mapping], float(gamma)
        prm = L.NsParams()
        L.check(lib.sipg_ns_default_params(C.byref(prm)))
        prm.k, prm.penalty, prm.nu, prm.dt, prm.order, prm.zeta = int(k), float(penalty), float(nu), float(dt), \
            int(order), float(zeta)
        prm.pressure_precond = L.PC[pressure_precond]
        prm.rtol_pressure, prm.rtol_viscous, prm.rtol_projection = rtol_pressure, rtol_viscous, rtol_projection
        prm.maxit, prm.maxit_projection = int(maxit), int(maxit_projection)
        h = C.c_void_p()
        L.check(lib.sipg_ns_create(C.byref(d), C.byref(prm), C.byref(h)))
        self._h = h
        self.params = prm
        pbc = lambda bcs: tuple("neumann" if b == "dirichlet" else b for b in bcs)
        meshes = []
        for which, (bl, bh) in enumerate(((bc_lo, bc_hi), (pbc(bc_lo), pbc(bc_hi)))):
            mh = C.c_void_p()
            L.check(lib.sipg_ns_mesh(h, which, C.byref(mh)))
            meshes.append(Mesh._view(mh, self, n, bl, bh, mapping, gamma, k, penalty))
        self.velocity_mesh, self.pressure_mesh = meshes
        if f64_arithmetic is not None:
            for m in meshes:
                m.set_f64_arithmetic(f64_arithmetic)
        self.n_dofs = self.velocity_mesh.n_dofs

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and L._lib is not None:
            L._lib.sipg_ns_destroy(h)
            self._h = None

    def set_velocity(self, u, level=0, stream=None):
        """Time level n - level (0: current; then 1, 2 in order); u: 3 * n_dofs on the device."""
        L.check(L.lib().sipg_ns_set_velocity(self._h, int(level), _vel(self.velocity_mesh, u, "u"),
                                             _stream_ptr(stream)))

    def step(self, f=(0.0, 0.0, 0.0), stream=None):
        """One step with the constant body force f; returns the solver statistics."""
        fa = (C.c_double * 3)(*[float(v) for v in f])
        st = L.NsStats()
        L.check(L.lib().sipg_ns_step(self._h, fa, _stream_ptr(stream), C.byref(st)))
        return {k: getattr(st, k) for k, _ in L.NsStats._fields_}

    def velocity(self, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(3 * self.n_dofs, dtype=torch.float64, device="cuda")
        L.check(L.lib().sipg_ns_velocity(self._h, _vel(self.velocity_mesh, out, "out"), _stream_ptr(stream)))
        return out

    def pressure(self, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        L.check(L.lib().sipg_ns_pressure(self._h, _dev(out, torch.float64, "out"), _stream_ptr(stream)))
        return out

    def wall_data(self, stream=None):
        """(div F^c(u) + nu curl omega) . n of the current velocity at the Gauss
        points of the wall faces (faces by cell, direction, side)."""
        torch = _torch()
        cnt = C.c_longlong()
        L.check(L.lib().sipg_ns_wall_data(self._h, None, C.byref(cnt), None))
        out = torch.empty(max(cnt.value, 1), dtype=torch.float64, device="cuda")
        L.check(L.lib().sipg_ns_wall_data(self._h, _dev(out, torch.float64, "out"), C.byref(cnt),
                                          _stream_ptr(stream)))
        return out[: cnt.value]
