"""The C ABI library builds, loads, and exports every function that
include/sipg.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    import shutil
    from paper_1607_01323_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists(build.OUT):
        pytest.skip("no nvcc and no built library")
    return build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sipg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sipg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_expected_api():
    names = declared_functions()
    for required in ["sipg_create_mesh", "sipg_set_degree", "sipg_set_penalty", "sipg_apply_laplace_f64",
                     "sipg_apply_laplace_f32", "sipg_apply_helmholtz_f64", "sipg_apply_inverse_mass_f64",
                     "sipg_diagonal_f64", "sipg_cg_solve", "sipg_adjoint_grad_nu", "sipg_autotune",
                     "sipg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_1607_01323_gb300 import _lib
    assert set(_lib.exported_symbols()) == set(declared_functions())


def test_host_only_entry_points(lib_path):
    from paper_1607_01323_gb300 import _lib
    L = _lib.lib()
    o = _lib.CgOpts()
    assert L.sipg_cg_default_opts(ctypes.byref(o)) == 0
    assert o.rtol == 1e-10 and o.maxit == 10000 and o.cheb_degree == 4 and o.cheb_range == 20.0
    assert o.precond == _lib.PC["jacobi"] and o.use_graph == 1
    # invalid arguments are rejected on the host before any CUDA call
    assert L.sipg_cg_default_opts(None) == _lib.EINVAL
    assert b"NULL" in L.sipg_last_error()
    d = _lib.MeshDesc()
    h = ctypes.c_void_p()
    assert L.sipg_create_mesh(ctypes.byref(d), ctypes.byref(h)) == _lib.EINVAL  # n = 0
    d.n[0] = d.n[1] = d.n[2] = 2
    for i in range(3):
        d.hi[i] = 1.0
    d.bc_lo[0], d.bc_hi[0] = _lib.BC["periodic"], _lib.BC["dirichlet"]
    assert L.sipg_create_mesh(ctypes.byref(d), ctypes.byref(h)) == _lib.EINVAL
    assert b"periodic" in L.sipg_last_error()
    for i in range(3):
        d.bc_lo[i] = d.bc_hi[i] = _lib.BC["periodic"]
    d.map, d.amplitude = _lib.MAP["perturbed"], -0.1
    assert L.sipg_create_mesh(ctypes.byref(d), ctypes.byref(h)) == _lib.EINVAL
    assert b"amplitude" in L.sipg_last_error()
    assert L.sipg_set_degree(None, 3) == _lib.EINVAL
    assert L.sipg_apply_laplace_f64(None, None, None, 1, None) == _lib.EINVAL


def test_product_path_does_not_import_the_oracle():
    """The CUDA path (package sources) never imports, links or calls oracle/."""
    pkg = os.path.join(ROOT, "paper_1607_01323_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_stepper_parameters_rejected_on_host(lib_path):
    """sipg_ns_create validates its parameters before any CUDA call."""
    from paper_1607_01323_gb300 import _lib
    L = _lib.lib()
    prm = _lib.NsParams()
    assert L.sipg_ns_default_params(ctypes.byref(prm)) == 0
    assert prm.k == 3 and prm.order == 3 and prm.zeta == 1.0 and prm.pressure_precond == _lib.PC["jacobi"]
    d = _lib.MeshDesc()
    for i in range(3):
        d.n[i], d.hi[i] = 2, 1.0
        d.bc_lo[i] = d.bc_hi[i] = _lib.BC["periodic"]
    d.bc_lo[1] = d.bc_hi[1] = _lib.BC["dirichlet"]
    h = ctypes.c_void_p()

    def rejected(**changes):
        p = _lib.NsParams()
        L.sipg_ns_default_params(ctypes.byref(p))
        for k, v in changes.items():
            setattr(p, k, v)
        return L.sipg_ns_create(ctypes.byref(d), ctypes.byref(p), ctypes.byref(h)) == _lib.EINVAL

    assert rejected(k=1)           # the pressure wall data need k >= 2
    assert rejected(order=4)
    assert rejected(nu=0.0)
    assert rejected(dt=-1.0)
    assert rejected(zeta=-1.0)
    assert rejected(pressure_precond=_lib.PC["invmass"])
    assert rejected(rtol_viscous=0.0)
    assert rejected(maxit_projection=0)
    d.bc_lo[1] = d.bc_hi[1] = _lib.BC["neumann"]  # outflow boundaries are not supported
    assert rejected()
    assert b"periodic sides and no-slip walls" in L.sipg_last_error()
    d.bc_lo[1] = d.bc_hi[1] = _lib.BC["dirichlet"]
    d.map, d.amplitude = _lib.MAP["perturbed"], 0.05
    assert rejected()
    assert b"separable" in L.sipg_last_error()
    assert L.sipg_ns_step(None, None, None, None) == _lib.EINVAL
    assert L.sipg_ns_set_velocity(None, 0, None, None) == _lib.EINVAL
