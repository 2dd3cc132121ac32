"""The allocation-free CG entry point (sipg_cg_solve_noalloc) against sipg_cg_solve.

Some callers cannot call cudaMalloc (device memory owned by their own pool or
caching allocator, a fixed memory budget, or loops that cannot take the
implicit synchronisation of cudaMalloc/cudaFree).  For them the library offers
a variant of the CG solve whose workspace is a static device array.  These
tests call both entry points through the C ABI with ctypes and check that the
allocation-free solve returns the same solution, on two calls in a row (the
second call runs on the scratch the first one left), that a call takes no
device memory while sipg_cg_solve on the same mesh does, plus the size limit.
The file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LO, HI = (0.0, -1.0, 0.0), (2 * np.pi, 1.0, np.pi)
BCL, BCH = ("periodic", "dirichlet", "periodic"), ("periodic", "dirichlet", "periodic")


def _solve(entry, mesh, b, x, precond, ncomp=1, op="laplace", mass_coef=0.0, nu=1.0):
    from paper_1607_01323_gb300 import _lib as L
    lib = L.lib()
    o = L.CgOpts()
    assert lib.sipg_cg_default_opts(C.byref(o)) == L.OK
    o.precond = L.PC[precond]
    o.op = L.OP[op]
    o.mass_coef = mass_coef
    o.nu = nu
    o.rtol = 1e-10
    it, rel = C.c_int(), C.c_double()
    st = getattr(lib, entry)(mesh.handle, C.byref(o), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), ncomp,
                             C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(it), C.byref(rel))
    return st, it.value, rel.value


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [("laplace_jacobi", "jacobi", 1, "laplace", 0.0, 1.0),
         ("laplace_invmass", "invmass", 1, "laplace", 0.0, 1.0),
         ("helmholtz_two_components_invmass", "invmass", 2, "helmholtz", 1500.0, 1 / 180),
         ("helmholtz_two_components_none", "none", 2, "helmholtz", 1500.0, 1 / 180)]


@pytest.mark.parametrize("arith", ["native", "double_float"])
@pytest.mark.parametrize("name,precond,ncomp,op,cm,nu", CASES, ids=[c[0] for c in CASES])
def test_noalloc_solve_matches_cg_solve(name, precond, ncomp, op, cm, nu, arith):
    from paper_1607_01323_gb300 import Mesh, inputs
    from paper_1607_01323_gb300 import _lib as L
    mesh = Mesh((6, 6, 6), LO, HI, BCL, BCH, mapping="channel", gamma=1.8, k=3)
    mesh.set_f64_arithmetic(arith)
    b = torch.tensor(inputs.uniform(0, "b", ncomp * mesh.n_dofs), device="cuda")
    x_ref = torch.zeros_like(b)
    st, it_ref, rel_ref = _solve("sipg_cg_solve", mesh, b, x_ref, precond, ncomp, op, cm, nu)
    assert st == L.OK and rel_ref <= 1e-10
    for call in range(2):
        # x restarts from zero on every call; the second call runs on the
        # scratch array as the first call left it
        x = torch.zeros_like(b)
        st, it, rel = _solve("sipg_cg_solve_noalloc", mesh, b, x, precond, ncomp, op, cm, nu)
        torch.cuda.synchronize()
        assert st == L.OK, L.lib().sipg_last_error()
        assert rel <= 1e-10 and it == it_ref
        assert (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item() <= 1e-12


def test_noalloc_takes_no_device_memory():
    """After one warm-up call (which may load the library's modules), a call on
    a fresh mesh near the array's capacity leaves the device's free memory
    unchanged; sipg_cg_solve on the same mesh allocates its workspace."""
    from paper_1607_01323_gb300 import Mesh, inputs
    from paper_1607_01323_gb300 import _lib as L
    warm = Mesh((2, 2, 2), LO, HI, BCL, BCH, mapping="channel", gamma=1.8, k=4)
    bw = torch.ones(warm.n_dofs, dtype=torch.float64, device="cuda")
    assert _solve("sipg_cg_solve_noalloc", warm, bw, torch.zeros_like(bw), "jacobi")[0] == L.OK
    mesh = Mesh((12, 12, 12), LO, HI, BCL, BCH, mapping="channel", gamma=1.8, k=4)  # 216,000 unknowns
    b = torch.tensor(inputs.uniform(0, "b", mesh.n_dofs), device="cuda")
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st, _, rel = _solve("sipg_cg_solve_noalloc", mesh, b, x, "jacobi")
    torch.cuda.synchronize()
    assert st == L.OK and rel <= 1e-10
    assert torch.cuda.mem_get_info()[0] == free0
    x2 = torch.zeros_like(b)
    st, _, _ = _solve("sipg_cg_solve", mesh, b, x2, "jacobi")
    torch.cuda.synchronize()
    assert st == L.OK
    workspace = 6 * 8 * mesh.n_dofs  # r, z, p, Ap, scratch, diagonal
    assert free0 - torch.cuda.mem_get_info()[0] >= workspace


def test_noalloc_size_limit():
    """A problem beyond the static array is rejected with a clear message."""
    from paper_1607_01323_gb300 import Mesh
    from paper_1607_01323_gb300 import _lib as L
    cap = C.c_longlong()
    assert L.lib().sipg_cg_noalloc_capacity(C.byref(cap)) == L.OK and cap.value == 16 << 20
    big = Mesh((16, 16, 16), LO, HI, BCL, BCH, mapping="channel", gamma=1.8, k=4)  # 512,000 unknowns
    b = torch.ones(big.n_dofs, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _, _ = _solve("sipg_cg_solve_noalloc", big, b, x, "jacobi")
    assert st == L.EINVAL
    assert b"static array" in L.lib().sipg_last_error()
