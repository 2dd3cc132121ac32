"""The allocation-free CG entry point (sipg_cg_solve_noalloc) against sipg_cg_solve.

Some callers cannot call cudaMalloc (device memory owned by their own pool or
caching allocator, a fixed memory budget, or loops that cannot take the
implicit synchronisation of cudaMalloc/cudaFree).  For them the library offers
a variant of the CG solve whose workspace is a static device array.  This test
calls both entry points through the C ABI with ctypes and checks that the
allocation-free solve returns the same solution, on two calls in a row (the
second call finds the previous call's data in the shared array), plus the
size limit.  It lives in its own file so that it is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(entry, mesh, b, x, precond):
    from paper_1607_01323_gb300 import _lib as L
    lib = L.lib()
    o = L.CgOpts()
    assert lib.sipg_cg_default_opts(C.byref(o)) == L.OK
    o.precond = L.PC[precond]
    o.rtol = 1e-10
    it, rel = C.c_int(), C.c_double()
    st = getattr(lib, entry)(mesh.handle, C.byref(o), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), 1,
                             C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(it), C.byref(rel))
    return st, it.value, rel.value


def test_noalloc_solve_matches_cg_solve():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_01323_gb300 import Mesh, inputs
    from paper_1607_01323_gb300 import _lib as L
    lo, hi = (0.0, -1.0, 0.0), (2 * np.pi, 1.0, np.pi)
    bcl, bch = ("periodic", "dirichlet", "periodic"), ("periodic", "dirichlet", "periodic")
    mesh = Mesh((6, 6, 6), lo, hi, bcl, bch, mapping="channel", gamma=1.8, k=3)
    for precond in ("jacobi", "invmass"):
        b = torch.tensor(inputs.uniform(0, "b", mesh.n_dofs), device="cuda")
        x_ref = torch.zeros_like(b)
        st, it_ref, rel_ref = _solve("sipg_cg_solve", mesh, b, x_ref, precond)
        assert st == L.OK and rel_ref <= 1e-10
        for call in range(2):
            # poison the output between calls; the solve starts from x = 0
            x = torch.zeros_like(b)
            st, it, rel = _solve("sipg_cg_solve_noalloc", mesh, b, x, precond)
            torch.cuda.synchronize()
            assert st == L.OK, L.lib().sipg_last_error()
            assert rel <= 1e-10 and it == it_ref
            assert (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item() <= 1e-12
    # a problem beyond the static array is rejected with a clear message
    cap = C.c_longlong()
    assert L.lib().sipg_cg_noalloc_capacity(C.byref(cap)) == L.OK and cap.value == 16 << 20
    big = Mesh((16, 16, 16), lo, hi, bcl, bch, mapping="channel", gamma=1.8, k=4)  # 512,000 unknowns
    b = torch.ones(big.n_dofs, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, _, _ = _solve("sipg_cg_solve_noalloc", big, b, x, "jacobi")
    assert st == L.EINVAL
    assert b"static array" in L.lib().sipg_last_error()
