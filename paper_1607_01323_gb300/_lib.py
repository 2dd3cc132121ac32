"""ctypes declarations of libsipg.so (the C ABI of include/sipg.h)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsipg.so")

OK, MAXITER, EINVAL, ECUDA, ENOMEM, BREAKDOWN, NONFINITE = 0, 1, -1, -2, -3, -4, -5
BC = {"periodic": 0, "dirichlet": 1, "neumann": 2}
MAP = {"affine": 0, "channel": 1, "channel_linear": 2, "perturbed": 3}
OP = {"laplace": 0, "helmholtz": 1, "viscous": 2}
PC = {"none": 0, "jacobi": 1, "invmass": 2, "cheb_f32": 3, "gmg_f32": 4}


class MeshDesc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("bc_lo", C.c_int * 3),
                ("bc_hi", C.c_int * 3), ("map", C.c_int), ("gamma", C.c_double), ("amplitude", C.c_double),
                ("seed", C.c_ulonglong)]


class CgOpts(C.Structure):
    _fields_ = [("op", C.c_int), ("mass_coef", C.c_double), ("nu", C.c_double), ("nu_cell", C.c_void_p),
                ("precond", C.c_int), ("cheb_degree", C.c_int), ("cheb_range", C.c_double),
                ("cheb_lmax", C.c_double), ("cheb_lanczos_steps", C.c_int), ("zero_mean", C.c_int),
                ("rtol", C.c_double), ("maxit", C.c_int), ("flexible", C.c_int), ("use_graph", C.c_int),
                ("check_every", C.c_int), ("mg_degree", C.c_int), ("mg_range", C.c_double),
                ("mg_coarse_tol", C.c_double), ("mg_coarse_maxdeg", C.c_int)]


class NsParams(C.Structure):
    _fields_ = [("k", C.c_int), ("penalty", C.c_double), ("nu", C.c_double), ("dt", C.c_double),
                ("order", C.c_int), ("zeta", C.c_double), ("pressure_precond", C.c_int),
                ("rtol_pressure", C.c_double), ("rtol_viscous", C.c_double), ("rtol_projection", C.c_double),
                ("maxit", C.c_int), ("maxit_projection", C.c_int)]


class NsStats(C.Structure):
    _fields_ = [("order", C.c_int), ("pressure_iters", C.c_int), ("viscous_iters", C.c_int),
                ("projection_iters", C.c_int), ("pressure_relres", C.c_double), ("viscous_relres", C.c_double)]


class SipgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libsipg status %d: %s" % (status, msg))
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "sipg_create_mesh": [C.POINTER(MeshDesc), C.POINTER(C.c_void_p)],
    "sipg_destroy_mesh": [C.c_void_p],
    "sipg_set_degree": [C.c_void_p, C.c_int],
    "sipg_set_penalty": [C.c_void_p, C.c_double],
    "sipg_n_dofs": [C.c_void_p, C.POINTER(C.c_longlong)],
    "sipg_n_cells": [C.c_void_p, C.POINTER(C.c_longlong)],
    "sipg_node_coordinates": [C.c_void_p, C.c_void_p],
    "sipg_penalty_values": [C.c_void_p, C.c_void_p],
    "sipg_apply_laplace_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "sipg_apply_laplace_f32": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "sipg_apply_helmholtz_f64": [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p],
    "sipg_apply_helmholtz_f32": [C.c_void_p, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_void_p],
    "sipg_apply_mass_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "sipg_apply_inverse_mass_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "sipg_diagonal_f64": [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_cg_default_opts": [C.POINTER(CgOpts)],
    "sipg_cg_solve": [C.c_void_p, C.POINTER(CgOpts), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                      C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "sipg_cg_solve_noalloc": [C.c_void_p, C.POINTER(CgOpts), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                              C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "sipg_cg_noalloc_capacity": [C.POINTER(C.c_longlong)],
    "sipg_apply_divergence_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_apply_viscous_f64": [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_apply_gradient_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_apply_convective_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_ns_default_params": [C.POINTER(NsParams)],
    "sipg_ns_create": [C.POINTER(MeshDesc), C.POINTER(NsParams), C.POINTER(C.c_void_p)],
    "sipg_ns_destroy": [C.c_void_p],
    "sipg_ns_mesh": [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)],
    "sipg_ns_set_velocity": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "sipg_ns_step": [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(NsStats)],
    "sipg_ns_velocity": [C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_ns_pressure": [C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_ns_wall_data": [C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong), C.c_void_p],
    "sipg_tau_div_f64": [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p],
    "sipg_apply_divdiv_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_project_divdiv_f64": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                C.POINTER(C.c_int)],
    "sipg_mg_setup": [C.c_void_p, C.POINTER(CgOpts), C.c_void_p],
    "sipg_mg_info": [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                     C.POINTER(C.c_int)],
    "sipg_mg_vcycle": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_adjoint_grad_nu": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "sipg_autotune": [C.c_void_p, C.c_int, C.c_char_p],
    "sipg_set_f64_arithmetic": [C.c_void_p, C.c_int],
    "sipg_get_f64_arithmetic": [C.c_void_p, C.POINTER(C.c_int)],
    "sipg_set_f32_mapping": [C.c_void_p, C.c_int],
    "sipg_get_cells_per_block": [C.c_void_p, C.c_int, C.POINTER(C.c_int)],
    "sipg_set_cells_per_block": [C.c_void_p, C.c_int, C.c_int],
    "sipg_profile_enable": [C.c_void_p, C.c_int],
    "sipg_profile_read": [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                          C.POINTER(C.c_longlong)],
}


def lib():
    """Load libsipg.so (built in-tree by __graft_entry__.build()).  There is no
    fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsipg.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = args
        L.sipg_last_error.restype = C.c_char_p
        L.sipg_last_error.argtypes = []
        _lib = L
    return _lib


def check(status, allow=(OK,)):
    if status not in allow:
        raise SipgError(status, lib().sipg_last_error().decode())
    return status


def exported_symbols():
    """Names of the sipg_* functions declared in include/sipg.h."""
    return sorted(list(_SIGS) + ["sipg_last_error"])
