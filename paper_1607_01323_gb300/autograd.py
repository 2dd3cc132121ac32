"""torch.autograd wrappers of the solve and the mass matrix (hand-written adjoint).

HelmholtzSolve: u = A(nu)^-1 f with A(nu) = mass_coef M + L(nu), nu per cell.
Its backward solves the adjoint system A lambda = dJ/du with the same CG (A is
symmetric) and returns dJ/dnu_e = -lambda^T (dA/dnu_e) u (sipg_adjoint_grad_nu)
and dJ/df = lambda.  MassApply: y = M x with backward M g (M symmetric).
All work runs in libsipg's kernels.
"""
import torch

from . import adjoint_grad_nu, apply_mass_f64, cg_solve


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nu_cell, f, mesh, mass_coef, rtol, precond):
        u, res = cg_solve(mesh, f.contiguous(), op="helmholtz", mass_coef=mass_coef, nu=0.0,
                          nu_cell=nu_cell.contiguous(), precond=precond, rtol=rtol)
        ctx.save_for_backward(nu_cell, u)
        ctx.mesh, ctx.mass_coef, ctx.rtol, ctx.precond = mesh, mass_coef, rtol, precond
        ctx.iters = res.iters
        return u

    @staticmethod
    def backward(ctx, gu):
        nu_cell, u = ctx.saved_tensors
        lam, _ = cg_solve(ctx.mesh, gu.contiguous(), op="helmholtz", mass_coef=ctx.mass_coef, nu=0.0,
                          nu_cell=nu_cell.contiguous(), precond=ctx.precond, rtol=ctx.rtol)
        g_nu = adjoint_grad_nu(ctx.mesh, nu_cell.contiguous(), u, lam)
        return g_nu, lam, None, None, None, None


class MassApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, mesh):
        ctx.mesh = mesh
        return apply_mass_f64(mesh, x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return apply_mass_f64(ctx.mesh, g.contiguous()), None


def helmholtz_solve(mesh, nu_cell, f, mass_coef, rtol=1e-12, precond="jacobi"):
    return HelmholtzSolve.apply(nu_cell, f, mesh, float(mass_coef), float(rtol), precond)


def mass_norm_loss(mesh, u, u_target):
    """J = 1/2 (u - u_t)^T M (u - u_t)."""
    e = u - u_target
    return 0.5 * torch.dot(e, MassApply.apply(e, mesh))
