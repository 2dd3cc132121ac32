"""Adjoint gradient of a viscous Helmholtz solve (oracle; test infrastructure).

The paper has no adjoint.  The operator is the one of Sec. 3.2 (iii) in
Laplace form with a per-cell viscosity: A(nu) = c_m M + L(nu).  For
A(nu) u = f and J = 1/2 (u - u_t)^T M (u - u_t):

  A lambda = M (u - u_t)              (A is symmetric)
  dJ/dnu_e = - lambda^T (dA/dnu_e) u
  dJ/df    = lambda.

dA/dnu_e is read off the element-coupling blocks of the oracle operator:
nu_e multiplies the cell stiffness of e, the consistency pieces in which the
gradient of a function of cell e appears, the Dirichlet faces of e, and the
penalty of every face where nu_e is the max of the two sides (half of it on a
tie, the mean of the one-sided derivatives).
"""
import numpy as np

from .sipg import MINUS, PLUS


def grad_nu(op, nu_cell, u, lam):
    """-lambda^T (dA/dnu_e) u for every cell e (u and lam are single-component)."""
    nu = np.asarray(nu_cell, dtype=np.float64)
    ncell, P = op.spec.ncell, op.P
    U = np.asarray(u, dtype=np.float64).reshape(ncell, P)
    Lm = np.asarray(lam, dtype=np.float64).reshape(ncell, P)
    g = np.zeros(ncell)
    for kc, geo in enumerate(op.geom):
        cells = np.nonzero(op.cell_key == kc)[0]
        g[cells] += np.einsum("ni,ij,nj->n", Lm[cells], geo.K, U[cells])
    for d, km, kp, em, ep in op.faces:
        cu, cv, pen = op.face_pieces(d, km, kp)
        tauF = np.maximum(op.tau[em], op.tau[ep])
        w_m = np.where(nu[em] > nu[ep], 1.0, np.where(nu[em] == nu[ep], 0.5, 0.0))
        w_p = 1.0 - w_m
        side = (em, ep)
        for t in (MINUS, PLUS):
            for s in (MINUS, PLUS):
                lt, us = Lm[side[t]], U[side[s]]
                c_u = np.einsum("ni,ij,nj->n", lt, cu[t][s], us)  # scaled by nu_s
                c_v = np.einsum("ni,ij,nj->n", lt, cv[t][s], us)  # scaled by nu_t
                c_p = tauF * np.einsum("ni,ij,nj->n", lt, pen[t][s], us)
                np.add.at(g, side[s], c_u)
                np.add.at(g, side[t], c_v)
                np.add.at(g, em, w_m * c_p)
                np.add.at(g, ep, w_p * c_p)
    for d, side_, bcells in op.bfaces:
        for kc in np.unique(op.cell_key[bcells]):
            cells = bcells[op.cell_key[bcells] == kc]
            bcons, bpen = op.boundary_pieces(kc, d, side_)
            B = (bcons + bcons.T)[None] + 2.0 * op.tau[cells, None, None] * bpen[None]
            g[cells] += np.einsum("ni,nij,nj->n", Lm[cells], B, U[cells])
    return -g


def grad_nu_magnitude(op, nu_cell, u, lam):
    """sum over the terms of -lambda^T (dA/dnu_e) u of their absolute values,
    |lambda|^T |dA/dnu_e| |u| per cell e, from the same element blocks as
    grad_nu: the scale of the rounding error of any evaluation of dJ/dnu_e
    (summation in any order gives an error of at most a small multiple of the
    unit roundoff times this sum)."""
    nu = np.asarray(nu_cell, dtype=np.float64)
    ncell, P = op.spec.ncell, op.P
    U = np.abs(np.asarray(u, dtype=np.float64)).reshape(ncell, P)
    Lm = np.abs(np.asarray(lam, dtype=np.float64)).reshape(ncell, P)
    g = np.zeros(ncell)
    for kc, geo in enumerate(op.geom):
        cells = np.nonzero(op.cell_key == kc)[0]
        g[cells] += np.einsum("ni,ij,nj->n", Lm[cells], np.abs(geo.K), U[cells])
    for d, km, kp, em, ep in op.faces:
        cu, cv, pen = op.face_pieces(d, km, kp)
        tauF = np.maximum(op.tau[em], op.tau[ep])
        w_m = np.where(nu[em] > nu[ep], 1.0, np.where(nu[em] == nu[ep], 0.5, 0.0))
        w_p = 1.0 - w_m
        side = (em, ep)
        for t in (MINUS, PLUS):
            for s in (MINUS, PLUS):
                lt, us = Lm[side[t]], U[side[s]]
                c_u = np.einsum("ni,ij,nj->n", lt, np.abs(cu[t][s]), us)
                c_v = np.einsum("ni,ij,nj->n", lt, np.abs(cv[t][s]), us)
                c_p = tauF * np.einsum("ni,ij,nj->n", lt, np.abs(pen[t][s]), us)
                np.add.at(g, side[s], c_u)
                np.add.at(g, side[t], c_v)
                np.add.at(g, em, w_m * c_p)
                np.add.at(g, ep, w_p * c_p)
    for d, side_, bcells in op.bfaces:
        for kc in np.unique(op.cell_key[bcells]):
            cells = bcells[op.cell_key[bcells] == kc]
            bcons, bpen = op.boundary_pieces(kc, d, side_)
            B = np.abs(bcons)[None] + np.abs(bcons.T)[None] + 2.0 * op.tau[cells, None, None] * np.abs(bpen)[None]
            g[cells] += np.einsum("ni,nij,nj->n", Lm[cells], B, U[cells])
    return g


def loss(op, u, u_target):
    """J = 1/2 (u - u_t)^T M (u - u_t)."""
    e = np.asarray(u) - np.asarray(u_target)
    return 0.5 * float(e @ op.mass_apply(e))
