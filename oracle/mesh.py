"""Structured hexahedral meshes and their iso-parametric mappings (oracle).

* Sec. 3.1: the domain is split into N_e hexahedra; interior faces, Dirichlet
  and Neumann boundaries.
* Sec. 5: geometries are described by iso-parametric polynomial mappings: the
  map of each cell is the degree-k Lagrange interpolant of the analytic map on
  the cell's Gauss-Lobatto nodes.
* Sec. 7.1: the channel grading x_2 -> delta tanh(gamma (2 x_2 - 1)) / tanh(gamma)
  of the wall-normal coordinate (here scaled to [lo_y, hi_y]).
* "perturbed": the box plus a seeded smooth displacement that vanishes on the
  box boundary (a non-separable map for general-metric tests; not in the
  paper, which treats general curved meshes through the same iso-parametric
  mapping).

Cells are numbered lexicographically, x fastest: cell = (iz * ny + iy) * nx + ix.
Nodes inside a cell are numbered i = (c * p + b) * p + a with a along x.
"""
from dataclasses import dataclass, field

import numpy as np

from .basis import gll_rule

PERIODIC, DIRICHLET, NEUMANN = "periodic", "dirichlet", "neumann"


@dataclass
class MeshSpec:
    nx: int
    ny: int
    nz: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc_lo: tuple = (PERIODIC, PERIODIC, PERIODIC)
    bc_hi: tuple = (PERIODIC, PERIODIC, PERIODIC)
    mapping: str = "affine"  # "affine", "channel", "channel_linear" or "perturbed"
    gamma: float = 1.8
    amplitude: float = 0.0   # "perturbed": size of the displacement relative to the box
    seed: int = 0            # "perturbed": selects the displacement's coefficients
    n: tuple = field(init=False)

    def __post_init__(self):
        self.n = (self.nx, self.ny, self.nz)
        for d in range(3):
            if (self.bc_lo[d] == PERIODIC) != (self.bc_hi[d] == PERIODIC):
                raise ValueError("periodic sides must be paired")

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz


def analytic_map(spec, s):
    """Physical coordinates of global reference coordinates s in [0,1]^3 (last axis)."""
    s = np.asarray(s, dtype=np.float64)
    lo = np.asarray(spec.lo, dtype=np.float64)
    hi = np.asarray(spec.hi, dtype=np.float64)
    x = lo + (hi - lo) * s
    if spec.mapping == "channel":
        g = spec.gamma
        t = np.tanh(g * (2.0 * s[..., 1] - 1.0)) / np.tanh(g)
        x[..., 1] = lo[1] + (hi[1] - lo[1]) * 0.5 * (1.0 + t)
    elif spec.mapping == "channel_linear":
        # the tanh grading at the cell boundaries eta_j = j / ny, linear in between
        g, ny = spec.gamma, spec.ny
        j = np.clip(np.floor(s[..., 1] * ny), 0, ny - 1)
        e0, e1 = j / ny, (j + 1) / ny
        y0 = np.tanh(g * (2.0 * e0 - 1.0)) / np.tanh(g)
        y1 = np.tanh(g * (2.0 * e1 - 1.0)) / np.tanh(g)
        t = y0 + (y1 - y0) * (s[..., 1] - e0) * ny
        x[..., 1] = lo[1] + (hi[1] - lo[1]) * 0.5 * (1.0 + t)
    elif spec.mapping == "perturbed":
        x = x + perturbation(spec, s)
    elif spec.mapping != "affine":
        raise ValueError("unknown mapping " + spec.mapping)
    return x


def perturbation_coefficients(seed):
    """c_i in [-1, 1] from 16-bit fields of the seed: c_i = 2 f_i / 65535 - 1."""
    return np.array([2.0 * ((int(seed) >> (16 * i)) & 0xFFFF) / 65535.0 - 1.0 for i in range(3)])


def perturbation(spec, s):
    """A smooth displacement that vanishes on the box boundary and couples the
    directions (a general, non-separable map for general-metric tests):
        w_i = amplitude (hi_i - lo_i) c_i b(s) cos(pi (s_(i+1) - s_(i+2))),
        b(s) = sin(pi s_x) sin(pi s_y) sin(pi s_z)."""
    c = perturbation_coefficients(spec.seed)
    L = np.asarray(spec.hi, dtype=np.float64) - np.asarray(spec.lo, dtype=np.float64)
    b = np.sin(np.pi * s[..., 0]) * np.sin(np.pi * s[..., 1]) * np.sin(np.pi * s[..., 2])
    w = np.zeros_like(s)
    for i in range(3):
        w[..., i] = spec.amplitude * L[i] * c[i] * b * np.cos(np.pi * (s[..., (i + 1) % 3] - s[..., (i + 2) % 3]))
    return w


def cell_index(spec, ix, iy, iz):
    return (np.asarray(iz) * spec.ny + np.asarray(iy)) * spec.nx + np.asarray(ix)


def cell_ijk(spec, cell):
    cell = np.asarray(cell)
    ix = cell % spec.nx
    iy = (cell // spec.nx) % spec.ny
    iz = cell // (spec.nx * spec.ny)
    return ix, iy, iz


def reference_nodes(p):
    """Reference coordinates (p^3, 3) of the GLL nodes of one cell, i = (c p + b) p + a."""
    z, _ = gll_rule(p)
    c, b, a = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    return np.stack([z[a.ravel()], z[b.ravel()], z[c.ravel()]], axis=-1)


def cell_node_coords(spec, p, cells):
    """Geometry nodes (len(cells), p^3, 3): the analytic map at the cell's GLL nodes.

    These are the support points of the iso-parametric degree-k mapping (Sec. 5)."""
    cells = np.atleast_1d(np.asarray(cells))
    ix, iy, iz = cell_ijk(spec, cells)
    ref = reference_nodes(p)
    origin = np.stack([ix, iy, iz], axis=-1).astype(np.float64)
    n = np.asarray(spec.n, dtype=np.float64)
    s = (origin[:, None, :] + ref[None, :, :]) / n
    return analytic_map(spec, s)


def neighbor(spec, cell, d, side):
    """Neighbour across face (d, side) of each cell, and the boundary kind there.

    Returns (nb, kind) arrays; nb = -1 where the face is on a non-periodic boundary.
    kind is 'interior' (including periodic) or the boundary condition name."""
    cell = np.atleast_1d(np.asarray(cell))
    ijk = list(cell_ijk(spec, cell))
    n = spec.n[d]
    step = 1 if side == 1 else -1
    j = ijk[d] + step
    bc = spec.bc_hi[d] if side == 1 else spec.bc_lo[d]
    on_boundary = (j < 0) | (j >= n)
    if bc == PERIODIC:
        j = j % n
        on_boundary = np.zeros_like(on_boundary)
    jj = np.where(on_boundary, 0, j)
    ijk[d] = jj
    nb = cell_index(spec, *ijk)
    nb = np.where(on_boundary, -1, nb)
    return nb, on_boundary, bc
