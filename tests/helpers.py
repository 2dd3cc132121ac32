"""Shared test helpers: mesh cases described once for both the oracle and the
CUDA library, seeded inputs, and the scaled parity metric."""
import math

import numpy as np

from oracle.mesh import MeshSpec
from paper_1607_01323_gb300 import inputs

TWO_PI = 2 * math.pi


def case(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3,
         mapping="affine", gamma=1.8, amplitude=0.0, seed=0):
    return dict(n=tuple(n), lo=tuple(lo), hi=tuple(hi), bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi), mapping=mapping,
                gamma=gamma, amplitude=amplitude, seed=seed)


def channel(n, wall="dirichlet", gamma=1.8, L=(TWO_PI, 2.0, math.pi)):
    return case(n, lo=(0.0, -L[1] / 2, 0.0), hi=(L[0], L[1] / 2, L[2]), bc_lo=("periodic", wall, "periodic"),
                bc_hi=("periodic", wall, "periodic"), mapping="channel", gamma=gamma)


def oracle_spec(c):
    return MeshSpec(c["n"][0], c["n"][1], c["n"][2], lo=c["lo"], hi=c["hi"], bc_lo=c["bc_lo"], bc_hi=c["bc_hi"],
                    mapping=c["mapping"], gamma=c["gamma"], amplitude=c.get("amplitude", 0.0), seed=c.get("seed", 0))


def gpu_mesh(c, k, penalty=1.0):
    from paper_1607_01323_gb300 import Mesh
    return Mesh(c["n"], c["lo"], c["hi"], c["bc_lo"], c["bc_hi"], mapping=c["mapping"], gamma=c["gamma"], k=k,
                penalty=penalty, amplitude=c.get("amplitude", 0.0), seed=c.get("seed", 0))


def ncell(c):
    return c["n"][0] * c["n"][1] * c["n"][2]


def uniform(n, stream="x", seed=0):
    return inputs.uniform(seed, stream, n)


def scaled_err(y, y_ref, norm_a, x):
    """max|y - y_ref| / (||A||_inf ||x||_inf): the parity metric."""
    return float(np.max(np.abs(np.asarray(y) - np.asarray(y_ref))) / (norm_a * np.max(np.abs(x))))
