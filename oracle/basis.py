"""1D quadrature rules and nodal Lagrange polynomials (oracle; test infrastructure).

All rules live on the reference interval [0, 1].

* Sec. 3.1: the shape functions are tensor products of 1D Lagrange polynomials
  on the Legendre-Gauss-Lobatto (GLL) nodes.
* Sec. 5: every non-convective integral uses a Gauss rule with n_q = k + 1
  points per direction.
"""
import numpy as np
from numpy.polynomial import legendre as L


def gauss_rule(n):
    """Gauss-Legendre rule with ``n`` points on [0, 1] (Sec. 5, n_q = k+1).

    numpy's ``leggauss`` serves as the library step; the map from [-1, 1]
    to [0, 1] halves the weights."""
    t, w = L.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gll_rule(p):
    """Gauss-Lobatto-Legendre nodes and weights with ``p = k + 1`` points on [0, 1].

    The interior nodes are the roots of P_k'(t); the weights on [-1, 1] are
    2 / (k (k+1) P_k(t_i)^2)."""
    if p < 2:
        raise ValueError("GLL rule needs at least 2 points")
    k = p - 1
    ck = np.zeros(k + 1)
    ck[k] = 1.0
    interior = np.sort(np.real(L.legroots(L.legder(ck)))) if k >= 2 else np.zeros(0)
    t = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (k * (k + 1) * L.legval(t, ck) ** 2)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[q, a] = l_a(x_q) by the product formula prod_{m != a} (x - z_m)/(z_a - z_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = len(nodes)
    V = np.ones((len(x), p))
    for a in range(p):
        for m in range(p):
            if m != a:
                V[:, a] *= (x - nodes[m]) / (nodes[a] - nodes[m])
    return V


def lagrange_derivatives(nodes, x):
    """D[q, a] = l_a'(x_q): the product rule applied to the product formula,
    sum_{m != a} 1/(z_a - z_m) prod_{n != a, m} (x - z_n)/(z_a - z_n)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = len(nodes)
    D = np.zeros((len(x), p))
    for a in range(p):
        for m in range(p):
            if m == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[m]))
            for n in range(p):
                if n != a and n != m:
                    term *= (x - nodes[n]) / (nodes[a] - nodes[n])
            D[:, a] += term
    return D
