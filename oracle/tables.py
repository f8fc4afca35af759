"""1D tables of the Q_p element (oracle; test infrastructure only).

Section 2.2 uses Q_p tensor-product Lagrange elements and Section 2.4 integrates with
(p+1)^d Gauss points (Table tab:input_parameters_3d: q = p + 1).  The paper does not
name the node family; this oracle takes Gauss-Lobatto-Legendre (GLL) nodes, which equal
equispaced nodes for p <= 2.

Everything is on the reference interval [0, 1].
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre points and weights on [0, 1] (numpy's leggauss, mapped)."""
    t, w = npleg.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gll_nodes(p: int) -> np.ndarray:
    """p+1 Gauss-Lobatto-Legendre nodes on [0, 1]: the end points and the roots of P_p'."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    interior = np.sort(npleg.Legendre.basis(p).deriv().roots().real) if p > 1 else np.zeros(0)
    t = np.concatenate(([-1.0], interior, [1.0]))
    return 0.5 * (t + 1.0)


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[q, i] = l_i(x_q), l_i the Lagrange polynomial of `nodes` with l_i(nodes_j) = delta_ij."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    out = np.ones((x.size, n))
    for i in range(n):
        for j in range(n):
            if j != i:
                out[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return out


def lagrange_derivatives(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[q, i] = l_i'(x_q) by the product rule: sum over m != i of the product with factor m differentiated."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    out = np.zeros((x.size, n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            out[:, i] += term
    return out


def element_tables(p: int):
    """(nodes, qp, w, B, D): GLL nodes, Gauss points/weights, B[q,i] = l_i(x_q), D[q,i] = l_i'(x_q)."""
    nodes = gll_nodes(p)
    xq, wq = gauss_legendre(p + 1)
    return nodes, xq, wq, lagrange_values(nodes, xq), lagrange_derivatives(nodes, xq)
