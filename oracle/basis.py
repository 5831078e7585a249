"""Lagrange interpolants on the GLL points (oracle; test infrastructure only).

Sec. 4, Eq. (18): the element map and every field are expanded in the
Lagrange polynomials h_i built on the p+1 GLL points xi_j.  Values and
derivatives are evaluated directly from the product definition

    h_i(x)  = prod_{m != i} (x - xi_m) / (xi_i - xi_m)
    h_i'(x) = sum_{m != i} 1/(xi_i - xi_m) prod_{l != i, m} (x - xi_l) / (xi_i - xi_l)

and not from any closed-form derivative matrix.
"""
from __future__ import annotations

import numpy as np


def lagrange_values(nodes, x) -> np.ndarray:
    """L[r, i] = h_i(x_r)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    L = np.ones((len(x), n))
    for i in range(n):
        for m in range(n):
            if m != i:
                L[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return L


def lagrange_derivatives(nodes, x) -> np.ndarray:
    """Dm[r, i] = h_i'(x_r)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    Dm = np.zeros((len(x), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for l in range(n):
                if l != i and l != m:
                    term *= (x - nodes[l]) / (nodes[i] - nodes[l])
            Dm[:, i] += term
    return Dm
