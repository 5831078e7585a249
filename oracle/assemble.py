"""Assembly A = Q^T A_L Q and Dirichlet restriction (oracle; test infrastructure only).

Eq. (21): the assembled matrix is Q^T A_L Q with A_L = block-diag(A^e) and Q
the Boolean global-to-local map (l2g).  Entry (g, g') of the assembled matrix
is the sum over elements e and local pairs (a, b) with l2g[e, a] = g,
l2g[e, b] = g' of A^e_ab.  Homogeneous Dirichlet conditions (BP3-BP6, Table 1)
remove the rows and columns of boundary nodes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble(l2g: np.ndarray, mats, n_global: int) -> sp.csr_matrix:
    """Sum the element matrices mats[e] (p1^3 x p1^3) into a global CSR matrix."""
    rows, cols, vals = [], [], []
    for e in range(l2g.shape[0]):
        idx = l2g[e]
        M = mats[e]
        rows.append(np.repeat(idx, len(idx)))
        cols.append(np.tile(idx, len(idx)))
        vals.append(M.reshape(-1))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_global, n_global)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    return A


def restrict(A: sp.csr_matrix, free: np.ndarray) -> sp.csr_matrix:
    """Rows and columns of the free (non-Dirichlet) nodes."""
    idx = np.flatnonzero(free)
    return A[idx][:, idx].tocsr()


def masked_apply(A: sp.csr_matrix, free: np.ndarray, u: np.ndarray) -> np.ndarray:
    """w = M A M u with M the 0/1 diagonal of free nodes (the restricted
    operator extended by zero rows and columns to the full node set)."""
    m = free.astype(np.float64)
    if u.ndim == 2:
        return m[:, None] * (A @ (m[:, None] * u))
    return m * (A @ (m * u))
