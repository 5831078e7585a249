"""Single rows of the assembled operators at any mesh size (oracle; test infrastructure only).

Row g of w = M Q^T A_L Q M u (Eq. (21)) only involves the elements that
contain node g, so it can be evaluated one node at a time on meshes far too
large to assemble: w_g = sum_{e owns g} sum_b A^e[a(e, g), b] u[l2g[e, b]].
"""
from __future__ import annotations

import numpy as np

from .element import element_matrices
from .mesh import box_mesh, elements_touching, global_count
from .quadrature import bp_rule


def _is_boundary(g, Ex, Ey, Ez, N):
    nx, ny, nz = N * Ex + 1, N * Ey + 1, N * Ez + 1
    I, J, K = g % nx, (g // nx) % ny, g // (nx * ny)
    return (I == 0) | (I == nx - 1) | (J == 0) | (J == ny - 1) | (K == 0) | (K == nz - 1)


def sampled_rows(bp: int, Ex: int, Ey: int, Ez: int, N: int, amp: float, u_of, nodes,
                 operator: str = "A", kappa_of=None) -> np.ndarray:
    """w[nodes] for operator "A" (stiffness, masked for BP3/5/6; mass for BP1) or
    "B" (mass in the BP's quadrature, unmasked).  ``u_of(ids)`` returns the input
    vector at the given global ids (shape [len(ids)] or [len(ids), ncomp]);
    ``kappa_of(e)`` returns kappa at element e's quadrature points (or None)."""
    nodes = np.asarray(nodes, dtype=np.int64)
    rule = bp_rule(bp, N)
    elems = elements_touching(Ex, Ey, Ez, N, nodes)
    coords, l2g = box_mesh(Ex, Ey, Ez, N, amp, elements=elems)
    dirichlet = bp not in (1, 2) and operator == "A"
    out = None
    where = {int(g): i for i, g in enumerate(nodes)}
    for el in range(len(elems)):
        idx = l2g[el]
        hit = [a for a, g in enumerate(idx) if int(g) in where]
        if not hit:
            continue
        which = "B" if (bp in (1, 2) or operator == "B") else "A"
        kap = None if kappa_of is None else kappa_of(int(elems[el]))
        M = element_matrices(coords[el], N, rule, kappa=kap, want=(which,), rows=hit)[which]
        ue = np.asarray(u_of(idx), dtype=np.float64)
        if dirichlet:
            bmask = _is_boundary(idx, Ex, Ey, Ez, N)
            ue = ue * (~bmask if ue.ndim == 1 else ~bmask[:, None])
        if out is None:
            out = np.zeros((len(nodes),) + ue.shape[1:])
        for r, a in enumerate(hit):
            out[where[int(idx[a])]] += M[r] @ ue
    if dirichlet:
        bmask = _is_boundary(nodes, Ex, Ey, Ez, N)
        out = out * (~bmask if out.ndim == 1 else ~bmask[:, None])
    return out


def all_nodes(Ex, Ey, Ez, N):
    return np.arange(global_count(Ex, Ey, Ez, N), dtype=np.int64)
