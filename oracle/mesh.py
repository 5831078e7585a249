"""Deformed-box mesh, global-to-local map Q and Dirichlet set (oracle; test infrastructure only).

Sec. 3: E elements arranged in a tensor-product array on a box; the elements
are treated as general curvilinear hexahedra with an iso-parametric map
(Eq. (18)) whose nodal coordinates x^e_ijk sit at the GLL points.

* Undeformed node of element (ex, ey, ez), local node (i, j, k):
  x = (ex + (xi_i + 1)/2) / Ex, and likewise y, z.
* Deformation of the benchmark workloads: every coordinate is shifted by the
  same scalar a * sin(pi x) sin(pi y) sin(pi z), the sines evaluated at the
  undeformed point.  It vanishes on the boundary of the unit cube, so the
  domain stays the unit cube.
* Element id e = ex + Ex (ey + Ey ez); local node a = i + p1 (j + p1 k) with
  p1 = N + 1 (i fastest).
* Canonical global id g = I + (N Ex + 1) (J + (N Ey + 1) K) with I = ex N + i
  etc.  l2g[e, a] = g is the Boolean map Q of Eq. (21): u_L = Q u.
* Dirichlet set: the nodes on the boundary of the box (I, J or K at 0 or its
  maximum).
"""
from __future__ import annotations

import numpy as np

from .quadrature import gll


def global_count(Ex: int, Ey: int, Ez: int, N: int) -> int:
    return (N * Ex + 1) * (N * Ey + 1) * (N * Ez + 1)


def element_ids_to_xyz(elements, Ex, Ey):
    e = np.asarray(elements, dtype=np.int64)
    return e % Ex, (e // Ex) % Ey, e // (Ex * Ey)


def box_mesh(Ex: int, Ey: int, Ez: int, N: int, amp: float, elements=None):
    """Coordinates ``coords[nel, p1^3, 3]`` and map ``l2g[nel, p1^3]`` for the
    given element ids (all elements if None)."""
    p1 = N + 1
    xi, _ = gll(N)
    if elements is None:
        elements = np.arange(Ex * Ey * Ez, dtype=np.int64)
    ex, ey, ez = element_ids_to_xyz(elements, Ex, Ey)
    nel = len(ex)
    coords = np.zeros((nel, p1 ** 3, 3))
    l2g = np.zeros((nel, p1 ** 3), dtype=np.int64)
    nx, ny = N * Ex + 1, N * Ey + 1
    for e in range(nel):
        for k in range(p1):
            for j in range(p1):
                for i in range(p1):
                    a = i + p1 * (j + p1 * k)
                    x0 = (ex[e] + (xi[i] + 1.0) / 2.0) / Ex
                    y0 = (ey[e] + (xi[j] + 1.0) / 2.0) / Ey
                    z0 = (ez[e] + (xi[k] + 1.0) / 2.0) / Ez
                    s = amp * np.sin(np.pi * x0) * np.sin(np.pi * y0) * np.sin(np.pi * z0)
                    coords[e, a] = (x0 + s, y0 + s, z0 + s)
                    I, J, K = ex[e] * N + i, ey[e] * N + j, ez[e] * N + k
                    l2g[e, a] = I + nx * (J + ny * K)
    return coords, l2g


def boundary_nodes(Ex: int, Ey: int, Ez: int, N: int) -> np.ndarray:
    """Boolean flag per global node: True on the boundary of the box."""
    nx, ny, nz = N * Ex + 1, N * Ey + 1, N * Ez + 1
    g = np.arange(nx * ny * nz, dtype=np.int64)
    I, J, K = g % nx, (g // nx) % ny, g // (nx * ny)
    return (I == 0) | (I == nx - 1) | (J == 0) | (J == ny - 1) | (K == 0) | (K == nz - 1)


def elements_touching(Ex: int, Ey: int, Ez: int, N: int, nodes) -> np.ndarray:
    """Ids of all elements that contain any of the given global nodes (used to
    evaluate single rows of the assembled operator at large sizes)."""
    nx, ny = N * Ex + 1, N * Ey + 1
    out = set()
    for g in np.asarray(nodes, dtype=np.int64):
        I, J, K = g % nx, (g // nx) % ny, g // (nx * ny)
        cx = {I // N, (I - 1) // N} if I % N == 0 else {I // N}
        cy = {J // N, (J - 1) // N} if J % N == 0 else {J // N}
        cz = {K // N, (K - 1) // N} if K % N == 0 else {K // N}
        for a in cx:
            for b in cy:
                for c in cz:
                    if 0 <= a < Ex and 0 <= b < Ey and 0 <= c < Ez:
                        out.add(int(a + Ex * (b + Ey * c)))
    return np.array(sorted(out), dtype=np.int64)
