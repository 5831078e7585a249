"""Node samples for checking large meshes row by row against the oracle.

For each probe element the sample holds its 8 vertex nodes (shared by up to 8
elements), one node inside each of its 12 edges (up to 4 elements), one inside
each of its 6 faces (2 elements) and some interior nodes (1 element), so every
sharing pattern of the gather-scatter sum is exercised; a few nodes drawn from
the whole mesh are added.
"""
from __future__ import annotations

import numpy as np


def probe_elements(dims, count: int = 5) -> list[int]:
    """The last element (it sits in the last thread block of every launch shape), the first,
    the middle one, the far corner of the first x-y layer and one in the last quarter."""
    Ex, Ey, Ez = dims
    E = Ex * Ey * Ez
    order = [E - 1, 0, E // 2, Ex * Ey - 1, (E * 3) // 4 + Ex // 2]
    out = []
    for e in order:
        if e not in out:
            out.append(e)
    return sorted(out[:count])


def element_node_sample(dims, N: int, e: int, n_interior: int, rng) -> list[int]:
    Ex, Ey, _ = dims
    nx, ny = N * Ex + 1, N * Ey + 1
    ex, ey, ez = e % Ex, (e // Ex) % Ey, e // (Ex * Ey)

    def gid(i, j, k):
        return (ex * N + i) + nx * ((ey * N + j) + ny * (ez * N + k))

    inner = list(range(1, N)) if N > 1 else []
    out = [gid(i, j, k) for k in (0, N) for j in (0, N) for i in (0, N)]
    if inner:
        pick = lambda: int(rng.choice(inner))  # noqa: E731
        for a in (0, N):
            for b in (0, N):
                out += [gid(pick(), a, b), gid(a, pick(), b), gid(a, b, pick())]
        for a in (0, N):
            out += [gid(a, pick(), pick()), gid(pick(), a, pick()), gid(pick(), pick(), a)]
        out += [gid(pick(), pick(), pick()) for _ in range(n_interior)]
    return out


def probe_nodes(dims, N: int, seed: int, n_interior: int = 24, n_random: int = 16, n_probe: int = 5) -> np.ndarray:
    """Sorted unique global node ids (canonical numbering of the box mesh)."""
    rng = np.random.default_rng(seed)
    Ex, Ey, Ez = dims
    n = (N * Ex + 1) * (N * Ey + 1) * (N * Ez + 1)
    out = []
    for e in probe_elements(dims, n_probe):
        out += element_node_sample(dims, N, e, n_interior, rng)
    out += [int(v) for v in rng.integers(0, n, n_random)] + [0, n - 1]
    return np.unique(np.array(out, dtype=np.int64))
