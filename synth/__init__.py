"""Seeded synthetic inputs for the CEED bake-off workloads.

This module is shared by the CPU oracle tests, the CUDA-path tests and the
benchmark.  It holds none of the method's arithmetic (no quadrature, no basis,
no geometry, no operator): only the random draws and the problem-size recipes
that define a workload.

* ``uniform_pm1`` -- the counter-based SplitMix64 generator (Steele, Lea and
  Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
  keyed by (seed, canonical global node id), mapped to a double in [-1, 1).
  The value of node ``g`` does not depend on the mesh partition or on the
  order in which nodes are visited.
* ``box_dims`` -- the element array for E = 2^k, the three directions
  differing by at most a factor of two (Sec. 3 of the paper).
* ``sweep_ks`` -- the k values for which 1e4 <= E N^3 <= 1e8.
* ``batched_problems`` -- the draws of the batched BP5 workload.
* ``fourier_modes`` / ``fourier_field`` -- the random Fourier field g(x) that
  defines the variable coefficient kappa = exp(g) of the adjoint workload.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    """One SplitMix64 output for each 64-bit state (state advanced by the golden gamma first)."""
    with np.errstate(over="ignore"):
        z = np.asarray(state, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, ids) -> np.ndarray:
    """Uniform doubles in [-1, 1): ``2 * ((x >> 11) * 2^-53) - 1`` with
    ``x = splitmix64(seed XOR (id * 0x9E3779B97F4A7C15))``."""
    ids = np.asarray(ids, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (ids * _GOLDEN)
    x = splitmix64(key)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def box_dims(k: int) -> tuple[int, int, int]:
    """(Ex, Ey, Ez) with Ex*Ey*Ez = 2^k and no two directions differing by more than 2x."""
    return (2 ** -(-k // 3), 2 ** -(-(k - 1) // 3), 2 ** (k // 3))


def sweep_ks(N: int, n_min: float = 1e4, n_max: float = 1e8) -> list[int]:
    """All k with n_min <= 2^k N^3 <= n_max (problem sizes stepping by 2x)."""
    return [k for k in range(0, 40) if n_min <= (2 ** k) * N ** 3 <= n_max]


def global_node_count(Ex: int, Ey: int, Ez: int, N: int) -> int:
    return (N * Ex + 1) * (N * Ey + 1) * (N * Ez + 1)


def batched_problems(n_problems: int = 256, seed: int = 0, orders=(3, 5, 7),
                     k_max: int = 16, amp_max: float = 0.1) -> list[dict]:
    """Draws for the batched BP5 workload: per problem E = k^3 with k log-uniform
    in [2, k_max] (k = min(k_max, floor(exp(U(ln 2, ln(k_max + 1)))))), N drawn
    from ``orders``, deformation amplitude U[0, amp_max], RHS seed = problem index."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        k = min(k_max, int(math.floor(math.exp(rng.uniform(math.log(2.0), math.log(k_max + 1.0))))))
        N = int(orders[int(rng.integers(0, len(orders)))])
        amp = float(rng.uniform(0.0, amp_max))
        out.append({"k": k, "N": N, "amp": amp, "rhs_seed": i})
    return out


def fourier_modes(seed: int, n_modes: int = 16, kmax: int = 4, amplitude: float = 0.5):
    """Random Fourier modes: integer wave vectors in {1..kmax}^3, coefficients
    c_m ~ U[-1, 1] scaled by amplitude / kmax, phases U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    kvec = rng.integers(1, kmax + 1, size=(n_modes, 3)).astype(np.float64)
    coef = rng.uniform(-1.0, 1.0, size=n_modes) * (amplitude / kmax)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return kvec, coef, phase


def fourier_field(modes, x: np.ndarray) -> np.ndarray:
    """g(x) = sum_m c_m sin(pi k_m . x + phi_m) at points x[..., 3]."""
    kvec, coef, phase = modes
    arg = math.pi * np.tensordot(np.asarray(x, dtype=np.float64), kvec.T, axes=1) + phase
    return np.sin(arg) @ coef
