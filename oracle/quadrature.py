"""Gauss-Lobatto-Legendre and Gauss-Legendre rules on [-1, 1] (oracle; test infrastructure only).

The paper's nodal points are the p+1 GLL points xi_j (Sec. 4, after Eq. (18));
BP1-BP4 integrate with q = p+2 GL points, BP5-BP6 with the q = p+1 GLL points
(Table 1).  The rules are the textbook ones (Deville, Fischer and Mund 2002):

* GLL: xi_0 = -1, xi_N = +1 and the N-1 roots of P_N'; weights 2 / (N (N+1) P_N(xi_j)^2).
* GL:  the q roots of P_q; weights 2 / ((1 - eta^2) P_q'(eta)^2).

Roots are found by Newton iteration in extended precision (numpy longdouble)
and rounded to double; symmetric pairs are made exact negatives and the middle
point of an odd rule is exactly 0.
"""
from __future__ import annotations

import numpy as np

_LD = np.longdouble


def legendre(n: int, x):
    """P_n(x), P_n'(x), P_n''(x) by the three-term recurrences

    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
    P'_{k+1}  = P'_{k-1}  + (2k+1) P_k,
    P''_{k+1} = P''_{k-1} + (2k+1) P'_k.
    """
    x = np.asarray(x, dtype=_LD)
    one = np.ones_like(x)
    zero = np.zeros_like(x)
    if n == 0:
        return one, zero, zero
    p_prev, p = one, x
    d_prev, d = zero, one
    dd_prev, dd = zero, zero
    for k in range(1, n):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        d_next = d_prev + (2 * k + 1) * p
        dd_next = dd_prev + (2 * k + 1) * d
        p_prev, p = p, p_next
        d_prev, d = d, d_next
        dd_prev, dd = dd, dd_next
    return p, d, dd


def _symmetrize(x: np.ndarray) -> np.ndarray:
    x = np.sort(np.asarray(x, dtype=np.float64))
    n = len(x)
    for i in range(n // 2):
        v = 0.5 * (x[n - 1 - i] - x[i])
        x[i], x[n - 1 - i] = -v, v
    if n % 2 == 1:
        x[n // 2] = 0.0
    return x


def _newton(f, x0, iters=100):
    x = np.asarray(x0, dtype=_LD)
    for _ in range(iters):
        val, der = f(x)
        step = val / der
        x = x - step
        if np.max(np.abs(step)) < _LD(1e-30):
            break
    return x


def gll(N: int):
    """N+1 GLL points (ascending, xi_0 = -1, xi_N = 1) and weights."""
    if N < 1:
        raise ValueError("GLL rule needs N >= 1")
    if N == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    j = np.arange(1, N, dtype=_LD)
    guess = -np.cos(np.pi * j / N)  # Chebyshev-Gauss-Lobatto interior points

    def f(x):
        _, d, dd = legendre(N, x)
        return d, dd

    interior = _newton(f, guess)
    x = np.concatenate(([_LD(-1)], interior, [_LD(1)]))
    p, _, _ = legendre(N, x)
    w = _LD(2) / (_LD(N * (N + 1)) * p * p)
    xs = _symmetrize(x.astype(np.float64))
    ws = w.astype(np.float64)
    ws = 0.5 * (ws + ws[::-1])
    return xs, ws


def gauss(q: int):
    """q Gauss-Legendre points (ascending) and weights."""
    if q < 1:
        raise ValueError("Gauss rule needs q >= 1")
    i = np.arange(q, dtype=_LD)
    guess = -np.cos(np.pi * (i + _LD(0.75)) / (q + _LD(0.5)))

    def f(x):
        p, d, _ = legendre(q, x)
        return p, d

    x = _newton(f, guess)
    _, d, _ = legendre(q, x)
    w = _LD(2) / ((_LD(1) - x * x) * d * d)
    xs = _symmetrize(x.astype(np.float64))
    ws = w.astype(np.float64)
    ws = 0.5 * (ws + ws[::-1])
    return xs, ws


def bp_rule(bp: int, N: int):
    """Quadrature rule of bake-off problem ``bp`` at order N (Table 1):
    BP1-BP4 use q = N+2 Gauss points, BP5-BP6 the q = N+1 GLL points."""
    if bp in (1, 2, 3, 4):
        return gauss(N + 2)
    if bp in (5, 6):
        return gll(N)
    raise ValueError(f"unknown bake-off problem {bp}")
