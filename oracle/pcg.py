"""Jacobi-preconditioned conjugate gradients (oracle; test infrastructure only).

Sec. 3: each bake-off problem is diagonally preconditioned CG on the assembled
system.  This is the textbook Hestenes-Stiefel PCG (Saad, Iterative Methods for
Sparse Linear Systems, Alg. 9.1) with M = diag(A):

    r0 = b - A x0,  z0 = M^-1 r0,  p0 = z0
    alpha = (r, z) / (A p, p);  x += alpha p;  r -= alpha A p
    z = M^-1 r;  beta = (r_new, z_new) / (r, z);  p = z + beta p

It stops at the first iteration with ||r||_2 <= tol ||b||_2 (the recursive
residual), or after exactly ``fixed_iters`` iterations when that is given.
"""
from __future__ import annotations

import numpy as np


def pcg(A, b: np.ndarray, diag: np.ndarray, tol: float = 1e-8, maxit: int = 10000,
        fixed_iters: int | None = None, x0: np.ndarray | None = None):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    z = r / diag
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    history = [float(np.linalg.norm(r))]
    its = 0
    limit = fixed_iters if fixed_iters is not None else maxit
    converged = False
    while its < limit:
        if fixed_iters is None and history[-1] <= tol * bnorm:
            converged = True
            break
        w = A @ p
        pAp = float(p @ w)
        if not (pAp > 0.0):
            raise FloatingPointError(f"CG breakdown: p^T A p = {pAp}")
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * w
        z = r / diag
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        its += 1
        history.append(float(np.linalg.norm(r)))
    if fixed_iters is None and not converged and history[-1] <= tol * bnorm:
        converged = True
    return x, {"iters": its, "res_norm": history[-1], "b_norm": bnorm,
               "rel_res": history[-1] / bnorm if bnorm > 0 else 0.0,
               "history": history, "converged": converged}
