"""Element stiffness and mass matrices by naive full quadrature (oracle; test infrastructure only).

Sec. 4: A_{l'l} = a(phi_l', phi_l) with a(v, u) = int mu grad v . grad u (Eqs. (6), (14))
and B_{l'l} = (phi_l', phi_l) (Eqs. (7), (15)), restricted to one element
Omega^e, with the element map of Eq. (18) and the q-point tensor quadrature of
Table 1.  Every element matrix is formed entry by entry from the 3D basis
tables -- no sum factorization:

    phi_a(eta_Q)       = h_i(eta_qx) h_j(eta_qy) h_k(eta_qz)
    J_dm(eta_Q)        = sum_a x^e_{a,d} d phi_a / d r_m      (Jacobian of Eq. (18))
    grad phi_a         = J^{-T} grad_r phi_a
    A^e_ab             = sum_Q w_Q |J_Q| kappa_Q grad phi_a . grad phi_b
    B^e_ab             = sum_Q w_Q |J_Q| phi_a phi_b

with w_Q = rho_qx rho_qy rho_qz.  Index conventions: quadrature point
Q = qx + q (qy + q qz) and local node a = i + p1 (j + p1 k).
"""
from __future__ import annotations

import numpy as np

from .basis import lagrange_derivatives, lagrange_values
from .quadrature import gll


def basis_tables(N: int, points):
    """3D tables Phi[Q, a] and dPhi[m][Q, a] (m = r, s, t) at the tensor points."""
    xi, _ = gll(N)
    h = lagrange_values(xi, points)
    dh = lagrange_derivatives(xi, points)
    q, p1 = h.shape

    def table(fz, fy, fx):
        t = np.einsum("zk,yj,xi->zyxkji", fz, fy, fx)
        return t.reshape(q ** 3, p1 ** 3)

    Phi = table(h, h, h)
    dPhi = [table(h, h, dh), table(h, dh, h), table(dh, h, h)]
    return Phi, dPhi


def tensor_weights(weights) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    return np.einsum("z,y,x->zyx", w, w, w).reshape(-1)


def element_geometry(xe: np.ndarray, dPhi):
    """Jacobian J[Q, d, m] = d x_d / d r_m, its determinant and inverse at each point."""
    J = np.stack([dPhi[m] @ xe for m in range(3)], axis=2)  # [Q, d, m]
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)  # Jinv[Q, m, d] = d r_m / d x_d
    return J, detJ, Jinv


def physical_gradients(Jinv: np.ndarray, dPhi) -> np.ndarray:
    """grad[Q, a, d] = sum_m (d r_m / d x_d) (d phi_a / d r_m)."""
    return sum(dPhi[m][:, :, None] * Jinv[:, m, None, :] for m in range(3))


_TABLES: dict = {}


def _cached_tables(N: int, points):
    key = (N, tuple(np.asarray(points, dtype=np.float64).tolist()))
    if key not in _TABLES:
        if len(_TABLES) > 4:
            _TABLES.clear()
        _TABLES[key] = basis_tables(N, points)
    return _TABLES[key]


def element_matrices(xe: np.ndarray, N: int, rule, kappa=None, want=("A", "B"), rows=None):
    """Stiffness A^e and/or mass B^e of one element with nodal coordinates
    ``xe[p1^3, 3]`` under the quadrature ``rule = (points, weights)``.
    ``kappa[Q]`` is the coefficient mu at the quadrature points (1 if None).
    ``rows`` (local node ids) restricts the result to those rows of the same
    entry-by-entry sums, A^e[rows, :] and B^e[rows, :]."""
    points, weights = rule
    Phi, dPhi = _cached_tables(N, points)
    sel = slice(None) if rows is None else np.asarray(rows, dtype=np.int64)
    wq = tensor_weights(weights)
    _, detJ, Jinv = element_geometry(xe, dPhi)
    scale = wq * detJ
    out = {}
    if "A" in want:
        coef = scale if kappa is None else scale * np.asarray(kappa, dtype=np.float64)
        if rows is None:
            grad = physical_gradients(Jinv, dPhi)
            Ae = np.zeros((Phi.shape[1], Phi.shape[1]))
            for d in range(3):
                Gd = grad[:, :, d]
                Ae += Gd.T @ (coef[:, None] * Gd)
        else:
            # the same sums for the requested rows only: one physical-gradient
            # component [Q, a] at a time instead of the whole [Q, a, 3] table
            Ae = np.zeros((len(sel), Phi.shape[1]))
            for d in range(3):
                Gd = sum(dPhi[m] * Jinv[:, m, d][:, None] for m in range(3))
                Ae += (coef[:, None] * Gd[:, sel]).T @ Gd
        out["A"] = Ae
    if "B" in want:
        out["B"] = Phi[:, sel].T @ (scale[:, None] * Phi)
    return out


def point_stiffness(xe: np.ndarray, N: int, rule, Q: int) -> np.ndarray:
    """d A^e / d kappa_Q: the element stiffness of the single quadrature point Q."""
    points, weights = rule
    _, dPhi = basis_tables(N, points)
    wq = tensor_weights(weights)
    _, detJ, Jinv = element_geometry(xe, dPhi)
    grad = physical_gradients(Jinv, dPhi)[Q]  # [a, d]
    return wq[Q] * detJ[Q] * (grad @ grad.T)
