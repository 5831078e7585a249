"""Adjoint gradient dJ/dkappa for variable-coefficient Poisson (oracle; test infrastructure only).

Eq. (4) with mu = kappa(x), beta = 0 and homogeneous Dirichlet conditions:
the discrete system is A(kappa) u = b with
A(kappa) = sum_{e,Q} kappa_{e,Q} A_{e,Q} (A_{e,Q} the stiffness of the single
quadrature point Q of element e).  For J = 1/2 (u - u*)^T B (u - u*):

    dJ/dkappa_{e,Q} = -lambda^T A_{e,Q} u,   A lambda = B (u - u*)   (A symmetric)
                    = -w_Q |J_Q| grad lambda(Q) . grad u(Q)   (element e's expansions)

The first form, with dense point matrices, is the definition; the second is
the same number evaluated from nodal values.
"""
from __future__ import annotations

import numpy as np

from .element import basis_tables, element_geometry, physical_gradients, tensor_weights
from .problems import BakeoffProblem


def objective(prob: BakeoffProblem, u: np.ndarray, u_star: np.ndarray) -> float:
    d = u - u_star
    return 0.5 * float(d @ (prob.B @ d))


def forward_adjoint(prob: BakeoffProblem, b: np.ndarray, u_star: np.ndarray, tol: float = 1e-13):
    """Solve the forward and adjoint systems; returns u, lambda, J and the infos."""
    u, info_u = prob.solve(b, tol=tol)
    rhs_adj = prob.rhs(u - u_star)
    lam, info_l = prob.solve(rhs_adj, tol=tol)
    return u, lam, objective(prob, u, u_star), (info_u[0], info_l[0])


def gradient(prob: BakeoffProblem, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """g[e, Q] = -w_Q |J_Q| grad lambda . grad u at every quadrature point."""
    points, weights = prob.rule
    _, dPhi = basis_tables(prob.N, points)
    wq = tensor_weights(weights)
    E = prob.coords.shape[0]
    g = np.zeros((E, len(wq)))
    for e in range(E):
        _, detJ, Jinv = element_geometry(prob.coords[e], dPhi)
        grad = physical_gradients(Jinv, dPhi)  # [Q, a, d]
        gu = np.einsum("Qad,a->Qd", grad, u[prob.l2g[e]])
        gl = np.einsum("Qad,a->Qd", grad, lam[prob.l2g[e]])
        g[e] = -wq * detJ * np.einsum("Qd,Qd->Q", gl, gu)
    return g
