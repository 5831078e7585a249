"""The bake-off problems end to end (oracle; test infrastructure only).

Table 1 and Sec. 3:

* BP1: B u = r, scalar, homogeneous Neumann, q = p+2 GL quadrature.
* BP3: A u = r, scalar, homogeneous Dirichlet, q = p+2 GL quadrature.
* BP5: A u = r, scalar, homogeneous Dirichlet, q = p+1 GLL quadrature (collocated).
* BP2: B u_i = r_i, three components, as BP1 (independent copies sharing the mesh).
* BP4: A u_i = r_i, three components, as BP3.
* BP6: A u_i = r_i, three components, as BP5; the components are independent
  copies of BP5 sharing the mesh and geometry.

Each is solved by Jacobi PCG (``pcg``) on the assembled, Dirichlet-restricted
system.  Vectors are indexed by the canonical global node id; components of a
vector field are stored ``[n_global, ncomp]``.  Dirichlet entries are zero.

The right-hand side b = M Q^T B_L Q f (mass matrix in the BP's own quadrature,
then masked).  For BP5/BP6 that is the diagonal GLL mass of the spectral
element method (Sec. 5, after Eq. (34)), which the collocated full quadrature
reproduces exactly.
"""
from __future__ import annotations

import numpy as np

from .assemble import assemble, masked_apply, restrict
from .element import basis_tables, element_matrices
from .mesh import box_mesh, boundary_nodes, global_count
from .pcg import pcg
from .quadrature import bp_rule


class BakeoffProblem:
    def __init__(self, bp: int, Ex: int, Ey: int, Ez: int, N: int, amp: float = 0.05,
                 kappa: np.ndarray | None = None, rule=None, beta: float = 0.0):
        if bp not in (1, 2, 3, 4, 5, 6):
            raise ValueError("bake-off problems are BP1..BP6")
        self.bp, self.N = bp, N
        self.dims = (Ex, Ey, Ez)
        self.ncomp = 3 if bp in (2, 4, 6) else 1
        self.rule = bp_rule(bp, N) if rule is None else rule
        self.q = len(self.rule[0])
        self.coords, self.l2g = box_mesh(Ex, Ey, Ez, N, amp)
        self.n_global = global_count(Ex, Ey, Ez, N)
        E = Ex * Ey * Ez
        mass_only = bp in (1, 2)
        want = ("B",) if mass_only else ("A", "B")
        Ae, Be = [], []
        for e in range(E):
            k_e = None if kappa is None else kappa[e]
            m = element_matrices(self.coords[e], N, self.rule, kappa=k_e, want=want)
            Be.append(m["B"])
            if "A" in m:
                Ae.append(m["A"])
        self.B = assemble(self.l2g, Be, self.n_global)
        self.A = self.B if mass_only else assemble(self.l2g, Ae, self.n_global)
        if beta != 0.0:
            if mass_only:
                raise ValueError("the Helmholtz term applies to BP3-BP6")
            # H = A + beta B, Eq. (17): the Galerkin form of Eq. (4) with constant beta
            self.A = (self.A + beta * self.B).tocsr()
        if mass_only:
            self.free = np.ones(self.n_global, dtype=bool)
        else:
            self.free = ~boundary_nodes(Ex, Ey, Ez, N)
        self.A_free = restrict(self.A, self.free)
        self.diag_free = self.A_free.diagonal()

    # -- node data ----------------------------------------------------------------
    def node_coords(self) -> np.ndarray:
        X = np.zeros((self.n_global, 3))
        X[self.l2g.reshape(-1)] = self.coords.reshape(-1, 3)
        return X

    def jacobi_inverse(self) -> np.ndarray:
        """1 / diag of the assembled operator on free nodes, 0 on Dirichlet nodes."""
        d = np.zeros(self.n_global)
        d[self.free] = 1.0 / self.diag_free
        return d

    # -- operators ----------------------------------------------------------------
    def apply(self, u: np.ndarray) -> np.ndarray:
        """w = M A M u (BP3-BP6) or w = B u (BP1, BP2), all components."""
        return masked_apply(self.A, self.free, u)

    def mass(self, u: np.ndarray) -> np.ndarray:
        """w = B u with B in the BP's own quadrature (unmasked)."""
        return self.B @ u

    def rhs(self, f_nodes: np.ndarray) -> np.ndarray:
        """b = M B f for nodal data f (masked on Dirichlet nodes)."""
        b = self.B @ f_nodes
        m = self.free.astype(np.float64)
        return b * (m[:, None] if b.ndim == 2 else m)

    def manufactured_rhs(self):
        """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) = -Lap u for u = sin sin sin,
        at the mapped node coordinates; returns (b, u_exact at the nodes)."""
        X = self.node_coords()
        s = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        return self.rhs(3.0 * np.pi ** 2 * s), s

    # -- solver -------------------------------------------------------------------
    def solve(self, b: np.ndarray, tol: float = 1e-8, maxit: int = 10000,
              fixed_iters: int | None = None):
        """Jacobi PCG per component; returns x (full node set) and per-component info."""
        b2 = b.reshape(self.n_global, -1)
        x = np.zeros_like(b2)
        infos = []
        for c in range(b2.shape[1]):
            xf, info = pcg(self.A_free, b2[self.free, c], self.diag_free, tol=tol,
                           maxit=maxit, fixed_iters=fixed_iters)
            x[self.free, c] = xf
            infos.append(info)
        return x.reshape(b.shape), infos

    def quadrature_points(self) -> np.ndarray:
        """Physical coordinates of every element's quadrature points, [E, q^3, 3]."""
        Phi, _ = basis_tables(self.N, self.rule[0])
        return np.einsum("Qa,ead->eQd", Phi, self.coords)
