"""Pins of the oracle's element matrices, mesh and assembly (CPU only).

* volume: 1^T B 1 = 1 (the deformed box is still the unit cube), exact to
  round-off with any rule that integrates |J| exactly;
* A 1 = 0 for the unconstrained stiffness; symmetry; SPD after masking;
* iso-parametric identity: the coordinate functions lie in the discrete space,
  so x^T A x = y^T A y = z^T A z = sum_Q w_Q |J_Q| and x^T A y = 0;
* undeformed box: the assembled matrix equals the Kronecker sum of 1D matrices
  (a textbook closed form), for both the GLL (BP5) and GL (BP3) rules;
* brute force: assembly by explicit loops over (e, a, b) into a dense matrix;
* the energy of sin(pi x) sin(pi y) sin(pi z) converges spectrally to 3 pi^2 / 8
  on the deformed mesh.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.assemble import assemble
from oracle.basis import lagrange_derivatives, lagrange_values
from oracle.element import basis_tables, element_geometry, element_matrices, tensor_weights
from oracle.mesh import box_mesh, boundary_nodes, global_count
from oracle.problems import BakeoffProblem
from oracle.quadrature import bp_rule, gauss, gll


def _assembled(bp, dims, N, amp, rule=None):
    return BakeoffProblem(bp, *dims, N, amp=amp, rule=rule)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_volume_exact_with_overintegration(N):
    q = -(-3 * N // 2) + 1
    prob = _assembled(3, (2, 1, 2), N, 0.05, rule=gauss(q))
    one = np.ones(prob.n_global)
    assert abs(one @ (prob.B @ one) - 1.0) < 1e-13


@pytest.mark.parametrize("bp", [1, 3, 5])
def test_volume_undeformed(bp):
    prob = _assembled(bp, (2, 2, 1), 3, 0.0)
    one = np.ones(prob.n_global)
    assert abs(one @ (prob.B @ one) - 1.0) < 1e-14


def test_volume_exact_with_bp_rule():
    """The deformation shifts all coordinates by one scalar s, so
    J = (h/2)(I + grad_r s 1^T) and |J| = (h/2)^3 (1 + sum_m d s / d r_m) is
    affine in s; each d s / d r_m has degree 2N-1 at most and integrates to the
    boundary values of s, which are zero.  Both BP rules are exact there."""
    for bp in (5, 3):
        for N in (2, 4, 6):
            prob = _assembled(bp, (1, 2, 1), N, 0.05)
            one = np.ones(prob.n_global)
            assert abs(one @ (prob.B @ one) - 1.0) < 1e-13


@pytest.mark.parametrize("bp,N", [(3, 2), (3, 3), (5, 2), (5, 4)])
def test_stiffness_kernel_symmetry_spd(bp, N):
    prob = _assembled(bp, (2, 1, 2), N, 0.05)
    A = prob.A.toarray()
    one = np.ones(prob.n_global)
    assert np.max(np.abs(A @ one)) < 1e-12 * np.max(np.abs(A))
    np.testing.assert_allclose(A, A.T, atol=1e-13 * np.max(np.abs(A)))
    Af = prob.A_free.toarray()
    assert np.linalg.eigvalsh(Af).min() > 0


@pytest.mark.parametrize("bp,N", [(3, 2), (3, 4), (5, 3), (5, 5)])
def test_isoparametric_identity(bp, N):
    prob = _assembled(bp, (2, 2, 1), N, 0.05)
    X = prob.node_coords()
    points, weights = prob.rule
    _, dPhi = basis_tables(N, points)
    wq = tensor_weights(weights)
    vol = sum(float(wq @ element_geometry(prob.coords[e], dPhi)[1]) for e in range(prob.coords.shape[0]))
    for d in range(3):
        assert abs(X[:, d] @ (prob.A @ X[:, d]) - vol) < 1e-12
    for d, d2 in ((0, 1), (0, 2), (1, 2)):
        assert abs(X[:, d] @ (prob.A @ X[:, d2])) < 1e-12
    one = np.ones(prob.n_global)
    assert abs(one @ (prob.B @ one) - vol) < 1e-13


def _one_d(E1, N, rule):
    """Assembled 1D stiffness and mass on [0, 1] with E1 equal elements."""
    xi, _ = gll(N)
    pts, wts = rule
    h = 1.0 / E1
    Jv = lagrange_values(xi, pts)
    Dv = lagrange_derivatives(xi, pts)
    Ae = Dv.T @ np.diag(wts) @ Dv * (2.0 / h)
    Be = Jv.T @ np.diag(wts) @ Jv * (h / 2.0)
    n = N * E1 + 1
    A1, B1 = np.zeros((n, n)), np.zeros((n, n))
    for e in range(E1):
        s = slice(e * N, e * N + N + 1)
        A1[s, s] += Ae
        B1[s, s] += Be
    return A1, B1


@pytest.mark.parametrize("bp,N,dims", [(5, 2, (2, 3, 1)), (5, 4, (2, 2, 2)), (3, 3, (3, 1, 2)), (1, 2, (2, 2, 1))])
def test_undeformed_kronecker_sum(bp, N, dims):
    prob = _assembled(bp, dims, N, 0.0)
    Ax, Bx = _one_d(dims[0], N, prob.rule)
    Ay, By = _one_d(dims[1], N, prob.rule)
    Az, Bz = _one_d(dims[2], N, prob.rule)
    K = np.kron
    Bref = K(Bz, K(By, Bx))
    np.testing.assert_allclose(prob.B.toarray(), Bref, atol=1e-15 * 10)
    if bp != 1:
        Aref = K(Bz, K(By, Ax)) + K(Bz, K(Ay, Bx)) + K(Az, K(By, Bx))
        np.testing.assert_allclose(prob.A.toarray(), Aref, atol=1e-13 * np.max(np.abs(Aref)))


def test_brute_force_assembly_2x2x2():
    N = 2
    coords, l2g = box_mesh(2, 2, 2, N, 0.05)
    ng = global_count(2, 2, 2, N)
    rule = bp_rule(5, N)
    mats = [element_matrices(coords[e], N, rule, want=("A",))["A"] for e in range(8)]
    dense = np.zeros((ng, ng))
    for e in range(8):
        for a in range(l2g.shape[1]):
            for b in range(l2g.shape[1]):
                dense[l2g[e, a], l2g[e, b]] += mats[e][a, b]
    np.testing.assert_allclose(assemble(l2g, mats, ng).toarray(), dense, atol=1e-14)
    # every global node is reached, shared coordinates agree bitwise
    X = np.full((ng, 3), np.nan)
    for e in range(8):
        for a in range(l2g.shape[1]):
            g = l2g[e, a]
            if not np.isnan(X[g, 0]):
                assert np.array_equal(X[g], coords[e, a])
            X[g] = coords[e, a]
    assert not np.isnan(X).any()
    # Dirichlet set = nodes on the faces of the unit cube
    bnd = boundary_nodes(2, 2, 2, N)
    on_face = np.any((np.abs(X) < 1e-14) | (np.abs(X - 1) < 1e-14), axis=1)
    np.testing.assert_array_equal(bnd, on_face)


def test_energy_converges_to_exact_on_deformed_mesh():
    exact = 3 * np.pi ** 2 / 8
    errs = []
    for N in (2, 4, 6, 8):
        prob = _assembled(5, (2, 2, 2), N, 0.05)
        X = prob.node_coords()
        u = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        errs.append(abs(u @ (prob.A @ u) - exact))
    assert all(errs[i] > errs[i + 1] for i in range(3)), errs
    assert errs[-1] < 1e-5 * exact


def test_mass_collocated_is_diagonal():
    prob = _assembled(5, (2, 1, 1), 4, 0.05)
    B = prob.B.toarray()
    assert np.count_nonzero(B - np.diag(np.diag(B))) == 0


def test_kappa_scales_stiffness():
    N = 3
    coords, _ = box_mesh(1, 1, 1, N, 0.05)
    rule = bp_rule(5, N)
    A1 = element_matrices(coords[0], N, rule, want=("A",))["A"]
    A2 = element_matrices(coords[0], N, rule, kappa=np.full((N + 1) ** 3, 2.5), want=("A",))["A"]
    np.testing.assert_allclose(A2, 2.5 * A1, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("bp,N", [(3, 3), (5, 4), (1, 2)])
def test_row_restricted_matrices_equal_full_rows(bp, N):
    """element_matrices(rows=...) (used for single rows of very large meshes) gives the rows
    of the full element matrices, with and without a coefficient."""
    coords, _ = box_mesh(2, 2, 2, N, 0.05, elements=np.array([5]))
    rule = bp_rule(bp, N)
    rows = [0, 3, (N + 1) ** 3 - 1, N + 2]
    kappa = np.linspace(0.5, 2.0, len(rule[0]) ** 3)
    for kap in (None, kappa):
        full = element_matrices(coords[0], N, rule, kappa=kap)
        part = element_matrices(coords[0], N, rule, kappa=kap, rows=rows)
        for which in ("A", "B"):
            scale = np.max(np.abs(full[which]))
            np.testing.assert_allclose(part[which], full[which][rows], rtol=0, atol=1e-15 * scale)
