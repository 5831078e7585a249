"""Pins of the oracle's PCG, right-hand sides, sampled rows and adjoint (CPU only).

* PCG against a dense direct solve on small meshes, to the residual tolerance;
* fixed-iteration mode runs exactly that many iterations; breakdown is detected;
* manufactured solution (config of a 4x4x4-style BP5 problem, scaled down):
  the nodal error against sin(pi x) sin(pi y) sin(pi z) decays spectrally in N
  (values recorded in tests/golden/manufactured_bp5.json by
  tests/golden/make_golden.py, which calls only the oracle);
* sampled rows equal the rows of the assembled operator;
* adjoint gradient: the nodal form equals the dense definition -lambda^T A_{e,Q} u,
  and it matches central finite differences of J.
"""
import json
import os

import numpy as np
import pytest

from oracle.adjoint import forward_adjoint, gradient, objective
from oracle.element import point_stiffness
from oracle.pcg import pcg
from oracle.problems import BakeoffProblem
from oracle.sampled import sampled_rows
from synth import fourier_field, fourier_modes, uniform_pm1


@pytest.mark.parametrize("bp,N", [(1, 2), (2, 2), (3, 2), (4, 2), (5, 3), (6, 2)])
def test_pcg_matches_direct_solve(bp, N):
    prob = BakeoffProblem(bp, 2, 2, 2, N, amp=0.05)
    r = uniform_pm1(0, np.arange(prob.n_global * prob.ncomp)).reshape(prob.n_global, -1)
    if prob.ncomp == 1:
        r = r[:, 0]
    b = prob.rhs(r)
    x, infos = prob.solve(b, tol=1e-12)
    Af = prob.A_free.toarray()
    b2 = b.reshape(prob.n_global, -1)
    x2 = x.reshape(prob.n_global, -1)
    for c in range(b2.shape[1]):
        xd = np.linalg.solve(Af, b2[prob.free, c])
        assert infos[c]["converged"]
        assert np.linalg.norm(x2[prob.free, c] - xd) <= 1e-9 * np.linalg.norm(xd)
        assert np.all(x2[~prob.free, c] == 0)


@pytest.mark.parametrize("vec,scalar", [(2, 1), (4, 3), (6, 5)])
def test_vector_problems_are_three_scalar_copies(vec, scalar):
    """Table 1: BP2/BP4/BP6 apply the operator of BP1/BP3/BP5 to each of three
    components; the vector oracle agrees with three independent scalar applies."""
    pv = BakeoffProblem(vec, 2, 1, 2, 3, amp=0.05)
    ps = BakeoffProblem(scalar, 2, 1, 2, 3, amp=0.05)
    u = uniform_pm1(4, np.arange(pv.n_global * 3)).reshape(pv.n_global, 3)
    wv = pv.apply(u)
    for c in range(3):
        np.testing.assert_array_equal(wv[:, c], ps.apply(u[:, c]))


def test_fixed_iterations_and_breakdown():
    prob = BakeoffProblem(5, 2, 1, 1, 3, amp=0.05)
    b = prob.rhs(uniform_pm1(1, np.arange(prob.n_global)))
    _, infos = prob.solve(b, fixed_iters=7)
    assert infos[0]["iters"] == 7 and len(infos[0]["history"]) == 8
    indefinite = -np.eye(4)
    with pytest.raises(FloatingPointError):
        pcg(indefinite, np.ones(4), np.ones(4), tol=1e-12)


def test_manufactured_convergence(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "manufactured_bp5.json")))
    errs = []
    for N in gold["orders"]:
        prob = BakeoffProblem(5, *gold["dims"], N, amp=gold["amp"])
        b, u_exact = prob.manufactured_rhs()
        x, infos = prob.solve(b, tol=gold["tol"])
        errs.append(float(np.max(np.abs(x - u_exact))))
        assert infos[0]["converged"]
    assert all(errs[i] > errs[i + 1] for i in range(len(errs) - 1)), errs
    np.testing.assert_allclose(errs, gold["max_nodal_error"], rtol=1e-6)


@pytest.mark.parametrize("bp,op", [(5, "A"), (3, "A"), (1, "A"), (5, "B"), (6, "A"), (2, "A"), (4, "A")])
def test_sampled_rows_equal_assembled_rows(bp, op):
    dims, N = (3, 2, 2), 3
    prob = BakeoffProblem(bp, *dims, N, amp=0.05)
    u = uniform_pm1(7, np.arange(prob.n_global * prob.ncomp)).reshape(prob.n_global, -1)
    if prob.ncomp == 1:
        u = u[:, 0]
    full = prob.apply(u) if op == "A" else prob.mass(u)
    nodes = np.array([0, 5, 17, 40, prob.n_global // 2, prob.n_global - 1])
    rows = sampled_rows(bp, *dims, N, 0.05, lambda ids: u[ids], nodes, operator=op)
    np.testing.assert_allclose(rows, full[nodes], rtol=0, atol=1e-13 * np.max(np.abs(full)))


def _adjoint_problem(N=2, dims=(2, 2, 2)):
    base = BakeoffProblem(5, *dims, N, amp=0.05)
    Xq = base.quadrature_points()
    kappa = np.exp(fourier_field(fourier_modes(0), Xq))
    kappa_star = np.exp(fourier_field(fourier_modes(1), Xq))
    prob = BakeoffProblem(5, *dims, N, amp=0.05, kappa=kappa)
    prob_star = BakeoffProblem(5, *dims, N, amp=0.05, kappa=kappa_star)
    b = prob.rhs(uniform_pm1(0, np.arange(prob.n_global)))
    u_star, _ = prob_star.solve(b, tol=1e-14)
    return prob, kappa, b, u_star, dims, N


def test_adjoint_gradient_equals_dense_definition():
    prob, kappa, b, u_star, dims, N = _adjoint_problem()
    u, lam, J, _ = forward_adjoint(prob, b, u_star)
    g = gradient(prob, u, lam)
    for e in (0, 3, 7):
        for Q in (0, 5, 13, 26):
            AQ = point_stiffness(prob.coords[e], N, prob.rule, Q)
            ref = -lam[prob.l2g[e]] @ AQ @ u[prob.l2g[e]]
            assert abs(g[e, Q] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_adjoint_gradient_matches_finite_differences():
    prob, kappa, b, u_star, dims, N = _adjoint_problem()
    u, lam, J, _ = forward_adjoint(prob, b, u_star)
    g = gradient(prob, u, lam)
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(3):
        d = rng.uniform(-1, 1, size=kappa.shape)
        d /= np.max(np.abs(d))
        Jp = objective(*_solve_at(kappa + h * d, b, u_star, dims, N))
        Jm = objective(*_solve_at(kappa - h * d, b, u_star, dims, N))
        fd = (Jp - Jm) / (2 * h)
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def _solve_at(kappa, b, u_star, dims, N):
    p = BakeoffProblem(5, *dims, N, amp=0.05, kappa=kappa)
    u, _ = p.solve(b, tol=1e-15, maxit=5000)
    return p, u, u_star


@pytest.mark.parametrize("bp", [3, 5, 6])
def test_helmholtz_constant_mode_and_manufactured_solution(bp):
    """H = A + beta B (Eq. (17)): A 1 = 0 on the unmasked matrix, so 1^T H 1 = beta |Omega| = beta;
    and for u = sin(pi x) sin(pi y) sin(pi z), -Lap u + beta u = (3 pi^2 + beta) u, so the discrete
    solution with that forcing approaches u (a dropped or mis-scaled beta term misses it by ~beta / 3 pi^2)."""
    beta = 7.5
    prob = BakeoffProblem(bp, 2, 2, 2, 5, amp=0.05, beta=beta)
    one = np.ones(prob.n_global)
    assert abs(one @ (prob.A @ one) - beta) < 1e-11
    X = prob.node_coords()
    s = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    f = (3 * np.pi ** 2 + beta) * s
    if prob.ncomp == 3:
        f = np.repeat(f[:, None], 3, axis=1)
        s = np.repeat(s[:, None], 3, axis=1)
    x, infos = prob.solve(prob.rhs(f), tol=1e-12)
    assert all(i["converged"] for i in infos)
    assert np.max(np.abs(x - s)) < 2e-3
    with pytest.raises(ValueError):
        BakeoffProblem(1, 1, 1, 1, 2, beta=1.0)


@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_threaded_pcg_follows_the_textbook_pcg(nthreads):
    """The multi-threaded C PCG of the CPU baseline takes the same iterates as oracle.pcg (to
    rounding: only the order of the inner-product sums differs), for any thread count, and a
    fixed thread count gives identical bits on repeated runs."""
    from oracle.cpu_pcg import pcg_threads
    prob = BakeoffProblem(5, 3, 2, 2, 4, amp=0.05)
    b = prob.rhs(uniform_pm1(0, np.arange(prob.n_global)))[prob.free]
    x_ref, info = pcg(prob.A_free, b, prob.diag_free, fixed_iters=25)
    x, hist = pcg_threads(prob.A_free, b, prob.diag_free, 25, nthreads)
    np.testing.assert_allclose(hist, info["history"], rtol=1e-9)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-11 * np.max(np.abs(x_ref)))
    x2, hist2 = pcg_threads(prob.A_free, b, prob.diag_free, 25, nthreads)
    assert np.array_equal(x, x2) and np.array_equal(hist, hist2)
