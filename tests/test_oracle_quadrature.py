"""Pins of the oracle's 1D rules and Lagrange basis (CPU only).

Closed forms (tests/golden/quadrature_closed_forms.json), the library routines
numpy.polynomial.legendre.leggauss / Legendre.deriv().roots(), exactness on
monomials, and the GLL/GL symmetry that the even-odd decomposition of
Eq. (37) relies on.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.basis import lagrange_derivatives, lagrange_values
from oracle.quadrature import bp_rule, gauss, gll

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _ev(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def test_closed_forms(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "quadrature_closed_forms.json")))
    for N, v in gold["gll"].items():
        x, w = gll(int(N))
        np.testing.assert_allclose(x, [_ev(s) for s in v["nodes"]], rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, [_ev(s) for s in v["weights"]], rtol=1e-14)
    for q, v in gold["gauss"].items():
        x, w = gauss(int(q))
        np.testing.assert_allclose(x, [_ev(s) for s in v["nodes"]], rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, [_ev(s) for s in v["weights"]], rtol=1e-14)


@pytest.mark.parametrize("q", range(1, 21))
def test_gauss_matches_library(q):
    x, w = gauss(q)
    xl, wl = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(x, xl, rtol=0, atol=2e-15)
    # leggauss refines eigenvalue roots with one Newton step in double, so its
    # weights carry errors of a few 1e-14 at q > 15
    np.testing.assert_allclose(w, wl, rtol=2e-13, atol=0)


@pytest.mark.parametrize("N", range(2, 17))
def test_gll_interior_nodes_are_roots_of_legendre_derivative(N):
    x, _ = gll(N)
    roots = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    np.testing.assert_allclose(x[1:-1], roots, rtol=0, atol=1e-12)
    assert x[0] == -1.0 and x[-1] == 1.0
    np.testing.assert_array_equal(x, -x[::-1])


def _exact_moment(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("N", range(1, 17))
def test_gll_exactness_degree(N):
    x, w = gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):
        assert abs(w @ x ** k - _exact_moment(k)) < 1e-13, k
    # degree 2N is not integrated exactly: the rule has exactly degree 2N-1
    assert abs(w @ x ** (2 * N) - _exact_moment(2 * N)) > 1e-11


@pytest.mark.parametrize("q", range(1, 18))
def test_gauss_exactness_degree(q):
    x, w = gauss(q)
    for k in range(0, 2 * q):
        assert abs(w @ x ** k - _exact_moment(k)) < 1e-13, k
    assert abs(w @ x ** (2 * q) - _exact_moment(2 * q)) > 1e-11


def test_table1_rules(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "table1_bps.json")))
    for bp in (1, 3, 5, 6):
        row = gold["problems"][str(bp)]
        for N in (1, 3, 7):
            x, _ = bp_rule(bp, N)
            assert len(x) == N + row["q_minus_p"]
            ref = gll(N)[0] if row["quadrature"] == "GLL" else gauss(N + 2)[0]
            np.testing.assert_array_equal(x, ref)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 10, 15])
def test_lagrange_cardinal_and_partition(N):
    xi, _ = gll(N)
    L = lagrange_values(xi, xi)
    np.testing.assert_allclose(L, np.eye(N + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 37)
    np.testing.assert_allclose(lagrange_values(xi, xs).sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(lagrange_derivatives(xi, xs).sum(axis=1), 0.0, atol=1e-10)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9, 12, 15])
def test_lagrange_derivative_exact_on_polynomials(N):
    xi, _ = gll(N)
    rng = np.random.default_rng(N)
    xs = rng.uniform(-1, 1, 11)
    Dm = lagrange_derivatives(xi, xs)
    for k in range(0, N + 1):
        exact = k * xs ** (k - 1) if k > 0 else np.zeros_like(xs)
        np.testing.assert_allclose(Dm @ xi ** k, exact, atol=1e-11 * max(1, N * N))


def test_interpolation_symmetry_eq37():
    """Eq. (37): S_ji = phi_i(xi_j) at q = p+2 GL points for p = 3 has the
    centro-symmetric pattern phi_i(xi_j) = phi_{p+2-i}(xi_{q+1-j}) (1-based);
    the derivative matrix is centro-antisymmetric."""
    for p in (2, 3, 4, 7):
        q = p + 2
        xi, _ = gll(p)
        eta, _ = gauss(q)
        S = lagrange_values(xi, eta)
        Dm = lagrange_derivatives(xi, eta)
        assert S.shape == (q, p + 1)
        np.testing.assert_allclose(S, S[::-1, ::-1], atol=1e-14)
        np.testing.assert_allclose(Dm, -Dm[::-1, ::-1], atol=1e-12)
    # p = 3, q = 5: 10 distinct entries, middle row symmetric (s9, s10, s10, s9)
    S = lagrange_values(gll(3)[0], gauss(5)[0])
    np.testing.assert_allclose(S[2], S[2][::-1], atol=1e-15)
