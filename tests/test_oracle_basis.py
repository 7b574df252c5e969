"""Pins for the oracle's 1D and temporal building blocks (CPU only)."""
from math import factorial

import numpy as np
import pytest

from oracle.basis import TimeMatrices, equispaced_nodes, gauss_legendre, lagrange, radau_right_nodes


def test_radau_nodes_match_textbook_abscissae():
    # Radau IIA abscissae (Hairer & Wanner, Solving ODEs II, Table IV.5.5/5.6)
    assert np.allclose(radau_right_nodes(0), [1.0], atol=1e-15)
    assert np.allclose(radau_right_nodes(1), [1.0 / 3.0, 1.0], atol=1e-15)
    s6 = np.sqrt(6.0)
    assert np.allclose(radau_right_nodes(2), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-14)


def test_radau_nodes_integrate_to_degree_2q():
    """The (q+1)-point right-Radau rule (weights from the Lagrange basis) integrates
    polynomials of degree 2q exactly on [0, 1] and no higher (Hairer & Wanner, Sec. IV.5)."""
    for q in range(4):
        nodes = radau_right_nodes(q)
        xs, ws = gauss_legendre(q + 2)
        V, _ = lagrange(nodes, xs)
        w = V @ ws                      # int of each Lagrange basis function
        for d in range(2 * q + 1):
            assert abs(w @ nodes ** d - 1.0 / (d + 1)) < 1e-13, (q, d)
        assert abs(w @ nodes ** (2 * q + 1) - 1.0 / (2 * q + 2)) > 1e-6, q


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_reproduces_polynomials_and_derivatives(p):
    rng = np.random.default_rng(p)
    coef = rng.standard_normal(p + 1)
    f = np.polynomial.Polynomial(coef)
    nodes = equispaced_nodes(p)
    x = np.linspace(-0.2, 1.3, 17)
    V, D = lagrange(nodes, x)
    assert np.allclose(f(nodes) @ V, f(x), atol=1e-12)
    assert np.allclose(f(nodes) @ D, f.deriv()(x), atol=1e-11)


@pytest.mark.parametrize("nq", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exact_to_degree_2nq_minus_1(nq):
    x, w = gauss_legendre(nq)
    for d in range(2 * nq):
        assert abs(np.dot(w, x ** d) - 1.0 / (d + 1)) < 1e-14
    d = 2 * nq
    assert abs(np.dot(w, x ** d) - 1.0 / (d + 1)) > 1e-8


def pade_stability(j, k, z):
    """(j, k) Pade approximant of exp(z) (closed form)."""
    num = sum(factorial(j + k - i) * factorial(j) / (factorial(j + k) * factorial(i) * factorial(j - i)) * z ** i
              for i in range(j + 1))
    den = sum(factorial(j + k - i) * factorial(k) / (factorial(j + k) * factorial(i) * factorial(k - i)) * (-z) ** i
              for i in range(k + 1))
    return num / den


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_dg_in_time_end_value_is_radau_iia_stability_function(q):
    """For y' = lam y the DG(q) slab system (Eq. dgintime) reads
    (Kt - z Wt) U = tau(0) y0 with z = lam dt; its end value U_q must be the
    (q, q+1) Pade approximant of e^z, the Radau IIA stability function
    (DG(q) in time coincides with Radau IIA for linear problems)."""
    tm = TimeMatrices(q)
    for z in [-0.3, -2.0, -25.0, 0.4, -1.0 + 0.5j]:
        U = np.linalg.solve(tm.Kt - z * tm.Wt, tm.tau0.astype(complex))
        assert abs(U[-1] - pade_stability(q, q + 1, z)) < 1e-12 * max(1.0, abs(U[-1]))


def test_dg1_time_matrices_closed_form():
    """q = 1, nodes {1/3, 1}: tau_0 = 3(1-s)/2, tau_1 = (3s-1)/2, integrated by hand."""
    tm = TimeMatrices(1)
    assert np.allclose(tm.Kt, [[1.125, 0.375], [-1.125, 0.625]], atol=1e-14)
    assert np.allclose(tm.Wt, np.diag([0.75, 0.25]), atol=1e-14)
    assert np.allclose(tm.tau0, [1.5, -0.5], atol=1e-14)
    # sum_{b,c} T3[a,b,c] s_b s_c = int tau_a(s) s^2 ds for U(s) = s
    s = tm.nodes
    assert np.allclose(np.einsum("abc,b,c->a", tm.T3, s, s), [0.125, 5.0 / 24.0], atol=1e-14)
    assert abs(tm.T3.sum() - 1.0) < 1e-14
