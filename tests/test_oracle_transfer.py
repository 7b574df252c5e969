"""Pins for the oracle's grid transfers (CPU only)."""
import numpy as np
import pytest

from oracle.fem import Discretisation, Problem
from oracle.transfer import injection, interpolation_1d, prolongation


def nodal(d, fx, fy, fp):
    """Global vector with the nodal values of the spatial fields at every temporal DoF."""
    xv, xp = d.node_coords()
    X, Y = np.meshgrid(xv, xv, indexing="xy")
    XP, YP = np.meshgrid(xp, xp, indexing="xy")
    blk = np.concatenate([fx(X, Y).ravel(), fy(X, Y).ravel(), fp(XP, YP).ravel()])
    return np.tile(blk, d.N * d.nt)


@pytest.mark.parametrize("k", [1, 2])
def test_prolongation_reproduces_coarse_polynomials(k):
    """P maps the coarse interpolant of any Q_{k+1} (velocity, vanishing on the
    boundary) / Q_k (pressure) polynomial to its fine interpolant."""
    pb = Problem()
    c = Discretisation(2, k, 1, 2, pb)
    f = Discretisation(4, k, 1, 2, pb)
    P = prolongation(f, c)
    bub = lambda X, Y: X * (1 - X) * Y * (1 - Y)
    fx = lambda X, Y: bub(X, Y) * (0.3 + X ** (k - 1) - 2 * Y ** (k - 1))
    fy = lambda X, Y: bub(X, Y) * (1.1 - X ** (k - 1) * Y ** (k - 1))
    fp = lambda X, Y: 0.7 - X ** k + 3 * (X * Y) ** k
    assert np.abs(P @ nodal(c, fx, fy, fp) - nodal(f, fx, fy, fp)).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_1d_interpolation_partition_of_unity_and_nestedness(p):
    P = interpolation_1d(3, p)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(P[::2], np.eye(3 * p + 1), atol=1e-15)   # coarse nodes are fine nodes


def test_restriction_is_adjoint_and_zero_on_dirichlet():
    pb = Problem()
    c = Discretisation(2, 2, 0, 3, pb)
    f = Discretisation(4, 2, 0, 3, pb)
    P = prolongation(f, c)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(f.ndofs), rng.standard_normal(c.ndofs)
    assert abs(np.dot(P.T @ x, y) - np.dot(x, P @ y)) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(y)
    assert np.all((P.T @ x)[c.dirichlet_mask()] == 0.0)
    assert np.all((P @ y)[f.dirichlet_mask()] == 0.0)


def test_injection_is_left_inverse_of_interpolation():
    pb = Problem()
    c = Discretisation(2, 1, 1, 2, pb)
    f = Discretisation(4, 1, 1, 2, pb)
    fx = lambda X, Y: np.sin(3 * X) * Y
    fy = lambda X, Y: np.cos(X + Y)
    fp = lambda X, Y: X - Y ** 2
    assert np.abs(injection(f, c, nodal(f, fx, fy, fp)) - nodal(c, fx, fy, fp)).max() < 1e-15
