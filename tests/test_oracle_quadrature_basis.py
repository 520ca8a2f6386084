"""Pins for the oracle's quadrature rules and bases against closed forms."""
import math

import numpy as np
import pytest

from oracle.basis import dubiner, legendre01, multi_indices, nbasis, taylor
from oracle.quadrature import line_rule, tet_rule, tri_rule


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_tet_rule_exact_monomials(n):
    x, w = tet_rule(n)
    for (a, b, c) in multi_indices(2 * n - 1):
        exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
        got = (w * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c).sum()
        assert abs(got - exact) <= 1e-15 + 1e-13 * exact


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_tri_and_line_rules_exact(n):
    x, w = tri_rule(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * x[:, 0] ** a * x[:, 1] ** b).sum() - exact) <= 1e-15 + 1e-13 * exact
    t, wt = line_rule(n)
    for a in range(2 * n):
        assert abs((wt * t ** a).sum() - 1.0 / (a + 1)) < 1e-14


def test_tet_rule_not_exact_beyond_degree():
    # a dropped point / wrong Jacobi weight would show up here or above
    x, w = tet_rule(2)
    got = (w * x[:, 2] ** 4).sum()
    assert abs(got - math.factorial(4) / math.factorial(7)) > 1e-8


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_dubiner_orthonormal(p):
    x, w = tet_rule(p + 2)
    v, _ = dubiner(p, x)
    G = (v * w[:, None]).T @ v
    assert np.abs(G - np.eye(nbasis(p))).max() < 5e-13
    assert abs(v[0, 0] - math.sqrt(6.0)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dubiner_spans_Pp_and_gradients(p):
    """L2 projection of a random degree-p polynomial reproduces it; gradients match the
    analytic derivative of that polynomial."""
    rng = np.random.default_rng(p)
    mons = multi_indices(p)
    cf = rng.standard_normal(len(mons))

    def poly(x):
        return sum(c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** d for c, (a, b, d) in zip(cf, mons))

    def grad(x):
        g = np.zeros_like(x)
        for c, (a, b, d) in zip(cf, mons):
            if a: g[:, 0] += c * a * x[:, 0] ** (a - 1) * x[:, 1] ** b * x[:, 2] ** d
            if b: g[:, 1] += c * b * x[:, 0] ** a * x[:, 1] ** (b - 1) * x[:, 2] ** d
            if d: g[:, 2] += c * d * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** (d - 1)
        return g

    xq, wq = tet_rule(p + 1)
    vq, _ = dubiner(p, xq)
    coef = (vq * wq[:, None]).T @ poly(xq)
    xs = rng.random((40, 3)) / 3.0
    vs, gs = dubiner(p, xs)
    assert np.abs(vs @ coef - poly(xs)).max() < 1e-11 * max(1.0, np.abs(poly(xs)).max())
    assert np.abs(np.einsum("qnd,n->qd", gs, coef) - grad(xs)).max() < 1e-10 * max(1.0, np.abs(grad(xs)).max())


@pytest.mark.parametrize("pt", [0, 1, 2, 3, 4])
def test_legendre_time_basis(pt):
    t, w = line_rule(pt + 2)
    g, dg = legendre01(pt, t)
    assert np.abs((g * w[:, None]).T @ g - np.eye(pt + 1)).max() < 1e-13
    g1, _ = legendre01(pt, 1.0)
    g0, _ = legendre01(pt, 0.0)
    for a in range(pt + 1):
        assert abs(g1[0, a] - math.sqrt(2 * a + 1)) < 1e-13
        assert abs(g0[0, a] - (-1) ** a * math.sqrt(2 * a + 1)) < 1e-13
    # derivative against a centred difference
    h = 1e-6
    gp, _ = legendre01(pt, t + h)
    gm, _ = legendre01(pt, t - h)
    assert np.abs((gp - gm) / (2 * h) - dg).max() < 1e-6


def test_taylor_monomials():
    x = np.array([[0.3, 0.2, 0.1]])
    v = taylor(2, x, np.array([0.1, 0.1, 0.1]), 0.5)
    # order (0,0,0), (0,0,1), (0,1,0), (1,0,0), (0,0,2), (0,1,1), (0,2,0), (1,0,1), (1,1,0), (2,0,0)
    y = (x[0] - 0.1) / 0.5
    want = [1, y[2], y[1], y[0], y[2] ** 2, y[1] * y[2], y[1] ** 2, y[0] * y[2], y[0] * y[1], y[0] ** 2]
    assert np.allclose(v[0], want, atol=1e-15)
