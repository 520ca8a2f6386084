"""The closed-form data are exact incompressible Navier-Stokes solutions (checked symbolically)."""
import numpy as np
import pytest

from inputs import BeltramiParams, SolenoidalModes, beltrami_pressure, beltrami_velocity


def test_beltrami_is_exact_navier_stokes():
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t")
    a, d, nu = sp.Rational(7, 10), sp.Rational(13, 10), sp.Rational(3, 10)
    f = sp.exp(-nu * d * d * t)
    u = -a * (sp.exp(a * x) * sp.sin(a * y + d * z) + sp.exp(a * z) * sp.cos(a * x + d * y)) * f
    v = -a * (sp.exp(a * y) * sp.sin(a * z + d * x) + sp.exp(a * x) * sp.cos(a * y + d * z)) * f
    w = -a * (sp.exp(a * z) * sp.sin(a * x + d * y) + sp.exp(a * y) * sp.cos(a * z + d * x)) * f
    V, X = [u, v, w], [x, y, z]
    p = -(u * u + v * v + w * w) / 2
    assert sp.simplify(sum(sp.diff(V[i], X[i]) for i in range(3))) == 0
    prm = BeltramiParams(a=0.7, d=1.3, nu=0.3)
    rng = np.random.default_rng(0)
    for _ in range(3):
        pt = rng.random(4)
        sub = {x: pt[0], y: pt[1], z: pt[2], t: pt[3]}
        for i in range(3):
            r = (sp.diff(V[i], t) + sum(V[j] * sp.diff(V[i], X[j]) for j in range(3)) + sp.diff(p, X[i])
                 - nu * sum(sp.diff(V[i], X[j], 2) for j in range(3)))
            assert abs(float(r.subs(sub))) < 1e-12
        xx = pt[None, :3]
        num = beltrami_velocity(xx, pt[3], prm)[0]
        assert np.allclose(num, [float(c.subs(sub)) for c in V], atol=1e-14)
        assert abs(beltrami_pressure(xx, pt[3], prm)[0] - float(p.subs(sub))) < 1e-13


def test_solenoidal_modes_divergence_free_and_no_slip():
    f = SolenoidalModes(seed=1)
    rng = np.random.default_rng(1)
    x = rng.random((20, 3))
    h = 1e-5
    div = sum((f(x + h * np.eye(3)[c]) - f(x - h * np.eye(3)[c]))[:, c] for c in range(3)) / (2 * h)
    assert np.abs(div).max() < 1e-7
    wall = rng.random((10, 3)); wall[:, 1] = 0.0
    assert np.abs(f(wall)).max() < 1e-14
    g = np.linspace(0, 1, 33)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    assert abs(np.linalg.norm(f(P), axis=1).max() - 0.1) < 1e-12


def test_abc_is_exact_navier_stokes():
    """Eq. CT_1 (the paper's convergence test): divergence-free, and with the stated pressure the
    momentum residual of the incompressible Navier-Stokes equations vanishes for any nu."""
    sp = pytest.importorskip("sympy")
    from inputs import abc_pressure, abc_velocity
    x, y, z, t, nu = sp.symbols("x y z t nu")
    f = sp.exp(-nu * t)
    V = [(sp.sin(z) + sp.cos(y)) * f, (sp.sin(x) + sp.cos(z)) * f, (sp.sin(y) + sp.cos(x)) * f]
    p = -(sp.cos(x) * sp.sin(y) + sp.sin(x) * sp.cos(z) + sp.sin(z) * sp.cos(y)) * sp.exp(-2 * nu * t)
    X = [x, y, z]
    assert sp.simplify(sum(sp.diff(V[i], X[i]) for i in range(3))) == 0
    for i in range(3):
        r = (sp.diff(V[i], t) + sum(V[j] * sp.diff(V[i], X[j]) for j in range(3)) + sp.diff(p, X[i])
             - nu * sum(sp.diff(V[i], X[j], 2) for j in range(3)))
        assert sp.simplify(sp.expand_trig(r)) == 0
    pt = np.array([0.3, -1.1, 2.0]); tt, nuv = 0.7, 0.4
    sub = {x: pt[0], y: pt[1], z: pt[2], t: tt, nu: nuv}
    assert np.allclose(abc_velocity(pt[None], tt, nuv)[0], [float(c.subs(sub)) for c in V], atol=1e-14)
    assert abs(abc_pressure(pt[None], tt, nuv)[0] - float(p.subs(sub))) < 1e-14


def test_periodic_kuhn_mesh():
    """Lattice vertices of the periodic box, positively oriented tetrahedra of volume h^3 / 6 once
    unwrapped, and every face shared by exactly two tetrahedra."""
    from inputs import kuhn_periodic_mesh
    n = 3
    v, t, per = kuhn_periodic_mesh(n)
    assert v.shape == (n ** 3, 3) and t.shape == (6 * n ** 3, 4) and np.allclose(per, 2 * np.pi)
    P = v[t]
    P = P[:, :1] + (P - P[:, :1]) - per * np.round((P - P[:, :1]) / per)
    vol = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], -1)) / 6
    assert np.allclose(vol, (2 * np.pi / n) ** 3 / 6)
    faces = {}
    for i, tt in enumerate(t):
        for f in range(4):
            faces.setdefault(tuple(sorted(np.delete(tt, f))), []).append(i)
    assert all(len(l) == 2 for l in faces.values()) and len(faces) == 2 * len(t)
