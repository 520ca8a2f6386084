"""Pins for the learned-preconditioner oracle: analytic backward pass vs central finite
differences in FP64, and the adjoint relation between neighbour gather and scatter."""
import numpy as np
import pytest

from oracle import gnn


def _graph(ne=30, seed=0):
    rng = np.random.default_rng(seed)
    nbr = rng.integers(-1, ne, size=(ne, 4))
    return nbr


def test_gather_scatter_adjoint():
    rng = np.random.default_rng(1)
    nbr = _graph()
    h = rng.standard_normal((30, 5)); g = rng.standard_normal((30, 5))
    assert abs(np.sum(g * gnn.gather_sum(h, nbr)) - np.sum(h * gnn.scatter_sum(g, nbr, 30))) < 1e-12


@pytest.mark.parametrize("L", [1, 3])
def test_backward_matches_finite_differences(L):
    rng = np.random.default_rng(2)
    ne, C, G = 30, 6, 2
    nbr = _graph(ne)
    p = gnn.init_params(C + G, C, H=8, L=L, seed=3)
    for k in p:                                   # non-zero biases exercise every term
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    geom = rng.random((ne, G))
    pairs = [(rng.standard_normal((ne, C)), rng.standard_normal((ne, C))) for _ in range(2)]
    loss, g = gnn.loss_and_grad(p, pairs, geom, nbr)
    h = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h; lp, _ = gnn.loss_and_grad(p, pairs, geom, nbr)
            flat[idx] = old - h; lm, _ = gnn.loss_and_grad(p, pairs, geom, nbr)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_scale_equivariance():
    """M(c r) = c M(r): the network sees r / RMS(r) and rescales its output."""
    rng = np.random.default_rng(4)
    ne, C, G = 20, 4, 2
    nbr = _graph(ne, 5)
    p = gnn.init_params(C + G, C, H=8, L=2, seed=6)
    r = rng.standard_normal((ne, C)); geom = rng.random((ne, G))
    a = gnn.apply(p, r, geom, nbr)
    b = gnn.apply(p, 7.5 * r, geom, nbr)
    assert np.abs(b - 7.5 * a).max() < 1e-12 * np.abs(b).max()
