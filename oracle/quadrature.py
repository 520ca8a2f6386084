"""Quadrature rules (the paper leaves them unspecified; reading R11).

Collapsed (Stroud conical product) rules built from Gauss-Jacobi rules, which
scipy supplies.  With n points per direction a tet / triangle rule integrates
every polynomial of total degree <= 2n-1 exactly.
"""
import math

import numpy as np
from scipy.special import roots_jacobi


def gauss_jacobi01(n: int, alpha: float):
    """n-point rule on [0,1] for the weight (1-x)^alpha."""
    x, w = roots_jacobi(n, alpha, 0.0)
    return (x + 1.0) / 2.0, w / 2.0 ** (alpha + 1.0)


def line_rule(n: int):
    """Gauss-Legendre on [0,1]; weights sum to 1."""
    return gauss_jacobi01(n, 0.0)


def tri_rule(n: int):
    """Reference triangle {xi, eta >= 0, xi + eta <= 1}; points (m, 2), weights sum to 1/2."""
    u, wu = gauss_jacobi01(n, 0.0)
    v, wv = gauss_jacobi01(n, 1.0)
    U, V = np.meshgrid(u, v, indexing="ij")
    W = np.outer(wu, wv)
    pts = np.stack([U * (1 - V), V], axis=-1).reshape(-1, 2)
    return pts, W.ravel()


def tet_rule(n: int):
    """Reference tetrahedron {xi, eta, zeta >= 0, sum <= 1}; points (m, 3), weights sum to 1/6."""
    u, wu = gauss_jacobi01(n, 0.0)
    v, wv = gauss_jacobi01(n, 1.0)
    w, ww = gauss_jacobi01(n, 2.0)
    U, V, Wc = np.meshgrid(u, v, w, indexing="ij")
    pts = np.stack([U * (1 - V) * (1 - Wc), V * (1 - Wc), Wc], axis=-1).reshape(-1, 3)
    wts = (wu[:, None, None] * wv[None, :, None] * ww[None, None, :]).ravel()
    return pts, wts


def n_linear(p: int) -> int:
    """Points per direction for products of two degree-p polynomials (degree 2p)."""
    return p + 1


def n_nonlinear(p: int) -> int:
    """Points per direction for cubic-in-solution integrands and non-polynomial data."""
    return int(math.ceil((3 * p + 2) / 2.0))
