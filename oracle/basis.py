"""Basis functions (Sec. 2.3).

* Tetrahedron: orthonormal Dubiner basis on T_ref = {xi,eta,zeta >= 0, xi+eta+zeta <= 1}
  (same span P_p as the paper's nodal basis of Eq. bf_1; reading R7), built here exactly
  with sympy and evaluated through its expanded monomial form.
* Dual cells: the scaled Taylor monomials of Eq. bf_2 (orthonormalised per cell elsewhere).
* Time: orthonormal Legendre polynomials on [0,1] (same span as the paper's Lagrange
  basis through Gauss-Legendre points; reading R8).

Multi-index order (shared convention, also used for the Taylor exponents):
for n = 0..p, for i = 0..n, for j = 0..n-i: (i, j, n-i-j).
Dubiner function (i,j,k), with u = xi/(1-eta-zeta), v = eta/(1-zeta), w = zeta:
  c * P_i(2u-1) (1-v)^i P_j^(2i+1,0)(2v-1) (1-w)^(i+j) P_k^(2i+2j+2,0)(2w-1),
  c = sqrt((2i+1)(2i+2j+2)(2i+2j+2k+3)).
"""
from functools import lru_cache

import numpy as np
import sympy as sp
from numpy.polynomial import legendre as npleg


def multi_indices(p: int):
    out = []
    for n in range(p + 1):
        for i in range(n + 1):
            for j in range(n - i + 1):
                out.append((i, j, n - i - j))
    return out


def nbasis(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


@lru_cache(maxsize=None)
def _dubiner_monomials(p: int):
    """Exact expansion of each Dubiner function in monomials xi^a eta^b zeta^c.

    Returns (coef[N, M] float64, exps[M, 3] int) with M = N monomials of degree <= p."""
    xi, eta, zeta = sp.symbols("xi eta zeta")
    s = 1 - eta - zeta
    t = 1 - zeta
    mons = multi_indices(p)
    col = {m: c for c, m in enumerate(mons)}
    coef = np.zeros((len(mons), len(mons)))
    for r, (i, j, k) in enumerate(mons):
        # s^i P_i(2 xi/s - 1) and t^j P_j^(2i+1,0)(2 eta/t - 1) are polynomials
        f1 = sp.expand(sp.cancel(s ** i * sp.jacobi(i, 0, 0, 2 * xi / s - 1)))
        f2 = sp.expand(sp.cancel(t ** j * sp.jacobi(j, 2 * i + 1, 0, 2 * eta / t - 1)))
        f3 = sp.jacobi(k, 2 * i + 2 * j + 2, 0, 2 * zeta - 1)
        c = sp.sqrt((2 * i + 1) * (2 * i + 2 * j + 2) * (2 * i + 2 * j + 2 * k + 3))
        poly = sp.Poly(sp.expand(c * f1 * f2 * f3), xi, eta, zeta)
        for (a, b, cc), val in poly.terms():
            # monomial xi^a eta^b zeta^cc stored under multi-index (a, b, cc)
            coef[r, col[(a, b, cc)]] = float(val)
    return coef, np.array(mons, dtype=np.int64)


def _monomials(x, exps):
    """x (m,3) -> values (m, M) and gradients (m, M, 3) of x^exps."""
    x = np.asarray(x, dtype=np.float64)
    m = x.shape[0]
    pmax = int(exps.max()) if exps.size else 0
    powv = np.ones((m, 3, pmax + 2))
    for e in range(1, pmax + 2):
        powv[:, :, e] = powv[:, :, e - 1] * x
    vals = np.ones((m, len(exps)))
    grads = np.zeros((m, len(exps), 3))
    for c, (a, b, d) in enumerate(exps):
        ea = (a, b, d)
        vals[:, c] = powv[:, 0, a] * powv[:, 1, b] * powv[:, 2, d]
        for dim in range(3):
            if ea[dim] == 0:
                continue
            g = float(ea[dim])
            for o in range(3):
                g = g * powv[:, o, ea[o] - (1 if o == dim else 0)]
            grads[:, c, dim] = g
    return vals, grads


def dubiner(p: int, xi):
    """Values (m, N) and reference gradients (m, N, 3) of the Dubiner basis at xi (m, 3)."""
    coef, exps = _dubiner_monomials(p)
    mv, mg = _monomials(xi, exps)
    return mv @ coef.T, np.einsum("qmd,nm->qnd", mg, coef)


def taylor(p: int, x, x0, h):
    """Scaled Taylor monomials of Eq. bf_2 at physical points x (m,3): values (m, N)."""
    y = (np.asarray(x, dtype=np.float64) - np.asarray(x0)) / h
    vals, _ = _monomials(y, np.array(multi_indices(p), dtype=np.int64))
    return vals


def legendre01(pt: int, tau):
    """gamma_a(tau) = sqrt(2a+1) P_a(2 tau - 1) and d/dtau, shapes (m, pt+1)."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    vals = np.zeros((tau.size, pt + 1))
    ders = np.zeros((tau.size, pt + 1))
    for a in range(pt + 1):
        c = np.zeros(a + 1); c[a] = 1.0
        s = np.sqrt(2 * a + 1)
        vals[:, a] = s * npleg.legval(2 * tau - 1, c)
        ders[:, a] = 2 * s * npleg.legval(2 * tau - 1, npleg.legder(c))
    return vals, ders
