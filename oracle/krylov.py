"""Krylov solvers: CG (for symmetric positive definite systems; Sec. 2.7, Cor. 1-2) and
restarted GMRES with modified Gram-Schmidt and Givens rotations (the paper's
unpreconditioned matrix-free GMRES).  Initial guess x0, stop on ||b - A x|| <= tol ||b||
in the Euclidean norm of the coefficient vector (reading R16)."""
import numpy as np


def cg(apply, b, x0, tol, maxit=100000):
    x = np.array(x0, dtype=np.float64, copy=True).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply(x)
    p = r.copy()
    rr = r @ r
    it = 0
    while np.sqrt(rr) > tol * bn and it < maxit:
        Ap = apply(p)
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / bn


def gmres(apply, b, x0, tol, restart=50, maxit=100000):
    x = np.array(x0, dtype=np.float64, copy=True).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn or it >= maxit:
            return x, it, beta / bn
        V = np.zeros((restart + 1, b.size))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart); sn = np.zeros(restart)
        g = np.zeros(restart + 1); g[0] = beta
        V[0] = r / beta
        k = 0
        for k in range(restart):
            w = apply(V[k])
            for i in range(k + 1):                       # modified Gram-Schmidt
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                           # apply previous rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            if abs(g[k + 1]) <= tol * bn or it >= maxit:
                break
        kk = k + 1
        y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
        x += V[:kk].T @ y
