"""Pins for the literal space-time blocks (Eqs. MD_2-MD_6, vis3, mj) and the pressure /
viscous operators (Eq. CS_19, A1_mod; Corollaries 1-4 of Sec. 2.7)."""
import numpy as np
import pytest
import scipy.linalg as sla

from inputs import kuhn_mesh
from oracle import operators as ops
from oracle.basis import multi_indices
from oracle.blocks import SpaceTimeDG, map_tet
from oracle.mesh import Mesh
from oracle.quadrature import tet_rule


def make(n, p, pt, dt=0.01, seed=0):
    v, t = kuhn_mesh(n, seed=seed)
    return SpaceTimeDG(Mesh(v, t), p, pt, dt)


def K_closed(pt):
    if pt == 0:
        return np.array([[1.0]])
    if pt == 1:
        s = np.sqrt(3.0)
        return np.array([[1.0, s], [-s, 3.0]])
    raise ValueError


@pytest.mark.parametrize("p,pt", [(1, 0), (2, 1), (3, 1)])
def test_K1_gradient_divergence_adjoint(p, pt):
    d = make(2, p, pt)
    for j in range(0, d.mesh.nf, 7):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            Q, D = fb["Q"][s], fb["D"][s]
            assert np.abs(Q + D.transpose(0, 2, 1)).max() <= 1e-14 * np.abs(Q).max()


@pytest.mark.parametrize("pt", [0, 1])
def test_time_structure_of_masses(pt):
    """M_j = I (x) K with K in closed form; Mbar_j = dt I; M_i = dt |J_i| I."""
    d = make(2, 2, pt, dt=0.02)
    K = K_closed(pt)
    N = d.N
    for j in range(0, d.mesh.nf, 11):
        fb = d.face_blocks(j)
        want = np.kron(K, np.eye(N))                      # index a*N + k
        assert np.abs(fb["M"] - want).max() < 1e-12
        assert np.abs(fb["Mbar"] - 0.02 * np.eye(d.Nst)).max() < 1e-14
    for i in range(0, d.mesh.ne, 5):
        assert np.abs(d.tet_blocks(i)["Mi"] - 0.02 * d.mesh.detJ[i] * np.eye(d.Nst)).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dual_basis_reproduces_polynomials(p):
    d = make(2, p, 0)
    rng = np.random.default_rng(1)
    mons = multi_indices(p)
    cf = rng.standard_normal(len(mons))
    f = lambda x: sum(c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** e for c, (a, b, e) in zip(cf, mons))
    for j in range(0, d.mesh.nf, 13):
        pts, coef = [], np.zeros(d.N)
        for _, V in d.mesh.dual_subtets(j):
            x, w = map_tet(V, *tet_rule(p + 2))
            coef += (d.psi(j, x) * w[:, None]).T @ f(x)
            pts.append(x)
        xs = np.vstack(pts)[::5]
        assert np.abs(d.psi(j, xs) @ coef - f(xs)).max() < 1e-11 * max(1, np.abs(f(xs)).max())


def _poly_field(p, rng):
    mons = multi_indices(p)
    cf = rng.standard_normal((3, len(mons)))

    def val(x, c):
        return sum(k * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** e for k, (a, b, e) in zip(cf[c], mons))

    def der(x, c, dim):
        out = np.zeros(len(x))
        for k, (a, b, e) in zip(cf[c], mons):
            ex = [a, b, e]
            if ex[dim] == 0:
                continue
            t = k * ex[dim]
            for o in range(3):
                t = t * x[:, o] ** (ex[o] - (1 if o == dim else 0))
            out += t
        return out
    return val, der


@pytest.mark.parametrize("p,pt", [(1, 0), (2, 1), (3, 0)])
def test_gradient_consistency(p, pt):
    """For a continuous q in P_p (no jump), Q_lj q_l + Q_rj q_r is the dual-basis moment of
    the gradient: dt * int_{H_j} psi_k d_c q at time mode 0, zero elsewhere."""
    d = make(2, p, pt, dt=0.05)
    val, der = _poly_field(p, np.random.default_rng(2))
    m = d.mesh
    P = np.zeros((m.ne, d.Nst))
    xq, wq = tet_rule(p + 1)
    for i in range(m.ne):
        x, w = map_tet(m.X[m.T[i]], xq, wq)
        ph, _ = d.phi(i, x)
        P[i, :d.N] = np.linalg.solve((ph * w[:, None]).T @ ph, (ph * w[:, None]).T @ val(x, 0))
    for j in np.nonzero(m.interior)[0][::9]:
        fb = d.face_blocks(j)
        l, r = fb["sides"]
        for c in range(3):
            got = fb["Q"][0][c] @ P[l] + fb["Q"][1][c] @ P[r]
            want = np.zeros(d.Nst)
            for _, V in m.dual_subtets(j):
                x, w = map_tet(V, *tet_rule(p + 1))
                want[:d.N] += 0.05 * (d.psi(j, x) * w[:, None]).T @ der(x, 0, c)
            assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("p,pt", [(1, 0), (2, 1), (3, 1)])
def test_divergence_consistency(p, pt):
    """For v in P_p (all components), Sum_{j in S_i} D_ij v_j = int_{T_i^st} phi~ div v (Eq. CS_10)."""
    d = make(2, p, pt, dt=0.05)
    val, der = _poly_field(p, np.random.default_rng(3))
    m = d.mesh
    V = np.zeros((m.nf, 3, d.Nst))
    for j in range(m.nf):
        for c in range(3):
            for _, Vt in m.dual_subtets(j):
                x, w = map_tet(Vt, *tet_rule(p + 1))
                V[j, c, :d.N] += (d.psi(j, x) * w[:, None]).T @ val(x, c)
    div = ops.divergence(d, V)
    for i in range(m.ne):
        x, w = map_tet(m.X[m.T[i]], *tet_rule(p + 1))
        ph, _ = d.phi(i, x)
        want = 0.05 * (ph * w[:, None]).T @ sum(der(x, c, c) for c in range(3))
        assert np.abs(div[i, :d.N] - want).max() < 1e-11 * max(1.0, np.abs(want).max())
        if d.Nst > d.N:
            assert np.abs(div[i, d.N:]).max() < 1e-12


def test_corollaries_1_2_cfg_tiny():
    """p_t = 0 (the 162-tet, p = 1 workload): A symmetric (Cor. 1), -A positive semidefinite
    (Cor. 2) with exactly one zero eigenvalue (the constant); pinned -A positive definite."""
    d = make(3, 1, 0, dt=0.01)
    A = ops.pressure_dense(d, pinned=False)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    ev = np.linalg.eigvalsh(-0.5 * (A + A.T))
    assert ev.min() > -1e-12 * ev.max()
    assert (ev < 1e-10 * ev.max()).sum() == 1
    assert np.abs(A @ np.tile(np.eye(d.N)[0], d.mesh.ne)).max() < 1e-14 * np.abs(A).max()
    Ap = ops.pressure_dense(d, pinned=True)
    np.linalg.cholesky(-Ap)
    assert np.linalg.eigvalsh(-Ap).min() > 0


def test_null_space_and_kronecker_structure_pt1():
    """p_t = 1: null(A) = constants (x) R^{N_gamma} (reading R4) and the literal space-time
    operator equals A^sp (x) dt^2 K^-1 (derived structure K2)."""
    d1 = make(2, 2, 1, dt=0.01)
    d0 = make(2, 2, 0, dt=0.01)
    A = ops.pressure_dense(d1, pinned=False)
    A0 = ops.pressure_dense(d0, pinned=False) / 0.01 ** 2
    ev = np.linalg.eigvals(A)
    assert (np.abs(ev) < 1e-10 * np.abs(ev).max()).sum() == 2
    assert ev.real.max() < 1e-10 * np.abs(ev).max()
    Tp = 0.01 ** 2 * np.linalg.inv(K_closed(1))
    N, Nst, ne = d1.N, d1.Nst, d1.mesh.ne
    for a in range(2):
        for b in range(2):
            ia = (np.arange(ne)[:, None] * Nst + a * N + np.arange(N)[None, :]).ravel()
            ib = (np.arange(ne)[:, None] * Nst + b * N + np.arange(N)[None, :]).ravel()
            assert np.abs(A[np.ix_(ia, ib)] - A0 * Tp[a, b]).max() < 1e-14 * np.abs(A).max()


def test_corollaries_3_4_viscous_spd():
    d = make(2, 2, 0, dt=0.02)
    L = ops.viscous_sparse(d, 0.3).toarray()
    assert np.abs(L - L.T).max() < 1e-14 * np.abs(L).max()
    np.linalg.cholesky(L)


def test_sparse_matches_matrix_free():
    d = make(2, 2, 1, dt=0.01)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((d.mesh.ne, d.Nst))
    A = ops.pressure_sparse(d)
    assert np.allclose(A @ x.ravel(), ops.pressure_apply(d, x).ravel(), rtol=0, atol=1e-15 * np.abs(x).max())
    L = ops.viscous_sparse(d, 0.2)
    assert np.allclose(L @ x.ravel(), ops.viscous_apply(d, x, 0.2).ravel(), rtol=0, atol=1e-15 * np.abs(x).max())


def test_viscous_kronecker_structure_and_time_decoupling():
    """p_t = 1: the literal space-time viscous operator of Eq. A1_mod equals D (x) K + G (x) I, with
    D = diag(|J_i|) (x) I_N the spatial mass (diagonal for the orthonormal basis) and G the spatial
    viscous part (the p_t = 0 operator minus D; symmetric positive definite).  Consequence used by
    the time-decoupled viscous solver: with K = W R W^-1, x = (I (x) W) y splits the system into one
    system per eigenvalue of K, and solving those reproduces the direct solve."""
    nu, dt = 0.2, 0.01
    d1 = make(2, 2, 1, dt=dt)
    d0 = make(2, 2, 0, dt=dt)
    N, ne = d1.N, d1.mesh.ne
    V1 = ops.viscous_sparse(d1, nu).toarray()
    V0 = ops.viscous_sparse(d0, nu).toarray()
    D = np.zeros_like(V0)
    for i in range(ne):
        Mi = d0.tet_blocks(i)["Mbar"]
        assert np.abs(Mi - np.diag(np.diag(Mi))).max() <= 1e-14 * np.abs(Mi).max()
        D[i * N:(i + 1) * N, i * N:(i + 1) * N] = Mi
    G = V0 - D
    assert np.abs(G - G.T).max() <= 1e-13 * np.abs(G).max()
    np.linalg.cholesky(G)
    K = K_closed(1)
    for a in range(2):
        for b in range(2):
            ia = (np.arange(ne)[:, None] * 2 * N + a * N + np.arange(N)[None, :]).ravel()
            ib = (np.arange(ne)[:, None] * 2 * N + b * N + np.arange(N)[None, :]).ravel()
            ref = D * K[a, b] + (G if a == b else 0.0)
            assert np.abs(V1[np.ix_(ia, ib)] - ref).max() <= 1e-13 * np.abs(V1).max()
    # decoupling: K has the complex pair 2 +- i sqrt(2); with its eigenvectors each time mode solves
    # (lambda D + G) y = b~ (complex symmetric), and x = W y
    lam, Wc = np.linalg.eig(K)
    assert np.allclose(sorted(lam, key=lambda z: z.imag), [2 - 1j * np.sqrt(2), 2 + 1j * np.sqrt(2)])
    rhs = np.random.default_rng(7).standard_normal(ne * 2 * N)
    x_direct = np.linalg.solve(V1, rhs)
    B = rhs.reshape(ne, 2, N)
    Bt = np.einsum("ab,ibk->iak", np.linalg.inv(Wc), B)
    Y = np.zeros_like(Bt, dtype=complex)
    for q in range(2):
        Y[:, q, :] = np.linalg.solve(lam[q] * D + G, Bt[:, q, :].ravel()).reshape(ne, N)
    X = np.einsum("ab,ibk->iak", Wc, Y)
    assert np.abs(X.imag).max() <= 1e-10 * np.abs(X).max()
    assert np.abs(X.real.ravel() - x_direct).max() <= 1e-11 * np.abs(x_direct).max()


def test_constant_mode_restriction():
    """Premise of the KRON_MG coarse correction: Dubiner function 0 is constant on the reference tet,
    so the piecewise-constant coarse space of a mesh is spanned by the coefficients k = 0, the
    Galerkin restriction R (-A) R^T of the pinned pressure operator is the matrix of the (0, 0)
    entries of its blocks, and that matrix is symmetric positive definite."""
    from oracle.basis import dubiner
    d = make(2, 2, 0, dt=0.01)
    xi = tet_rule(3)[0]
    phi, _ = dubiner(2, xi)
    assert np.abs(phi[:, 0] - phi[0, 0]).max() <= 1e-14 and np.abs(phi[:, 1:]).max() > 0.1
    A = -ops.pressure_dense(d, pinned=True)
    N, ne = d.N, d.mesh.ne
    R = np.zeros((ne, ne * N))
    R[np.arange(ne), np.arange(ne) * N] = 1.0
    A0 = R @ A @ R.T
    assert np.array_equal(A0, A[::N, ::N])
    assert np.abs(A0 - A0.T).max() <= 1e-14 * np.abs(A0).max()
    np.linalg.cholesky(A0)
    # a coefficient vector with only constant modes is a piecewise-constant field
    c = np.random.default_rng(3).standard_normal(ne)
    x = R.T @ c
    assert np.array_equal(x.reshape(ne, N)[:, 1:], np.zeros((ne, N - 1)))
