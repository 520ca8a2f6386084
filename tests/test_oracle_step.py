"""Pins for the oracle's Picard pressure-correction step (Sec. 2.6)."""
import numpy as np
import pytest

from inputs import BeltramiParams, beltrami_velocity, kuhn_mesh
from oracle import operators as ops
from oracle.blocks import SpaceTimeDG, map_tet
from oracle.krylov import cg, gmres
from oracle.mesh import Mesh
from oracle.step import initial_state, time_step


def make(n, p, pt, dt):
    v, t = kuhn_mesh(n, seed=0)
    return SpaceTimeDG(Mesh(v, t), p, pt, dt)


def test_krylov_solvers_match_direct():
    d = make(2, 2, 1, 0.01)
    A = ops.pressure_sparse(d)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0]); b[ops.pin_index(d)] = 0.0
    from scipy.sparse.linalg import spsolve
    xd = spsolve(A.tocsc(), b)
    x, it, res = gmres(lambda v: A @ v, b, np.zeros_like(b), 1e-13, restart=50)
    assert res <= 1e-13 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    d0 = make(2, 2, 0, 0.01)
    A0 = ops.pressure_sparse(d0)
    b0 = rng.standard_normal(A0.shape[0]); b0[ops.pin_index(d0)] = 0.0
    x, it, res = cg(lambda v: -(A0 @ v), -b0, np.zeros_like(b0), 1e-13)
    xd = spsolve(A0.tocsc(), b0)
    assert res <= 1e-13 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("p,pt,npic", [(1, 0, 2), (2, 1, 2)])
def test_step_is_discretely_divergence_free(p, pt, npic):
    """After the update (Eq. A3_mod), Sum_j D_ij v_j = 0 (Eq. CS_15) on every unpinned tet."""
    prm = BeltramiParams(nu=0.1)
    d = make(2, p, pt, 0.01)
    st = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    st = time_step(d, st, prm.nu, npic, lambda x, t: beltrami_velocity(x, t, prm), method="direct")
    div = ops.divergence(d, st.V)
    b0 = np.abs(ops.divergence(d, ops.project_initial(d, lambda x: beltrami_velocity(x, 0.0, prm)))).max()
    assert np.abs(div[1:]).max() < 1e-12 * max(b0, 1e-3)


def test_krylov_step_matches_direct_step():
    prm = BeltramiParams(nu=0.1)
    d = make(2, 1, 1, 0.01)
    vbc = lambda x, t: beltrami_velocity(x, t, prm)
    s0 = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    a = time_step(d, s0, prm.nu, 2, vbc, tol=1e-13, method="direct")
    b = time_step(d, s0, prm.nu, 2, vbc, tol=1e-13, method="krylov")
    assert np.linalg.norm(a.P - b.P) <= 1e-8 * np.linalg.norm(a.P)
    assert np.linalg.norm(a.V - b.V) <= 1e-10 * np.linalg.norm(a.V)


def test_free_stream_preserved():
    """A uniform velocity with matching boundary data stays uniform, pressure stays 0."""
    d = make(2, 1, 1, 0.05)
    u = np.array([1.0, 0.5, -0.3])
    const = lambda x, t=0.0: np.tile(u, (len(x), 1))
    st = initial_state(d, const)
    V0 = st.V.copy()
    st = time_step(d, st, 0.2, 2, const, method="direct")
    assert np.abs(st.V - V0).max() < 1e-12
    assert np.abs(st.P).max() < 1e-9


def _l2_velocity_error(d, st, prm):
    vbar = ops.average(d, st.V)
    err = 0.0
    for i in range(d.mesh.ne):
        x, w = map_tet(d.mesh.X[d.mesh.T[i]], *d.tet_nl)
        ph, _ = d.phi(i, x)
        vh = np.stack([ph @ (d.g1 @ vbar[i, c].reshape(d.Ng, d.N)) for c in range(3)], 1)
        err += (w * ((vh - beltrami_velocity(x, st.t, prm)) ** 2).sum(1)).sum()
    return np.sqrt(err)


def test_design_order_velocity_p1_pt1():
    """Beltrami data, p = p_t = 1, N_pic = 2, dt ~ h: L2 velocity error at t_end decays at
    order >= p + 1 - 0.3 (Table 2 reports p + 1 for velocity)."""
    prm = BeltramiParams(nu=0.1)
    errs = []
    for n in (2, 3, 4):
        d = make(n, 1, 1, 0.05 / n)
        st = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
        for _ in range(n):
            st = time_step(d, st, prm.nu, 2, lambda x, t: beltrami_velocity(x, t, prm), method="direct")
        errs.append(_l2_velocity_error(d, st, prm))
    orders = [np.log(errs[k] / errs[k + 1]) / np.log((k + 3) / (k + 2)) for k in range(2)]
    assert min(orders) >= 1.7, (errs, orders)


def _project_pressure(d, fn):
    """L2 projection of a scalar function onto each tet's pressure basis (p_t = 0)."""
    P = np.zeros((d.mesh.ne, d.Nst))
    for i in range(d.mesh.ne):
        x, w = map_tet(d.mesh.X[d.mesh.T[i]], *d.tet_nl)
        ph, _ = d.phi(i, x)
        G = ph.T @ (w[:, None] * ph)
        P[i] = np.linalg.solve(G, ph.T @ (w * fn(x)))
    return P


def test_theta_method_from_zero_pressure_rescales_the_pressure():
    """Eqs. CS_15_theta / CS_16_theta: the momentum of a dual cell sees the pressure only through
    p^{n+theta} = theta p^{n+1} + (1-theta) p^n.  From p^n = 0 the theta step therefore takes the
    same velocity iterates as the implicit step, with p^{n+1} = p^{n+1}(theta = 1) / theta."""
    prm = BeltramiParams(nu=0.1)
    d = make(2, 1, 0, 0.02)
    vbc = lambda x, t: beltrami_velocity(x, t, prm)
    s0 = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    a = time_step(d, s0, prm.nu, 2, vbc, tol=1e-13, method="direct")
    for th in (0.5, 0.51, 0.8):
        b = time_step(d, s0, prm.nu, 2, vbc, tol=1e-13, method="direct", theta=th)
        assert np.abs(b.V - a.V).max() <= 1e-13 * np.abs(a.V).max()
        assert np.abs(th * b.P - a.P).max() <= 1e-12 * np.abs(a.P).max()


@pytest.mark.parametrize("theta", [0.5, 0.51, 0.75, 1.0])
def test_theta_method_on_uniform_flow_with_linear_pressure(theta):
    """Inviscid uniform Dirichlet flow u with a linear pressure c.x at t^n: the velocity stays u,
    and since a steady u needs p^{n+theta} constant, p^{n+1} = -(1-theta)/theta (c.x - C), where C
    is the constant that the pin (constant mode of tet 0) removes.  The discrete gradient of a
    linear pressure is exact and nu = 0 leaves the predictor a pure mass solve, so one Picard
    iteration already reaches this; the second changes nothing."""
    d = make(2, 2, 0, 0.05)
    u = np.array([0.7, -0.2, 0.4])
    const = lambda x, t=0.0: np.tile(u, (len(x), 1))
    c = np.array([0.3, -1.1, 0.6])
    st = initial_state(d, const)
    V0 = st.V.copy()
    st.P = _project_pressure(d, lambda x: x @ c)
    C = np.zeros_like(st.P)
    C[:, 0] = st.P[0, 0]                         # the Dubiner constant mode has the same value on every tet
    out = time_step(d, st, 0.0, 2, const, tol=1e-13, method="direct", theta=theta)
    assert np.abs(out.V - V0).max() <= 1e-12
    expect = -(1.0 - theta) / theta * (st.P - C)
    assert np.abs(out.P - expect).max() <= 1e-10 * max(np.abs(st.P).max(), 1.0)


def test_theta_method_rejects_space_time_pressure():
    d = make(2, 1, 1, 0.02)
    s0 = initial_state(d, lambda x: np.zeros((len(x), 3)))
    with pytest.raises(ValueError):
        time_step(d, s0, 0.1, 1, lambda x, t: np.zeros((len(x), 3)), method="direct", theta=0.5)
    d0 = make(2, 1, 0, 0.02)
    s0 = initial_state(d0, lambda x: np.zeros((len(x), 3)))
    with pytest.raises(ValueError):
        time_step(d0, s0, 0.1, 1, lambda x, t: np.zeros((len(x), 3)), method="direct", theta=0.4)
