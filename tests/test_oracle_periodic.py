"""Pins for the oracle on periodic meshes: the ABC-flow convergence test of the paper (Sec. 3.2,
Eq. CT_1, Table 1) on [-pi, pi)^3 with periodic boundaries everywhere."""
import numpy as np
import pytest

from inputs import abc_pressure, abc_velocity, kuhn_periodic_mesh
from oracle import operators as ops
from oracle.blocks import SpaceTimeDG, map_tet
from oracle.mesh import Mesh
from oracle.step import initial_state, time_step


def make(n, p, pt, dt):
    v, t, per = kuhn_periodic_mesh(n)
    return SpaceTimeDG(Mesh(v, t, period=per), p, pt, dt)


def test_periodic_faces_and_dual_cells():
    """Every face is interior (2 N_e faces), its normal points from l(j) towards r(j)'s image
    next to it, and the dual cells tile the periodic box."""
    d = make(3, 1, 0, 0.05)
    m = d.mesh
    assert m.interior.all() and m.nf == 2 * m.ne
    vol = 0.0
    for j in range(m.nf):
        (_, Vl), (_, Vr) = m.dual_subtets(j)
        assert np.dot(m.normal[j], Vr[3] - Vl[3]) > 0
        vol += sum(abs(np.linalg.det((V[1:] - V[0]).T)) / 6 for V in (Vl, Vr))
    assert abs(vol - (2 * np.pi) ** 3) < 1e-10


def test_periodic_constant_null_space():
    """Without the pin, constants are the null space of the periodic pressure operator."""
    d = make(3, 2, 1, 0.05)
    ne, N, Ng = d.mesh.ne, d.N, d.Ng
    P = np.zeros((ne, d.Nst))
    for i in range(ne):                            # constant 1 in every time function
        x, w = map_tet(d.mesh.tet_coords(i), *d.tet_nl)
        ph, _ = d.phi(i, x)
        c = np.linalg.solve(ph.T @ (w[:, None] * ph), ph.T @ w)
        for a in range(Ng):
            P[i, a * N:(a + 1) * N] = c
    y = ops.pressure_apply(d, P, pinned=False)
    A = ops.pressure_sparse(d, pinned=False)
    assert np.abs(y).max() <= 1e-12 * abs(A).max() * np.abs(P).max()


def test_periodic_free_stream_and_divergence():
    """A uniform velocity stays uniform with zero pressure; with ABC data a step leaves the
    discrete divergence at rounding level."""
    d = make(3, 1, 1, 0.05)
    u = np.array([0.7, -0.4, 0.2])
    const = lambda x, t=0.0: np.tile(u, (len(x), 1))
    st = initial_state(d, const)
    V0 = st.V.copy()
    st = time_step(d, st, 0.0, 2, const, method="direct")
    assert np.abs(st.V - V0).max() < 1e-12 and np.abs(st.P).max() < 1e-10
    st = initial_state(d, lambda x: abc_velocity(x, 0.0, 1.0))
    st = time_step(d, st, 1.0, 2, lambda x, t: abc_velocity(x, t, 1.0), method="direct")
    assert np.abs(ops.divergence(d, st.V)).max() < 1e-12


def _errors(d, st):
    """L2 errors at t of the velocity averaged onto the tets and of the pressure, the constant
    removed from both pressures by their means (Sec. 3.2: the exact pressure is defined up to a
    constant, chosen from the numerical mean)."""
    vbar = ops.average(d, st.V)
    ev, ws, ph_all, pe_all = 0.0, [], [], []
    for i in range(d.mesh.ne):
        x, w = map_tet(d.mesh.tet_coords(i), *d.tet_nl)
        ph, _ = d.phi(i, x)
        vh = np.stack([ph @ (d.g1 @ vbar[i, c].reshape(d.Ng, d.N)) for c in range(3)], 1)
        ev += (w * ((vh - abc_velocity(x, st.t, 0.0)) ** 2).sum(1)).sum()
        ph_all.append(ph @ (d.g1 @ st.P[i].reshape(d.Ng, d.N)))
        pe_all.append(abc_pressure(x, st.t, 0.0))
        ws.append(w)
    w, a, b = np.concatenate(ws), np.concatenate(ph_all), np.concatenate(pe_all)
    a = a - (w * a).sum() / w.sum()
    b = b - (w * b).sum() / w.sum()
    return np.sqrt(ev), np.sqrt((w * (a - b) ** 2).sum())


def test_steady_abc_orders_p1():
    """Steady ABC flow (nu = 0, p = 1, p_t = 0, N_pic = 2) to t = 0.1 with dt = 0.1 / n (dt
    proportional to h, as the paper's CFL condition): on n = 3, 4, 5 the velocity error decays at
    order >= 1.6 and the pressure error at order >= 1.9 (Table 1 reports 2.0 for both at p = 1;
    the velocity order here is 1.65, 1.75, and 1.78, 1.91 on n = 4, 6, 8)."""
    errs = []
    for n in (3, 4, 5):
        d = make(n, 1, 0, 0.1 / n)
        st = initial_state(d, lambda x: abc_velocity(x, 0.0, 0.0))
        for _ in range(n):
            st = time_step(d, st, 0.0, 2, lambda x, t: abc_velocity(x, t, 0.0), method="direct")
        errs.append(_errors(d, st))
    ev, ep = np.array(errs).T
    ov = [np.log(ev[0] / ev[1]) / np.log(4 / 3), np.log(ev[1] / ev[2]) / np.log(5 / 4)]
    op = [np.log(ep[0] / ep[1]) / np.log(4 / 3), np.log(ep[1] / ep[2]) / np.log(5 / 4)]
    assert min(ov) >= 1.6 and min(op) >= 1.9, (errs, ov, op)


def test_steady_abc_orders_p2():
    """The same at p = 2 (N_pic = 3) on n = 3, 4: velocity order >= 2.3 and pressure order >= 2.7
    (Table 1: 2.4 and 3.0; measured here 2.60 and 2.95, and 2.60 and 2.94 from n = 4 to 6)."""
    errs = []
    for n in (3, 4):
        d = make(n, 2, 0, 0.1 / n)
        st = initial_state(d, lambda x: abc_velocity(x, 0.0, 0.0))
        for _ in range(n):
            st = time_step(d, st, 0.0, 3, lambda x, t: abc_velocity(x, t, 0.0), method="direct")
        errs.append(_errors(d, st))
    (v3, p3), (v4, p4) = errs
    ov, op = np.log(v3 / v4) / np.log(4 / 3), np.log(p3 / p4) / np.log(4 / 3)
    assert ov >= 2.3 and op >= 2.7, (errs, ov, op)


def test_unsteady_abc_orders_p1_pt1():
    """Unsteady ABC flow (nu = 1, p = p_t = 1, N_pic = 2, space-time pressure and implicit
    viscosity) to t = 0.1 with dt = 0.1 / n on n = 3, 4: velocity order >= 1.7, pressure order
    >= 1.4 (Table 2: 2.0 and 1.5-1.6; measured here 1.88 and 1.98, and 2.11 and 2.10 from n = 4
    to 6)."""
    nu = 1.0
    errs = []
    for n in (3, 4):
        d = make(n, 1, 1, 0.1 / n)
        st = initial_state(d, lambda x: abc_velocity(x, 0.0, nu))
        for _ in range(n):
            st = time_step(d, st, nu, 2, lambda x, t: abc_velocity(x, t, nu), method="direct")
        vbar = ops.average(d, st.V)
        ev, ws, pa, pb = 0.0, [], [], []
        for i in range(d.mesh.ne):
            x, w = map_tet(d.mesh.tet_coords(i), *d.tet_nl)
            ph, _ = d.phi(i, x)
            vh = np.stack([ph @ (d.g1 @ vbar[i, c].reshape(d.Ng, d.N)) for c in range(3)], 1)
            ev += (w * ((vh - abc_velocity(x, st.t, nu)) ** 2).sum(1)).sum()
            pa.append(ph @ (d.g1 @ st.P[i].reshape(d.Ng, d.N))); pb.append(abc_pressure(x, st.t, nu)); ws.append(w)
        w, a, b = np.concatenate(ws), np.concatenate(pa), np.concatenate(pb)
        a, b = a - (w * a).sum() / w.sum(), b - (w * b).sum() / w.sum()
        errs.append((np.sqrt(ev), np.sqrt((w * (a - b) ** 2).sum())))
    (v3, p3), (v4, p4) = errs
    ov, op = np.log(v3 / v4) / np.log(4 / 3), np.log(p3 / p4) / np.log(4 / 3)
    assert ov >= 1.7 and op >= 1.4, (errs, ov, op)
