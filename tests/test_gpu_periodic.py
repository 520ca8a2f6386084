"""Periodic boundaries on the GPU path (Sec. 3.2, Eq. CT_1): step parity with the oracle on the
periodic Kuhn mesh of [-pi, pi)^3, and the convergence orders of the ABC-flow test (Tables 1-2)
reproduced by the GPU path on the meshes and time steps the oracle's pins use."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import abc_pressure, abc_velocity, kuhn_periodic_mesh
from oracle import operators as ops
from oracle.blocks import SpaceTimeDG, map_tet
from oracle.mesh import Mesh
from oracle.step import initial_state, time_step

STEP_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_07384_gb300.build import build
    build()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make(n, p, pt, dt, **kw):
    import paper_1601_07384_gb300 as g
    v, t, per = kuhn_periodic_mesh(n)
    gs = g.Solver(g.Mesh(v, t, period=per), g.Reference(p, pt), dt, **kw)
    return gs, SpaceTimeDG(Mesh(v, t, period=per), p, pt, dt)


def moments(gs, d, V):
    return gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)


def oracle_moments(d, V):
    U = np.zeros((d.mesh.nf, 2, 3, d.Nst))
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            U[j, s] = (fb["Mij"][s] @ V[j].T).T
    return U


def test_periodic_blocks_match_oracle_operator():
    """The per-face blocks of the periodic mesh (dual cells across the box faces) against the
    oracle's operator, one application, 1e-12."""
    gs, d = make(3, 2, 1, 0.05)
    x = np.random.default_rng(4).standard_normal(d.mesh.ne * d.Nst)
    y = gs.pressure_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ops.pressure_apply(d, x).ravel()) <= 1e-12


@pytest.mark.parametrize("precision,method", [("fp64", "kron_cg"), ("mixed_f32", "kron_mg")])
def test_periodic_steps_match_oracle(precision, method):
    """Two steps of unsteady ABC flow (nu = 1, p = 2, p_t = 1) on the periodic 3^3 mesh, initial
    data through the host callback: pressure and velocity to 1e-10."""
    nu, dt = 1.0, 0.05
    gs, d = make(3, 2, 1, dt, precision=precision)
    gs.set_initial(lambda x, t: abc_velocity(x, 0.0, nu))
    so = initial_state(d, lambda x: abc_velocity(x, 0.0, nu))
    for _ in range(2):
        gs.step(nu, 2, method=method, tol=1e-13)
        so = time_step(d, so, nu, 2, lambda x, t: abc_velocity(x, t, nu), tol=1e-13, method="direct")
    P, V, t = gs.get_state()
    assert abs(t - so.t) < 1e-14
    assert rel(P.cpu().numpy(), so.P.ravel()) <= STEP_TOL
    assert rel(moments(gs, d, V), oracle_moments(d, so.V)) <= STEP_TOL


def _errors(d, P, V, t, nu):
    """L2 errors of the averaged velocity and of the mean-free pressure at time t (Sec. 3.2)."""
    vbar = ops.average(d, V)
    ev, ws, pa, pb = 0.0, [], [], []
    for i in range(d.mesh.ne):
        x, w = map_tet(d.mesh.tet_coords(i), *d.tet_nl)
        ph, _ = d.phi(i, x)
        vh = np.stack([ph @ (d.g1 @ vbar[i, c].reshape(d.Ng, d.N)) for c in range(3)], 1)
        ev += (w * ((vh - abc_velocity(x, t, nu)) ** 2).sum(1)).sum()
        pa.append(ph @ (d.g1 @ P[i].reshape(d.Ng, d.N))); pb.append(abc_pressure(x, t, nu)); ws.append(w)
    w, a, b = np.concatenate(ws), np.concatenate(pa), np.concatenate(pb)
    a, b = a - (w * a).sum() / w.sum(), b - (w * b).sum() / w.sum()
    return np.sqrt(ev), np.sqrt((w * (a - b) ** 2).sum())


def _gpu_run(n, p, pt, nu, npic, dt, nsteps):
    gs, d = make(n, p, pt, dt, precision="mixed_f32")
    gs.set_initial(lambda x, t: abc_velocity(x, 0.0, nu))
    for _ in range(nsteps):
        gs.step(nu, npic, method="kron_mg", tol=1e-12)
    P, V, t = gs.get_state()
    return _errors(d, P.cpu().numpy().reshape(d.mesh.ne, d.Nst), V.cpu().numpy().reshape(d.mesh.nf, 3, d.Nst), t, nu)


def _orders(errs, ns):
    ev, ep = np.array(errs).T
    f = [np.log(ns[k] / ns[k + 1]) for k in range(len(ns) - 1)]
    return ([np.log(ev[k] / ev[k + 1]) / -f[k] for k in range(len(f))],
            [np.log(ep[k] / ep[k + 1]) / -f[k] for k in range(len(f))])


@pytest.mark.parametrize("p,npic,ns,vmin,pmin", [(1, 2, (3, 4, 5), 1.6, 1.9), (2, 3, (3, 4), 2.3, 2.7)])
def test_steady_abc_orders_on_gpu(p, npic, ns, vmin, pmin):
    """Steady ABC flow (nu = 0, p_t = 0) to t = 0.1 with dt = 0.1 / n (Table 1: 2.0 / 2.0 at p = 1,
    2.4 / 3.0 at p = 2), the same thresholds as the oracle's pins."""
    errs = [_gpu_run(n, p, 0, 0.0, npic, 0.1 / n, n) for n in ns]
    ov, op = _orders(errs, ns)
    print(f"p={p}: errors {errs}, velocity orders {ov}, pressure orders {op}")
    assert min(ov) >= vmin and min(op) >= pmin, (errs, ov, op)


def test_steady_abc_order_p3_on_gpu():
    """p = 3 with dt proportional to h / (2p + 1) (the explicit-DG CFL scaling): dt = 0.3 / (7 n),
    7 n / 3 steps to t = 0.1 (n = 3, 6): velocity order >= 3.2, pressure order >= 3.5 (Table 1: 3.4
    and 3.9)."""
    ns = (3, 6)
    errs = [_gpu_run(n, 3, 0, 0.0, 3, 0.3 / (7 * n), 7 * n // 3) for n in ns]
    ov, op = _orders(errs, ns)
    print(f"p=3: errors {errs}, velocity orders {ov}, pressure orders {op}")
    assert min(ov) >= 3.2 and min(op) >= 3.5, (errs, ov, op)


def test_unsteady_abc_orders_on_gpu():
    """Unsteady ABC flow (nu = 1, p = p_t = 1, N_pic = 2) to t = 0.1 with dt = 0.1 / n on n = 3, 4, 6
    (Table 2: 2.0 velocity, 1.5-1.6 pressure): velocity >= 1.7, pressure >= 1.4."""
    ns = (3, 4, 6)
    errs = [_gpu_run(n, 1, 1, 1.0, 2, 0.1 / n, n) for n in ns]
    ov, op = _orders(errs, ns)
    print(f"p=p_t=1: errors {errs}, velocity orders {ov}, pressure orders {op}")
    assert min(ov) >= 1.7 and min(op) >= 1.4, (errs, ov, op)
