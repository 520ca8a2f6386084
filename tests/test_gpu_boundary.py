"""The data and memory boundary of the C ABI against the oracle:

* initial and Dirichlet velocity from a host callback (stdg_set_initial_fn, stdg_set_boundary_fn),
* the solenoidal no-slip field of the largest configuration as a device kind (STDG_FIELD_CURL_MODES),
* every device array from the caller's allocator (stdg_solver_create_alloc, PyTorch's caching
  allocator in the Python binding), counted byte by byte."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import BeltramiParams, SolenoidalModes, beltrami_velocity, kuhn_mesh
from oracle import operators as ops
from oracle.blocks import SpaceTimeDG
from oracle.mesh import Mesh
from oracle.step import initial_state, time_step

STEP_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_07384_gb300.build import build
    build()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def moments(gs, d, V):
    return gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)


def oracle_moments(d, V):
    U = np.zeros((d.mesh.nf, 2, 3, d.Nst))
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            U[j, s] = (fb["Mij"][s] @ V[j].T).T
    return U


def modes_field(g, sm):
    return g.curl_modes(sm.k, sm.a, sm.phi, sm.scale)


def setup(n, p, pt, dt=0.01, **kw):
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(n, seed=0)
    return g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, **kw), SpaceTimeDG(Mesh(v, t), p, pt, dt)


@pytest.mark.parametrize("p,pt", [(2, 1), (3, 1)])
def test_curl_modes_initial_projection_matches_oracle(p, pt):
    """The seeded solenoidal field curl(b Psi) (64 modes, |v|max 0.1) projected on the device
    equals the oracle's projection of the same field evaluated by the input generator."""
    import paper_1601_07384_gb300 as g
    sm = SolenoidalModes(seed=1)
    gs, d = setup(2, p, pt)
    gs.set_initial(modes_field(g, sm))
    _, V, _ = gs.get_state()
    Uo = oracle_moments(d, ops.project_initial(d, lambda x: sm(x)))
    assert rel(moments(gs, d, V), Uo) <= 1e-12


def test_callback_initial_projection_matches_oracle():
    """Any velocity through the host callback: the same projection as the oracle's."""
    sm = SolenoidalModes(seed=3, vmax=0.5)
    gs, d = setup(2, 3, 1)
    calls = []

    def v0(x, t):
        calls.append(len(x))
        assert np.all(t == 0.0)
        return sm(x)

    gs.set_initial(v0)
    nq1 = -(-(3 * 3 + 2) // 2)                                      # ceil((3p+2)/2) points per direction
    assert calls and calls[0] == d.mesh.nf * 2 * nq1 ** 3
    _, V, _ = gs.get_state()
    Uo = oracle_moments(d, ops.project_initial(d, lambda x: sm(x)))
    assert rel(moments(gs, d, V), Uo) <= 1e-12


@pytest.mark.parametrize("precision,method", [("fp64", "kron_cg"), ("mixed_f32", "kron_mg")])
def test_step_with_callback_data_and_counted_allocator(precision, method):
    """Two steps with initial and Dirichlet data from host callbacks (Beltrami, t-dependent) and
    every device array from PyTorch's caching allocator: equal to the oracle's steps, and equal to
    the same steps with the device Beltrami kind; every byte handed out comes back at destroy."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(2, 2, 1, precision=precision, allocator="torch")
    seen_t = []

    def vbc(x, t):
        seen_t.append((t.min(), t.max()))
        return beltrami_velocity(x, t, prm)

    gs.set_initial(lambda x, t: beltrami_velocity(x, 0.0, prm))
    gs.set_boundary(vbc)
    gk, _ = setup(2, 2, 1, precision=precision, allocator="cuda")
    gk.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gk.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    for k in range(2):
        gs.step(prm.nu, 2, method=method, tol=1e-13)
        gk.step(prm.nu, 2, method=method, tol=1e-13)
        so = time_step(d, so, prm.nu, 2, lambda x, tt: beltrami_velocity(x, tt, prm), tol=1e-13, method="direct")
        lo, hi = seen_t[-1]
        assert lo >= k * 0.01 - 1e-15 and hi <= (k + 1) * 0.01 + 1e-15 and hi > lo
    P, V, _ = gs.get_state()
    Pk, Vk, _ = gk.get_state()
    assert rel(P.cpu().numpy(), so.P.ravel()) <= STEP_TOL
    assert rel(moments(gs, d, V), oracle_moments(d, so.V)) <= STEP_TOL
    assert rel(P.cpu().numpy(), Pk.cpu().numpy()) <= 1e-11       # data rounded differently, solves to 1e-13
    live, count = gs.alloc_stats()
    assert count > 20 and live > 0
    assert torch.cuda.memory_allocated() >= live
    gs.__del__()
    assert gs.alloc_stats()[0] == 0


def test_allocator_owns_the_device_memory():
    """With the caller's allocator the library obtains no device memory of its own: the drop in free
    device memory over solver creation and a step is what PyTorch's allocator reserved (plus a small
    allowance for kernel modules and CUDA graphs), for a solver of ~0.4 GB."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.01)
    v, t = kuhn_mesh(8, seed=0)
    mesh, ref = g.Mesh(v, t), g.Reference(3, 1)
    warm = g.Solver(mesh, ref, 0.005, precision="mixed_f32", allocator="cuda")    # loads the kernels once
    warm.set_initial(g.beltrami(prm.a, prm.d, prm.nu)); warm.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    warm.step(prm.nu, 1, method="kron_mg", tol=1e-10)
    del warm
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    s = g.Solver(mesh, ref, 0.005, precision="mixed_f32", allocator="torch")
    s.set_initial(g.beltrami(prm.a, prm.d, prm.nu)); s.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    s.step(prm.nu, 1, method="kron_mg", tol=1e-10)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    res1 = torch.cuda.memory_reserved()
    live, count = s.alloc_stats()
    assert live > 250e6, live
    assert res1 - res0 >= live
    assert (free0 - free1) <= (res1 - res0) + 96 * 2 ** 20, (free0 - free1, res1 - res0)


def test_noslip_step_with_curl_modes_matches_oracle():
    """The largest configuration's data at small size: the solenoidal field as initial velocity,
    no-slip walls (zero Dirichlet data), nu = 1e-3, dt = 0.01, p = p_t = 2: two steps against the oracle."""
    import paper_1601_07384_gb300 as g
    sm = SolenoidalModes(seed=1)
    nu = 1e-3
    gs, d = setup(2, 2, 2, precision="mixed_f32")
    gs.set_initial(modes_field(g, sm))
    gs.set_boundary(g.zero())
    so = initial_state(d, lambda x: sm(x))
    zero = lambda x, tt: np.zeros(np.shape(x))
    for _ in range(2):
        gs.step(nu, 3, method="kron_mg", tol=1e-13)
        so = time_step(d, so, nu, 3, zero, tol=1e-13, method="direct")
    P, V, _ = gs.get_state()
    assert rel(P.cpu().numpy(), so.P.ravel()) <= STEP_TOL
    assert rel(moments(gs, d, V), oracle_moments(d, so.V)) <= STEP_TOL


def test_callback_errors_surface():
    import paper_1601_07384_gb300 as g
    gs, _ = setup(2, 1, 0)

    def bad(x, t):
        raise ValueError("boom")

    with pytest.raises(ValueError, match="boom"):
        gs.set_initial(bad)
    with pytest.raises(g.StdgError, match="EINVAL"):
        gs.set_boundary(g.curl_modes(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0)))
