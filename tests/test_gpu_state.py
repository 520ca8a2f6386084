"""State handling on the GPU path: a run resumed from a saved state repeats the uninterrupted run
bit for bit, and a non-finite value in the state or a right-hand side stops the step or solve with
STDG_ENAN (found on the host from the residual norms; no device-side fault is involved)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import BeltramiParams, kuhn_mesh


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_07384_gb300.build import build
    build()


def make(precision="mixed_f32", n=3, p=2, pt=1, dt=0.01):
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(n, seed=0)
    s = g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, precision=precision)
    prm = BeltramiParams(nu=0.1)
    s.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    s.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    return s


@pytest.mark.parametrize("precision,method", [("mixed_f32", "kron_mg"), ("fp64", "kron_cg")])
def test_resume_from_saved_state_is_bitwise(precision, method):
    """5 steps in one solver against 2 steps, stdg_get_state to host buffers, a fresh solver,
    stdg_set_state, 3 more steps: identical bits (every reduction has a fixed order)."""
    nu = 0.1
    a = make(precision)
    for _ in range(5):
        a.step(nu, 2, method=method, tol=1e-10)
    Pa, Va, ta = a.get_state()
    b = make(precision)
    for _ in range(2):
        b.step(nu, 2, method=method, tol=1e-10)
    P2, V2, t2 = b.get_state()
    Ph, Vh = P2.cpu().clone(), V2.cpu().clone()
    del b
    c = make(precision)
    c.set_state(Ph.cuda(), Vh.cuda(), t2)
    for _ in range(3):
        c.step(nu, 2, method=method, tol=1e-10)
    Pc, Vc, tc = c.get_state()
    assert tc == ta
    assert torch.equal(Pc, Pa) and torch.equal(Vc, Va)


def test_nan_in_state_gives_enan():
    import paper_1601_07384_gb300 as g
    s = make("fp64")
    P, V, t = s.get_state()
    V[17] = float("nan")
    s.set_state(P, V, t)
    with pytest.raises(g.StdgError, match="ENAN"):
        s.step(0.1, 2, method="kron_cg", tol=1e-10)


@pytest.mark.parametrize("method", ["kron_cg", "gmres", "kron_mg"])
def test_nan_in_rhs_gives_enan(method):
    import paper_1601_07384_gb300 as g
    s = make("fp64")
    b = torch.randn(s.ne * s.Nst, dtype=torch.float64, device="cuda")
    b[5] = float("inf")
    with pytest.raises(g.StdgError, match="ENAN"):
        s.solve(b, tol=1e-10, method=method)
    x = torch.zeros_like(b)
    b[5] = float("nan")
    with pytest.raises(g.StdgError, match="ENAN"):
        s.solve_noalloc(b, x, tol=1e-10)
