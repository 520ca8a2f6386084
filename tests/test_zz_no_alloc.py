"""stdg_solve_noalloc -- the pressure solve for callers that may not allocate device memory
while running (their device memory belongs to another allocator, or allocation latency is not
acceptable in their loop).  It must give what stdg_solve(KRON_CG) gives, call after call, with
its work vectors in the library's fixed device array, and solve the oracle's pinned system.
This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_07384_gb300.build import build
    build()


def make(n, p, pt, dt=0.01):
    # stdg_solve is compared in its unbatched configuration (one host check per CG iteration), the
    # iteration the allocation-free variant runs; graph batching may add up to 7 iterations.
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh
    v, t = kuhn_mesh(n, seed=0)
    return g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, graph_batch=1)


@pytest.mark.parametrize("n,p,pt", [(3, 1, 0), (2, 2, 1), (4, 3, 1)])
def test_noalloc_solve_matches_solve_twice_in_a_row(n, p, pt):
    s = make(n, p, pt)
    rng = np.random.default_rng(n + p + pt)
    for call in range(2):
        b = rng.standard_normal(s.ne * s.Nst)
        b[[a * s.N for a in range(s.Ng)]] = 0.0          # pinned entries
        bt = torch.from_numpy(b).cuda()
        x_ref, st_ref = s.solve(bt, tol=1e-12, method="kron_cg")
        x = torch.full_like(bt, float("nan"))            # whatever the caller's buffer held
        x, st = s.solve_noalloc(bt, x, tol=1e-12)
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.abs(xn - xr).max() <= 1e-12 * np.abs(xr).max(), call
        assert st["rel_residual"] <= 2e-12 and st["iterations"] == st_ref["iterations"]


@pytest.mark.parametrize("n,p,pt", [(3, 1, 0), (3, 2, 1)])
def test_noalloc_on_a_fresh_solver_matches_oracle_and_allocates_nothing(n, p, pt):
    """First call on a solver that never ran stdg_solve (no Krylov vectors exist): the solution of
    the oracle's pinned system (sparse LU) within cond * tol; after the one call that resolves the
    array's address, a call changes neither free device memory nor the caller's allocator."""
    from scipy.sparse.linalg import spsolve
    from inputs import kuhn_mesh
    from oracle import operators as ops
    from oracle.blocks import SpaceTimeDG
    from oracle.mesh import Mesh
    s = make(n, p, pt)
    v, t = kuhn_mesh(n, seed=0)
    d = SpaceTimeDG(Mesh(v, t), p, pt, 0.01)
    A = ops.pressure_sparse(d)
    rng = np.random.default_rng(40 + n + p)
    tol = 1e-12
    cond = np.linalg.cond(A.toarray())
    for call in range(3):
        b = rng.standard_normal((d.mesh.ne, d.Nst))
        b[0, ops.pin_index(d)] = 0.0
        bt = torch.from_numpy(b.ravel()).cuda()
        x = torch.zeros_like(bt)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        n0 = s.alloc_stats()[1]
        x, st = s.solve_noalloc(bt, x, tol=tol)
        torch.cuda.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0
            assert s.alloc_stats()[1] == n0
        xn = x.cpu().numpy()
        assert np.linalg.norm(b.ravel() - A @ xn) <= 2 * tol * np.linalg.norm(b)
        xd = spsolve(A.tocsc(), b.ravel())
        assert np.linalg.norm(xn - xd) <= 10 * cond * tol * np.linalg.norm(xd)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import paper_1601_07384_gb300 as g
    s = make(11, 3, 1)                                   # 7986 tets x 40 = 319,440 > 262,144
    b = torch.zeros(s.ne * s.Nst, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(g.StdgError, match="allocation-free limit"):
        s.solve_noalloc(b, x)
