"""GPU path vs the oracle, element by element, through the C ABI.

Tolerances: one operator application in FP64 agrees to 1e-12 relative (max-norm over the
output, scaled by the output's max); solves are compared through residuals measured with the
oracle's operator and against the oracle's direct solution within cond * tol; a full time step
(pressure and velocity coefficients) agrees to 1e-10 relative when both sides solve to 1e-13
(the GPU iteratively, the oracle by sparse LU)."""
import functools
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from inputs import BeltramiParams, beltrami_velocity, kuhn_mesh
from oracle import operators as ops
from oracle.blocks import SpaceTimeDG
from oracle.mesh import Mesh
from oracle.step import initial_state, time_step

STEP_TOL = 1e-10          # relative, pressure and velocity coefficients after each FP64 step
CASES = [(3, 1, 0), (2, 2, 1), (2, 3, 1), (2, 4, 2), (3, 2, 0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1601_07384_gb300.build import build
    build()


def setup(n, p, pt, dt=0.01, seed=0, **kw):
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(n, seed=seed)
    gs = g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, **kw)
    d = SpaceTimeDG(Mesh(v, t), p, pt, dt)
    return gs, d


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("n,p,pt", CASES)
def test_assembled_blocks_match_oracle_operator(n, p, pt):
    gs, d = setup(n, p, 0, dt=1.0)
    A = ops.pressure_dense(d, pinned=False) if d.mesh.ne * d.Nst <= 2000 else None
    if A is None:
        pytest.skip("dense oracle too large")
    B = gs.blocks()
    N = d.N
    scale = np.abs(A).max()
    for i in range(d.mesh.ne):
        assert np.abs(B["Bdiag"][i] - A[i * N:(i + 1) * N, i * N:(i + 1) * N]).max() <= 1e-12 * scale
    for j in np.nonzero(d.mesh.interior)[0]:
        l, r = d.mesh.left[j], d.mesh.right[j]
        assert np.abs(B["Aoff"][j] - A[l * N:(l + 1) * N, r * N:(r + 1) * N]).max() <= 1e-12 * scale


@pytest.mark.parametrize("n,p,pt", CASES)
@pytest.mark.parametrize("pinned", [True, False])
def test_pressure_apply_matches_oracle(n, p, pt, pinned):
    gs, d = setup(n, p, pt)
    x = np.random.default_rng(n + 10 * p + pt).standard_normal(d.mesh.ne * d.Nst)
    y = gs.pressure_apply(torch.from_numpy(x).cuda(), pinned=pinned).cpu().numpy()
    yo = ops.pressure_apply(d, x, pinned=pinned).ravel()
    assert rel(y, yo) <= 1e-12


@pytest.mark.parametrize("n,p,pt", CASES)
@pytest.mark.parametrize("pinned", [True, False])
def test_factored_operator_matches_oracle_and_assembled(n, p, pt, pinned):
    """Gradient -> M_j^-1 -> divergence per dual cell (Eq. CS_19 read literally) against the
    oracle, and against the assembled five-point blocks on the same input."""
    gs, d = setup(n, p, pt)
    x = np.random.default_rng(7 + n + 10 * p + pt).standard_normal(d.mesh.ne * d.Nst)
    xd = torch.from_numpy(x).cuda()
    yf = gs.pressure_apply_factored(xd, pinned=pinned).cpu().numpy()
    ya = gs.pressure_apply(xd, pinned=pinned).cpu().numpy()
    yo = ops.pressure_apply(d, x, pinned=pinned).ravel()
    assert rel(yf, yo) <= 1e-12
    assert rel(yf, ya) <= 1e-12


@pytest.mark.parametrize("n,p,pt", CASES)
def test_update_rhs_and_moments_match_oracle(n, p, pt):
    """v = -M^-1 Q dp (Eq. A3_mod with F = 0) compared through the basis-independent moments
    int phi~ v_h; then b = Sum_j D_ij v_j (Eq. A2_mod right-hand side) = -A dp."""
    gs, d = setup(n, p, pt)
    m = d.mesh
    dp = np.random.default_rng(7).standard_normal((m.ne, d.Nst))
    zeroF = torch.zeros(m.nf * 3 * d.Nst, dtype=torch.float64, device="cuda")
    V = gs.velocity_update(zeroF, torch.from_numpy(dp.ravel()).cuda())
    U = gs.velocity_moments(V).cpu().numpy().reshape(m.nf, 2, 3, d.Nst)
    Vo = ops.velocity_update(d, np.zeros((m.nf, 3, d.Nst)), dp, np.zeros((m.nf, 3, d.Nst)))
    Uo = np.zeros_like(U)
    for j in range(m.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            Uo[j, s] = (fb["Mij"][s] @ Vo[j].T).T
    assert rel(U, Uo) <= 1e-12
    b = gs.pressure_rhs(V, pinned=False).cpu().numpy()
    bo = ops.pressure_rhs(d, Vo, pinned=False).ravel()
    assert rel(b, bo) <= 1e-12
    Ad = ops.pressure_apply(d, dp, pinned=False).ravel()
    assert rel(b, -Ad) <= 1e-11


@pytest.mark.parametrize("n,p,pt,method", [(n, p, pt, m) for (n, p, pt) in [(3, 1, 0), (2, 2, 1), (2, 3, 1)]
                                            for m in ["kron_cg", "gmres"]] + [(3, 1, 0, "cg"), (3, 2, 0, "cg")])
def test_solve_matches_direct(n, p, pt, method):
    """The paper's solvers (GMRES; CG on -A for p_t = 0, Cor. 1-2) and the Kronecker-decoupled CG
    against the oracle's sparse-direct solution of the same pinned system."""
    from scipy.sparse.linalg import spsolve
    gs, d = setup(n, p, pt, restart=50, max_iters=50000)
    b = np.random.default_rng(3).standard_normal((d.mesh.ne, d.Nst))
    b[0, ops.pin_index(d)] = 0.0
    tol = 1e-12
    x, st = gs.solve(torch.from_numpy(b.ravel()).cuda(), tol=tol, method=method)
    x = x.cpu().numpy()
    A = ops.pressure_sparse(d)
    assert np.linalg.norm(b.ravel() - A @ x) <= 2 * tol * np.linalg.norm(b)
    assert st["rel_residual"] <= 2 * tol
    xd = spsolve(A.tocsc(), b.ravel())
    cond = np.linalg.cond(A.toarray()) if A.shape[0] <= 3000 else 1e8
    assert np.linalg.norm(x - xd) <= 10 * cond * tol * np.linalg.norm(xd)


def test_cg_rejects_pt_positive():
    import paper_1601_07384_gb300 as g
    gs, d = setup(2, 1, 1)
    b = torch.zeros(d.mesh.ne * d.Nst, dtype=torch.float64, device="cuda"); b[5] = 1.0
    with pytest.raises(g.StdgError, match="EINVAL"):
        gs.solve(b, method="cg")


@pytest.mark.parametrize("p,pt,npic", [(1, 0, 2), (2, 1, 2)])
@pytest.mark.parametrize("precision", ["fp64", "df32", "mixed_f32"])
def test_step_matches_oracle(p, pt, npic, precision):
    """One full Picard pressure-correction step (Sec. 2.6) on Beltrami data; df32 runs the
    pressure and viscous operators on the binary64-accurate pair kernel."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(2, p, pt, dt=0.01, precision=precision)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    st = gs.step(prm.nu, npic, method="kron_cg", tol=1e-13)
    P, V, t = gs.get_state()
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    # initial projection agrees (through basis-independent moments)
    so1 = time_step(d, so, prm.nu, npic, lambda x, tt: beltrami_velocity(x, tt, prm), tol=1e-13, method="direct")
    assert abs(t - 0.01) < 1e-15
    assert rel(P.cpu().numpy(), so1.P.ravel()) <= STEP_TOL
    U = gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)
    Uo = np.zeros_like(U)
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            Uo[j, s] = (fb["Mij"][s] @ so1.V[j].T).T
    assert rel(U, Uo) <= 1e-10
    assert st["max_divergence"] <= 1e-11


@pytest.mark.parametrize("theta", [0.5, 0.75])
def test_theta_steps_match_oracle(theta):
    """Two steps of the semi-implicit theta variant (Sec. 2.7, Eq. CS_16_theta) at p_t = 0: the
    second step starts from a nonzero p^n, so the (1 - theta) p^n part of Lambda is exercised."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(2, 2, 0, dt=0.01)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_theta(theta)
    vbc = lambda x, tt: beltrami_velocity(x, tt, prm)
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    for _ in range(2):
        gs.step(prm.nu, 2, method="kron_cg", tol=1e-13)
        so = time_step(d, so, prm.nu, 2, vbc, tol=1e-13, method="direct", theta=theta)
    P, V, t = gs.get_state()
    assert rel(P.cpu().numpy(), so.P.ravel()) <= STEP_TOL
    U = gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)
    Uo = np.zeros_like(U)
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            Uo[j, s] = (fb["Mij"][s] @ so.V[j].T).T
    assert rel(U, Uo) <= 1e-10


def test_theta_rejected_for_space_time_pressure():
    import paper_1601_07384_gb300 as g
    gs, _ = setup(2, 1, 1)
    with pytest.raises(g.StdgError, match="EINVAL"):
        gs.set_theta(0.5)
    gs0, _ = setup(2, 1, 0)
    with pytest.raises(g.StdgError, match="EINVAL"):
        gs0.set_theta(0.3)
    gs0.set_theta(1.0)


def test_initial_projection_matches_oracle():
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(2, 3, 1, dt=0.01)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    _, V, _ = gs.get_state()
    U = gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)
    Vo = ops.project_initial(d, lambda x: beltrami_velocity(x, 0.0, prm))
    Uo = np.zeros_like(U)
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s in range(len(fb["sides"])):
            Uo[j, s] = (fb["Mij"][s] @ Vo[j].T).T
    assert rel(U, Uo) <= 1e-12


def _oracle_rows(om, d, x, rows):
    """Rows of the unpinned A x computed one by one from the literal space-time blocks:
    gradient, M_j^-1, divergence per interior dual cell of each sampled tet (Eq. CS_19)."""
    out = []
    for i in rows:
        yi = np.zeros(d.Nst)
        for f in range(4):
            j = om.t2f[i, f]
            if not om.interior[j]:
                continue
            fb = d.face_blocks(j)
            s = fb["sides"].index(i)
            l, r = fb["sides"]
            for c in range(3):
                gg = np.linalg.solve(fb["M"], fb["Q"][0][c] @ x[l] + fb["Q"][1][c] @ x[r])
                yi += fb["D"][s][c] @ gg
        out.append(yi)
    return out


def test_large_mesh_sampled_rows():
    """The workload of the timed benchmark (24^3 hexes x 6 = 82,944 tets, p = 3, p_t = 1):
    sampled rows of A x computed one by one by the oracle, for the FP64 operator, the
    binary32-pair operator (both to 1e-12) and the binary32 operator (to 4e-6)."""
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(24, seed=0)
    om = Mesh(v, t)
    d = SpaceTimeDG(om, 3, 1, 0.005)
    x = np.random.default_rng(11).standard_normal((om.ne, d.Nst))
    rows = np.random.default_rng(12).choice(om.ne, 12, replace=False)
    expect = _oracle_rows(om, d, x, rows)
    xd = torch.from_numpy(x.ravel()).cuda()
    for prec, tol in (("fp64", 1e-12), ("df32", 1e-12), ("mixed_f32", 4e-6)):
        gs = g.Solver(g.Mesh(v, t), g.Reference(3, 1), 0.005, precision=prec)
        if prec == "mixed_f32":
            y = gs.pressure_apply_f32(xd.float(), pinned=False).double().cpu().numpy()
        else:
            y = gs.pressure_apply(xd, pinned=False).cpu().numpy()
        y = y.reshape(om.ne, d.Nst)
        for i, yi in zip(rows, expect):
            assert rel(y[i], yi) <= tol, (prec, i)
        del gs


def test_largest_mesh_sampled_rows():
    """The largest configuration (40^3 hexes x 6 = 384,000 tets, p = 4, p_t = 4: 67.2 M pressure
    unknowns, ~84 GB of blocks on the device): sampled rows of the FP64 and binary32-pair
    operators against the oracle, one row at a time."""
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(40, seed=0)
    om = Mesh(v, t)
    d = SpaceTimeDG(om, 4, 4, 0.01)
    x = np.random.default_rng(21).standard_normal((om.ne, d.Nst))
    rows = np.concatenate([[0, om.ne - 1], np.random.default_rng(22).choice(om.ne, 6, replace=False)])
    expect = _oracle_rows(om, d, x, rows)
    xd = torch.from_numpy(x.ravel()).cuda()
    for prec, tol in (("fp64", 1e-12), ("df32", 1e-12), ("mixed_f32", 4e-6)):
        gs = g.Solver(g.Mesh(v, t), g.Reference(4, 4), 0.01, precision=prec)
        if prec == "mixed_f32":       # the binary32 kernel of the inner iterations (N = 35: split rows)
            y = gs.pressure_apply_f32(xd.float(), pinned=False).double().cpu().numpy().reshape(om.ne, d.Nst)
        else:
            y = gs.pressure_apply(xd, pinned=False).cpu().numpy().reshape(om.ne, d.Nst)
        for i, yi in zip(rows, expect):
            assert rel(y[i], yi) <= tol, (prec, i)
        del gs
        torch.cuda.empty_cache()


def test_largest_configuration_step_properties():
    """One time step of the largest configuration as the benchmark runs it (40^3 x 6 = 384,000 tets,
    p = p_t = 4, the solenoidal field with no-slip walls, nu = 1e-3, dt = 0.01, 3 Picard iterations,
    KRON_MG in mixed precision to 1e-10), checked through properties that hold at any size: every
    pressure solve's true residual (binary64 operator) meets the tolerance, the discrete divergence
    (Eq. CS_15) of the new velocity vanishes to rounding against the velocity's size, the state is
    finite and the kinetic-energy proxy does not grow (no forcing, walls at rest)."""
    import paper_1601_07384_gb300 as g
    from inputs import SolenoidalModes
    v, t = kuhn_mesh(40, seed=0)
    gs = g.Solver(g.Mesh(v, t), g.Reference(4, 4), 0.01, precision="mixed_f32")
    sm = SolenoidalModes(seed=1)
    gs.set_initial(g.curl_modes(sm.k, sm.a, sm.phi, sm.scale))
    gs.set_boundary(g.zero())
    _, V0, _ = gs.get_state()
    e0 = float(torch.linalg.norm(V0))
    st = gs.step(1e-3, 3, method="kron_mg", tol=1e-10)
    P, V, tt = gs.get_state()
    assert abs(tt - 0.01) < 1e-15
    assert max(st["press_residual"]) <= 1e-10
    assert torch.isfinite(P).all() and torch.isfinite(V).all()
    vmax = float(V.abs().max())
    assert st["max_divergence"] <= 1e-12 * vmax
    assert float(torch.linalg.norm(V)) <= 1.001 * e0
    del gs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,p,pt", [(3, 1, 0), (2, 2, 1), (2, 3, 1), (2, 4, 2)])
@pytest.mark.parametrize("prec,tol", [("mixed_f32", 4e-6), ("mixed_bf16", 5e-2)])
def test_lowprec_operator_matches_oracle(n, p, pt, prec, tol):
    """Binary32 / bfloat16 blocks with binary32 accumulation (warp-per-tet kernel): error bounded
    by the storage precision of the blocks (2^-24 / 2^-9 relative per entry)."""
    gs, d = setup(n, p, pt, precision=prec)
    x = np.random.default_rng(5).standard_normal(d.mesh.ne * d.Nst)
    y = gs.pressure_apply_f32(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    yo = ops.pressure_apply(d, x.astype(np.float32).astype(np.float64)).ravel()
    assert rel(y, yo) <= tol


@pytest.mark.parametrize("n,p,pt", [(3, 1, 0), (2, 2, 1), (2, 3, 1), (2, 4, 2), (9, 1, 0)])
@pytest.mark.parametrize("prec", ["fp64", "df32", "mixed_f32"])
@pytest.mark.parametrize("method", ["kron_pcg", "kron_mg"])
def test_preconditioned_and_mixed_solves_match_direct(n, p, pt, prec, method):
    """Block-Jacobi Kronecker CG (with or without the agglomeration coarse correction), in FP64 or as
    FP64 iterative refinement around a binary32 inner solve: same FP64 residual tolerance, same
    solution.  n = 9 gives the coarse correction several levels with partly filled cells."""
    from scipy.sparse.linalg import spsolve
    gs, d = setup(n, p, pt, precision=prec, max_iters=50000)
    b = np.random.default_rng(9).standard_normal((d.mesh.ne, d.Nst))
    b[0, ops.pin_index(d)] = 0.0
    tol = 1e-11
    x, st = gs.solve(torch.from_numpy(b.ravel()).cuda(), tol=tol, method=method)
    x = x.cpu().numpy()
    A = ops.pressure_sparse(d)
    assert np.linalg.norm(b.ravel() - A @ x) <= 2 * tol * np.linalg.norm(b)
    xd = spsolve(A.tocsc(), b.ravel())
    assert np.linalg.norm(x - xd) <= 1e-5 * np.linalg.norm(xd)


@pytest.mark.parametrize("prec", ["fp64", "mixed_f32"])
def test_coarse_correction_cuts_iterations(prec):
    """Block Jacobi leaves the smooth error between tets, so its CG needs O(1/h) iterations; the
    constant-mode coarse correction removes it.  On 4,374 tets (p = 2) it needs under half the
    iterations and reaches the same residual."""
    gs, d = setup(9, 2, 0, precision=prec, max_iters=50000, graph_batch=1)
    b = np.random.default_rng(4).standard_normal((d.mesh.ne, d.Nst))
    b[0, ops.pin_index(d)] = 0.0
    bt = torch.from_numpy(b.ravel()).cuda()
    _, s1 = gs.solve(bt, tol=1e-10, method="kron_pcg")
    x, s2 = gs.solve(bt, tol=1e-10, method="kron_mg")
    assert s1["rel_residual"] <= 1e-10 and s2["rel_residual"] <= 1e-10
    assert s2["iterations"] <= 0.5 * s1["iterations"], (s1["iterations"], s2["iterations"])


@pytest.mark.parametrize("precision", ["fp64", "mixed_f32"])
def test_step_with_coarse_correction_matches_oracle(precision):
    """A full Picard step whose pressure solves use the coarse-corrected block CG."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(2, 2, 1, dt=0.01, precision=precision)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    st = gs.step(prm.nu, 2, method="kron_mg", tol=1e-13)
    P, V, _ = gs.get_state()
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    so1 = time_step(d, so, prm.nu, 2, lambda x, tt: beltrami_velocity(x, tt, prm), tol=1e-13, method="direct")
    assert rel(P.cpu().numpy(), so1.P.ravel()) <= STEP_TOL
    U = gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)
    Uo = np.zeros_like(U)
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s_ in range(len(fb["sides"])):
            Uo[j, s_] = (fb["Mij"][s_] @ so1.V[j].T).T
    assert rel(U, Uo) <= 1e-10
    assert st["max_divergence"] <= 1e-11


def test_bf16_inner_solve_still_reaches_fp64_tolerance():
    """bfloat16 blocks make a poor inner preconditioner (cond(A) * 2^-9 >> 1), but the binary64
    outer flexible CG owns the residual: the solve reaches 1e-11 and agrees with the direct solve."""
    import paper_1601_07384_gb300 as g
    gs, d = setup(2, 2, 1, precision="mixed_bf16", max_iters=50000)
    b = np.random.default_rng(9).standard_normal((d.mesh.ne, d.Nst))
    b[0, ops.pin_index(d)] = 0.0
    x, st = gs.solve(torch.from_numpy(b.ravel()).cuda(), tol=1e-11, method="kron_pcg")
    A = ops.pressure_sparse(d)
    assert np.linalg.norm(b.ravel() - A @ x.cpu().numpy()) <= 2e-11 * np.linalg.norm(b)
    assert st["rel_residual"] <= 1e-11


@pytest.mark.parametrize("n,p,pt", CASES)
@pytest.mark.parametrize("pinned", [True, False])
def test_df32_operator_matches_oracle(n, p, pt, pinned):
    """FP64-accurate operator from binary32 pairs (warp-per-tet kernel): 1e-12 like FP64."""
    gs, d = setup(n, p, pt, precision="df32")
    x = np.random.default_rng(n + 10 * p + pt).standard_normal(d.mesh.ne * d.Nst)
    y = gs.pressure_apply(torch.from_numpy(x).cuda(), pinned=pinned).cpu().numpy()
    yo = ops.pressure_apply(d, x, pinned=pinned).ravel()
    assert rel(y, yo) <= 1e-12


@pytest.mark.parametrize("batch", [1, 8])
def test_graph_batched_cg_matches_unbatched(batch):
    """Graph-batched block CG (B iterations per launch) returns a solution meeting the tolerance;
    iteration counts are multiples of B."""
    gs, d = setup(2, 3, 1, graph_batch=batch)
    b = np.random.default_rng(2).standard_normal((d.mesh.ne, d.Nst))
    b[0, ops.pin_index(d)] = 0.0
    x, st = gs.solve(torch.from_numpy(b.ravel()).cuda(), tol=1e-11, method="kron_pcg")
    A = ops.pressure_sparse(d)
    assert np.linalg.norm(b.ravel() - A @ x.cpu().numpy()) <= 2e-11 * np.linalg.norm(b)
    assert st["iterations"] % batch == 0


def test_step_with_previous_viscous_solvers():
    """STDG_VISC_SOLVER=gmres selects the previous viscous solvers (CG for p_t = 0, GMRES(20)
    right-preconditioned by the exact tet-diagonal blocks otherwise); the variable is read once per
    process, so the FP64 step-parity tests run again in a subprocess with it set."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, STDG_VISC_SOLVER="gmres")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(root, "tests", "test_gpu_parity.py"), "-q",
                        "-m", "gpu", "-k", "test_step_matches_oracle and not benchmarked and fp64"],
                       capture_output=True, text=True, timeout=900, cwd=root, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert "2 passed" in r.stdout


@pytest.mark.parametrize("kernel", ["tma", "warp"])
@pytest.mark.parametrize("p,pt", [(3, 1), (4, 4)])
@pytest.mark.parametrize("prec,tol", [("mixed_f32", 4e-6), ("df32", 1e-12)])
def test_alternative_operator_kernels_match_oracle(kernel, p, pt, prec, tol, monkeypatch):
    """STDG_OP_KERNEL selects the operator kernels kept for comparison with the default ones: "warp"
    (one warp per staged tet, also for the pair policy at N = 35) and "tma" (block-staged TMA
    kernels).  The same operator (Eq. CS_19) to the same tolerances as the default kernels, at
    the benchmarked degrees; the pinned solver of the pressure system, so the pin rows are covered."""
    monkeypatch.setenv("STDG_OP_KERNEL", kernel)
    gs, d = setup(2, p, pt, precision=prec)
    x = np.random.default_rng(6).standard_normal(d.mesh.ne * d.Nst)
    if prec == "mixed_f32":
        y = gs.pressure_apply_f32(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
        yo = ops.pressure_apply(d, x.astype(np.float32).astype(np.float64)).ravel()
    else:
        y = gs.pressure_apply(torch.from_numpy(x).cuda()).cpu().numpy()
        yo = ops.pressure_apply(d, x).ravel()
    assert rel(y, yo) <= tol


# ------------------------------------------------------------------ steps at the benchmarked degrees
def _moments(gs, d, V):
    return gs.velocity_moments(V).cpu().numpy().reshape(d.mesh.nf, 2, 3, d.Nst)


def _oracle_moments(d, V):
    U = np.zeros((d.mesh.nf, 2, 3, d.Nst))
    for j in range(d.mesh.nf):
        fb = d.face_blocks(j)
        for s_ in range(len(fb["sides"])):
            U[j, s_] = (fb["Mij"][s_] @ V[j].T).T
    return U


@functools.lru_cache(maxsize=None)
def _oracle_beltrami_step(p, pt, npic, nu, dt):
    """The oracle's step from the projected Beltrami field on the 48-tet mesh (sparse LU solves)."""
    v, t = kuhn_mesh(2, seed=0)
    d = SpaceTimeDG(Mesh(v, t), p, pt, dt)
    prm = BeltramiParams(nu=nu)
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    so1 = time_step(d, so, nu, npic, lambda x, tt: beltrami_velocity(x, tt, prm), tol=1e-13, method="direct")
    return d, so1, _oracle_moments(d, so1.V)


@pytest.mark.parametrize("p,pt,npic", [(3, 1, 3), (4, 4, 2)])
@pytest.mark.parametrize("precision,method", [("fp64", "kron_cg"), ("df32", "kron_mg"), ("mixed_f32", "kron_mg"),
                                              ("df32", "kron_pcg")])
def test_step_matches_oracle_at_benchmarked_degrees(p, pt, npic, precision, method):
    """A full Picard step (Sec. 2.6) at the degrees the benchmark runs: p = 3, p_t = 1 (N = 20: the
    <20,2> viscous fast-diagonalisation, the N = 20 binary32 operator and convection) and
    p = p_t = 4 (N = 35, Ng = 5).  Both sides solve to 1e-13; pressure and velocity to 1e-10."""
    import paper_1601_07384_gb300 as g
    nu, dt = 0.1, 0.01
    d, so1, Uo = _oracle_beltrami_step(p, pt, npic, nu, dt)
    prm = BeltramiParams(nu=nu)
    v, t = kuhn_mesh(2, seed=0)
    gs = g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, precision=precision)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    st = gs.step(nu, npic, method=method, tol=1e-13)
    P, V, _ = gs.get_state()
    ep = rel(P.cpu().numpy(), so1.P.ravel())
    ev = rel(_moments(gs, d, V), Uo)
    print(f"p={p} pt={pt} {precision}/{method}: pressure {ep:.2e} velocity {ev:.2e} iters {st['press_iters']}")
    assert ep <= STEP_TOL and ev <= STEP_TOL
    # the solvers stop on their recurrence residual; the true residual of the returned x (reported)
    # stays within a small multiple of it at this tolerance, 3e-12 measured
    assert max(st["press_residual"]) <= 1e-11


@pytest.mark.parametrize("p,pt,npic", [(3, 1, 3), (4, 4, 2)])
@pytest.mark.parametrize("inner64", [False, True])
def test_mixed_viscous_inner_solves_match_oracle(p, pt, npic, inner64, monkeypatch):
    """The mixed-precision viscous solves (binary64 refinement around inner COCG solves of the
    time-decoupled systems of Eq. A1_mod) with binary32 inner vectors (default) and with binary64
    inner vectors (STDG_VISC_INNER64=1): the step matches the oracle's to 1e-10 either way, and the
    viscous solves reach their binary64 tolerance."""
    import paper_1601_07384_gb300 as g
    if inner64:
        monkeypatch.setenv("STDG_VISC_INNER64", "1")
    nu, dt = 0.1, 0.01
    d, so1, Uo = _oracle_beltrami_step(p, pt, npic, nu, dt)
    prm = BeltramiParams(nu=nu)
    v, t = kuhn_mesh(2, seed=0)
    gs = g.Solver(g.Mesh(v, t), g.Reference(p, pt), dt, precision="mixed_f32")
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    st = gs.step(nu, npic, method="kron_mg", tol=1e-13)
    P, V, _ = gs.get_state()
    ep = rel(P.cpu().numpy(), so1.P.ravel())
    ev = rel(_moments(gs, d, V), Uo)
    print(f"p={p} pt={pt} inner64={inner64}: pressure {ep:.2e} velocity {ev:.2e} visc iters {st['visc_iters']}")
    assert ep <= STEP_TOL and ev <= STEP_TOL


@pytest.mark.parametrize("p,pt", [(3, 1), (4, 4), (2, 2), (4, 1)])
@pytest.mark.parametrize("kernel", ["default", "generic"])
def test_convection_matches_oracle(p, pt, kernel, monkeypatch):
    """The convective term alone (Eq. convdg: the volume integral of grad(phi~) . v vbar and the
    Rusanov face fluxes, Beltrami Dirichlet data on the boundary faces) for seeded random velocity
    averages, element by element against the oracle's, with the compile-time-degree kernels (the
    default at (p, p_t) = (3, 1) and (4, 4)) and with the runtime-degree kernel
    (STDG_CONV_KERNEL=generic).  Both evaluate every product and sum binary64-accurately."""
    import paper_1601_07384_gb300 as g
    if kernel == "generic":
        monkeypatch.setenv("STDG_CONV_KERNEL", "generic")
    nu, dt = 0.1, 0.01
    prm = BeltramiParams(nu=nu)
    gs, d = setup(2, p, pt, dt=dt)
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    ne, Nst = d.mesh.ne, d.Nst
    vbar = np.random.default_rng(17).standard_normal((ne, 3, Nst)) * 0.3
    ups = gs.convection(torch.from_numpy(np.ascontiguousarray(vbar.transpose(1, 0, 2))).cuda())
    ups = ups.cpu().numpy().reshape(3, ne, Nst).transpose(1, 0, 2)
    uo = ops.convection(d, vbar, 0.0, lambda x, tt: beltrami_velocity(x, tt, prm))
    err = rel(ups, uo)
    where = np.unravel_index(np.abs(ups - uo).argmax(), ups.shape)
    print(f"p={p} pt={pt} {kernel}: max rel {err:.2e} at (tet, c, st) = {where}")
    assert err <= 1e-12


@pytest.mark.parametrize("tol,bound", [(1e-13, STEP_TOL), (1e-12, 1e-8)])
def test_tiny_configuration_five_steps(tol, bound):
    """The tiny configuration end to end: 3^3 hexahedra x 6 = 162 jittered tets, p = 1, p_t = 0,
    nu = 0.1, dt = 0.01, 5 steps of 2 Picard iterations, FP64, the paper's CG on the system with the
    pressure pinned at one point, Beltrami data; compared with the oracle (sparse LU) after every step.
    At the configuration's CG tolerance 1e-12 the deviation is bounded by cond * 1e-12; with both
    sides at 1e-13 it meets the 1e-10 step tolerance."""
    import paper_1601_07384_gb300 as g
    prm = BeltramiParams(nu=0.1)
    gs, d = setup(3, 1, 0, dt=0.01)
    gs.set_initial(g.beltrami(prm.a, prm.d, prm.nu))
    gs.set_boundary(g.beltrami(prm.a, prm.d, prm.nu))
    so = initial_state(d, lambda x: beltrami_velocity(x, 0.0, prm))
    vbc = lambda x, tt: beltrami_velocity(x, tt, prm)
    worst = []
    for k in range(5):
        st = gs.step(prm.nu, 2, method="cg", tol=tol)
        so = time_step(d, so, prm.nu, 2, vbc, tol=1e-13, method="direct")
        P, V, t = gs.get_state()
        ep, ev = rel(P.cpu().numpy(), so.P.ravel()), rel(_moments(gs, d, V), _oracle_moments(d, so.V))
        worst.append((ep, ev))
        assert abs(t - so.t) < 1e-14
        assert ep <= bound and ev <= bound, (k, ep, ev)
        assert max(st["press_residual"]) <= tol
    print("per-step (pressure, velocity) deviation:", [f"{a:.1e}/{b:.1e}" for a, b in worst])


@pytest.mark.parametrize("precision", ["mixed_f32", "df32"])
def test_solve_meets_tolerance_in_binary64_at_benchmark_size(precision):
    """The chosen solver at the benchmark workload (82,944 tets, p = 3, p_t = 1): the returned x meets
    ||b - A x|| <= 1e-10 ||b|| with the residual evaluated by the plain binary64 operator kernel (itself
    equal to the oracle's operator to 1e-12), not only by the solver's own recurrence, and the residual
    the solver reports agrees with that evaluation."""
    import paper_1601_07384_gb300 as g
    v, t = kuhn_mesh(24, seed=0)
    mesh, ref = g.Mesh(v, t), g.Reference(3, 1)
    gs = g.Solver(mesh, ref, 0.005, precision=precision)
    g64 = g.Solver(mesh, ref, 0.005, precision="fp64")
    rng = np.random.default_rng(31)
    b = rng.standard_normal(gs.ne * gs.Nst)
    b[[a * gs.N for a in range(gs.Ng)]] = 0.0
    bt = torch.from_numpy(b).cuda()
    x, st = gs.solve(bt, tol=1e-10, method="kron_mg")
    r = bt - g64.pressure_apply(x)
    rel_true = float(torch.linalg.norm(r) / torch.linalg.norm(bt))
    print(f"{precision}: reported {st['rel_residual']:.3e}, binary64 operator {rel_true:.3e}, "
          f"iterations {st['iterations']} (outer {st['restarts']})")
    assert rel_true <= 1e-10
    assert abs(st["rel_residual"] - rel_true) <= 0.1 * rel_true + 1e-13
