#!/usr/bin/env python
"""Benchmark of the staggered space-time DG pressure-correction time step on one GB300.

Workload (default, "big"): unit cube, 40^3 hexahedra x 6 = 384,000 jittered tetrahedra (seed 0),
p = 4, p_t = 4 (N = 35, Nst = 175, 67,200,000 pressure DoFs), initial velocity the seeded solenoidal
field curl(b Psi) (64 Fourier modes drawn from splitmix64(seed 1), amplitude |k|^-3 in Psi, scaled
to |v|max = 0.1) with no-slip walls, nu = 1e-3, dt = 0.01, 3 Picard iterations per step, pressure
and viscous solves to a 1e-10 relative residual.  "mid": 24^3 x 6 = 82,944 tets, p = 3, p_t = 1,
Beltrami data, nu = 0.01, dt = 0.005.  A "step" is one full time step (stdg_step: averaging,
convection, viscous solves, pressure right-hand side, pressure solve, velocity update, n_picard times).

Metric: seconds per time step with the chosen solver (Kronecker-decoupled block CG with the
agglomeration coarse correction, mixed precision by default), next to the plain FP64 solvers (the
paper's GMRES(50), and unpreconditioned Kronecker CG); the dominant operator kernel's achieved
throughput is reported as a roofline (HBM for binary32 blocks, the FP64 pipe or the derived
pair-arithmetic peak for the binary64-accurate kernels).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload big|mid|...]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s/time-step at 1e-10 residual (chosen vs plain FP64 GMRES); matvec HBM GB/s"
WORKLOADS = {
    # the largest single-GPU configuration: p = p_t = 4 on 40^3 x 6 tets, solenoidal data, no-slip walls
    "big": dict(n=40, p=4, pt=4, nu=1e-3, dt=0.01, npic=3, tol=1e-10, restart=50, data="solenoidal",
                restart_every=0, gmres_cap=300, plain_cg_cap=1500, e2e_steps=2),
    "mid": dict(n=24, p=3, pt=1, nu=0.01, dt=0.005, npic=3, tol=1e-10, restart=50, data="beltrami",
                restart_every=6, gmres_cap=5000, plain_cg_cap=20000, e2e_steps=0),
    "tiny": dict(n=3, p=1, pt=0, nu=0.1, dt=0.01, npic=2, tol=1e-12, restart=50, data="beltrami",
                 restart_every=0, gmres_cap=5000, plain_cg_cap=20000, e2e_steps=0),
    "prof": dict(n=16, p=3, pt=1, nu=0.01, dt=0.005, npic=3, tol=1e-10, restart=50, data="beltrami",
                 restart_every=6, gmres_cap=5000, plain_cg_cap=20000, e2e_steps=0),
    "learned": dict(n=6, p=3, pt=1, nu=0.01, dt=0.005, npic=3, tol=1e-10, restart=50, data="beltrami",
                    restart_every=6, gmres_cap=5000, plain_cg_cap=20000, e2e_steps=0),
    "theta": dict(n=24, p=3, pt=0, nu=0.01, dt=0.005, npic=2, tol=1e-10, restart=50, data="beltrami",
                  restart_every=6, gmres_cap=5000, plain_cg_cap=20000, e2e_steps=0),
    # the degrees of the largest configuration (p = p_t = 4, nu = 1e-3, dt = 0.01) on a 12^3 mesh
    "hi": dict(n=12, p=4, pt=4, nu=1e-3, dt=0.01, npic=3, tol=1e-10, restart=50, data="solenoidal",
               restart_every=0, gmres_cap=2000, plain_cg_cap=20000, e2e_steps=0),
}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12      # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz
# binary64-accurate products from binary32 pairs: 12 FP32 lane operations per multiply-add term
# (1 mul, 3 fma, TwoSum 6 adds, 2 adds) on 152 SMs x 128 FP32 lanes x 2070 MHz
DF_OPS_PER_TERM = 12
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / DF_OPS_PER_TERM * 2 / 1e12
COUNTS_FILE = os.path.join(ROOT, "profiles", "bench_operator_counts.json")


def nbasis(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def workload_name(w):
    ne = 6 * w["n"] ** 3
    N = nbasis(w["p"]); Nst = N * (w["pt"] + 1)
    data = ("seeded solenoidal curl(b Psi) data (64 modes, |v|max 0.1), no-slip walls" if w["data"] == "solenoidal"
            else "Beltrami data")
    return (f"Kuhn {w['n']}^3 hex x 6 = {ne:,} tets, p={w['p']}, p_t={w['pt']} ({ne * Nst:,} pressure DoFs), "
            f"{data}, nu={w['nu']}, dt={w['dt']}, {w['npic']} Picard iterations/step, tol {w['tol']:g}")


def set_data(solver, g, w):
    """Initial and Dirichlet velocity of the workload (device field kinds)."""
    if w["data"] == "solenoidal":
        from inputs import SolenoidalModes
        sm = SolenoidalModes(seed=1)
        solver.set_initial(g.curl_modes(sm.k, sm.a, sm.phi, sm.scale))
        solver.set_boundary(g.zero())
    else:
        fld = g.beltrami(np.pi / 4, np.pi / 2, w["nu"])
        solver.set_initial(fld)
        solver.set_boundary(fld)


def mesh_counts(n):
    ne = 6 * n ** 3; nb = 12 * n * n
    return ne, (4 * ne - nb) // 2, nb


def operator_cost(w, entry_bytes=8, vec_bytes=8):
    """Algorithmic bytes and flops of one five-point operator application (assembled form:
    symmetric diagonal blocks counted packed, every off-diagonal block once, x read once, y
    written once; flops = 2 Ng per applied block entry)."""
    ne, nint, _ = mesh_counts(w["n"])
    N = nbasis(w["p"]); Ng = w["pt"] + 1
    entries = ne * N * (N + 1) // 2 + nint * N * N
    bytes_alg = entry_bytes * entries + 2 * vec_bytes * ne * N * Ng
    flops = 2 * Ng * (ne * N * N + 2 * nint * N * N)
    return bytes_alg, flops


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, dev):
        self.dev, self.lines, self.proc = dev, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_operator_sample(w, reps=3, n_sample=3):
    """The oracle's matrix-free pressure operator (as it stands) on a small mesh of the same
    family, degrees and time step: seconds per application on that mesh, and its interior faces."""
    from inputs import kuhn_mesh
    from oracle import operators as ops
    from oracle.blocks import SpaceTimeDG
    from oracle.mesh import Mesh
    v, t = kuhn_mesh(n_sample, seed=0)
    d = SpaceTimeDG(Mesh(v, t), w["p"], w["pt"], w["dt"])
    for j in range(d.mesh.nf):
        d.face_blocks(j)                                       # precompute (untimed)
    x = np.random.default_rng(0).standard_normal((d.mesh.ne, d.Nst))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        ops.pressure_apply(d, x)
        times.append(time.perf_counter() - t0)
    return float(np.median(times)), int(d.mesh.interior.sum())


_ORACLE = {}


def _oracle_init(w, n_sample):
    """Pool initializer: the oracle's discretisation of the sample mesh, blocks precomputed (untimed)."""
    from inputs import kuhn_mesh
    from oracle.blocks import SpaceTimeDG
    from oracle.mesh import Mesh
    v, t = kuhn_mesh(n_sample, seed=0)
    d = SpaceTimeDG(Mesh(v, t), w["p"], w["pt"], w["dt"])
    for j in range(d.mesh.nf):
        d.face_blocks(j)
    _ORACLE["d"] = d
    _ORACLE["x"] = np.random.default_rng(0).standard_normal((d.mesh.ne, d.Nst))


def _oracle_apply(_):
    from oracle import operators as ops
    t0 = time.perf_counter()
    ops.pressure_apply(_ORACLE["d"], _ORACLE["x"])
    return time.perf_counter() - t0, int(_ORACLE["d"].mesh.interior.sum())


class OracleOnHostCores:
    """The oracle's operator sample run at once in one process per host core (spawned, one BLAS
    thread each): every process applies the operator to its own copy of the sample mesh, so the
    host's throughput is `cores` applications per per-process time.  sample() returns seconds per
    application of the full mesh on all cores (extrapolated by interior faces), and the sample's
    interior faces."""

    def __init__(self, w, n_sample=3, cores=None):
        import multiprocessing as mp
        self.w = w
        self.cores = cores or os.cpu_count() or 1
        os.environ["OMP_NUM_THREADS"] = "1"
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(w, n_sample))

    def sample(self):
        res = self.pool.map(_oracle_apply, range(self.cores), chunksize=1)
        t_app = float(np.median([r[0] for r in res]))
        nint_s = res[0][1]
        _, nint, _ = mesh_counts(self.w["n"])
        return t_app * nint / nint_s / self.cores, nint_s

    def close(self):
        self.pool.close()
        self.pool.join()


def operator_alone_ms(solver, lowprec, reps):
    """Average duration of one pressure-operator launch, CUDA events on the solver's stream: the
    binary32 / bfloat16 kernel of the inner iterations if lowprec, else the binary64-accurate one."""
    import torch
    x = torch.randn(solver.ne * solver.Nst, dtype=torch.float64, device="cuda")
    xf = x.float()
    y = torch.empty_like(x)
    yf = torch.empty_like(xf)
    run = (lambda: solver.pressure_apply_f32(xf, yf)) if lowprec else \
        (lambda: solver.pressure_apply(x, y))
    run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(solver.stream)
    for _ in range(reps):
        run()
    e1.record(solver.stream)
    torch.cuda.synchronize()
    del x, xf, y, yf
    return e0.elapsed_time(e1) / reps


def job_seconds_per_step(ms, steps, world, device="cuda"):
    """Whole-job time of the timed region: the maximum over ranks of each rank's `ms`, and the
    seconds per step it implies when every rank (a replica) runs `steps` steps of the same workload
    (steps * world steps in that time).  Collective only when world > 1."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, ms_max / 1e3 / (steps * world)


def cpu_baseline_line(host, w, ops_per_step):
    s_op, nint_s = host.sample()
    cores = host.cores
    return {"value": s_op * ops_per_step, "unit": "s/step", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": (f"extrapolated: the oracle's matrix-free pressure operator (FP64, as it stands) applied on "
                       f"the {nint_s}-interior-face 3^3 mesh of the same family/p/p_t, once in each of {cores} "
                       f"processes on {cores} host cores at once; per-application time scaled to "
                       f"{mesh_counts(w['n'])[1]:,} interior faces, divided by {cores} cores, times "
                       f"{ops_per_step:.0f} operator applications per step (the GPU arm's count); "
                       f"the other per-step work is not included")}


def reference_arm(args, w, world, rank):
    if rank != 0:
        return
    counts = json.load(open(COUNTS_FILE)) if os.path.exists(COUNTS_FILE) else {}
    entry = counts.get(workload_name(w)) if isinstance(counts, dict) else None
    if entry is None:
        print(json.dumps({"impl": "reference", "unavailable": "no operator-application count recorded for this "
                          "workload (profiles/bench_operator_counts.json)"}))
        return
    per_step_ops = entry["operator_applications_per_step"]
    host = OracleOnHostCores(w)
    for _ in range(args.warmup):
        host.sample()
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        line = cpu_baseline_line(host, w, per_step_ops)
        vals.append(line["value"])
    wall = time.perf_counter() - t_all
    host.close()
    v = float(np.median(vals))
    line["value"] = v
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "s/step", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
                      "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": workload_name(w), "parallelism": "replicas"},
                      "cpu_baseline": line,
                      "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                      "wall_s": wall}))


def learned_protocol(args, g, torch):
    """The learned-preconditioner protocol (32^3 hexahedra x 6 = 196,608 tets, p = 3, p_t = 1, the
    seeded solenoidal field with no-slip walls, a sweep over nu in {1e-2, 3e-3, 1e-3}): for each nu,
    `train_steps` steps of the chosen solver
    (KRON_MG, mixed precision) from the initial state, harvesting (residual, missed error) pairs from
    the outer iterations of its pressure solves at evenly spaced steps; then one network (3 message-
    passing layers, hidden 64, bfloat16 weights on the tensor cores) trained on the pairs of all three;
    then for each nu, from the state after its training steps, `eval_steps` steps with KRON_MG and the
    same steps with KRON_MG_GNN (every inner-solve step of the outer flexible iteration followed by a
    step along the network's direction), with pressure iterations, s/step and fallbacks.  The
    configuration names neither data nor time step: Beltrami data diverges within ~100 steps on this
    mesh even at dt = 0.001, so the stable no-slip field of the largest configuration is used, with
    its dt = 0.01 (convective CFL number of the DG scheme about 0.2)."""
    from inputs import kuhn_mesh
    from inputs import SolenoidalModes
    n, p, pt, dt, npic, tol = args.learned_n, 3, 1, args.learned_dt, 3, 1e-10
    sm = SolenoidalModes(seed=1)
    init, wall = g.curl_modes(sm.k, sm.a, sm.phi, sm.scale), g.zero()
    nus = [1e-2, 3e-3, 1e-3]
    T, E = args.train_steps, args.eval_steps
    v, t = kuhn_mesh(n, seed=0)
    mesh, ref = g.Mesh(v, t), g.Reference(p, pt)
    s = g.Solver(mesh, ref, dt, precision="mixed_f32")
    s.gnn_init(hidden=64, layers=3, bf16=True, seed=0)
    per_nu, marks = args.learned_pairs // len(nus), max(T // 8, 1)
    states, t_train_steps = {}, []
    for nu in nus:
        s.set_initial(init); s.set_boundary(wall)
        for k in range(T):
            harvest = k % marks == 0
            s.gnn_autoharvest_mg(2 if harvest else 0, args.learned_pairs)
            torch.cuda.synchronize(); a = time.perf_counter()
            s.step(nu, npic, method="kron_mg", tol=tol)
            torch.cuda.synchronize(); t_train_steps.append(time.perf_counter() - a)
        s.gnn_autoharvest_mg(0, args.learned_pairs)
        P, V, tt = s.get_state()
        states[nu] = (P.cpu(), V.cpu(), tt)
    torch.cuda.synchronize()
    a = time.perf_counter()
    l0, l1 = s.gnn_train(epochs=args.learned_epochs, lr=2e-3, batch=4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - a
    res = {}
    for nu in nus:
        res[str(nu)] = {}
        for method in ["kron_mg", "kron_mg_gnn"]:
            P, V, tt = states[nu]
            s.set_state(P.cuda(), V.cuda(), tt)
            its, secs, fb = [], [], 0
            for _ in range(E):
                torch.cuda.synchronize(); a = time.perf_counter()
                st = s.step(nu, npic, method=method, tol=tol)
                torch.cuda.synchronize(); secs.append(time.perf_counter() - a)
                its.append(st["press_iters"]); fb += st["fallbacks"]
            inner = [sum(x) for x in its]
            res[str(nu)][method] = {"s_per_step": float(np.median(secs)), "inner_iters_per_step_mean": float(np.mean(inner)),
                                    "press_iters_first_last": [its[0], its[-1]], "skipped_network_steps": fb}
        b, l = res[str(nu)]["kron_mg"], res[str(nu)]["kron_mg_gnn"]
        res[str(nu)]["iteration_ratio"] = l["inner_iters_per_step_mean"] / b["inner_iters_per_step_mean"]
        res[str(nu)]["time_ratio"] = l["s_per_step"] / b["s_per_step"]
    print(json.dumps({"learned_preconditioner": {
        "workload": f"Kuhn {n}^3 hex x 6 = {6 * n ** 3:,} tets, p={p}, p_t={pt}, seeded solenoidal curl(b Psi) data, "
                    f"no-slip walls, dt={dt}, nu in {nus}",
        "train_steps_per_nu": T, "eval_steps_per_nu": E, "pairs": args.learned_pairs,
        "train_loss_first_last": [l0, l1], "train_seconds": t_train, "epochs": args.learned_epochs,
        "train_phase_s_per_step_median": float(np.median(t_train_steps)),
        "network": "3 message-passing layers, hidden 64, bf16 weights, dense products on tcgen05 tensor cores; "
                   "its direction taken as an extra step of the binary64 flexible outer CG of KRON_MG",
        "results": res}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="big", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end arm (0: the workload's default, else --steps)")
    ap.add_argument("--gmres-max-iters", type=int, default=0,
                    help="iteration cap per pressure solve of the plain FP64 GMRES(50) arm (0: workload default)")
    ap.add_argument("--plain-cg-max-iters", type=int, default=0,
                    help="iteration cap per pressure solve of the plain FP64 Kronecker CG arm (0: workload default)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 comparison arms (mixed vs FP64 step error, plain GMRES, plain CG)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--counts-out", default="",
                    help="merge this run's operator applications per step into this JSON file "
                         "(profiles/bench_operator_counts.json is the copy the reference arm reads)")
    ap.add_argument("--precision", default="mixed_f32", choices=["fp64", "df32", "mixed_f32", "mixed_bf16"])
    ap.add_argument("--solver", default="kron_mg", choices=["kron_cg", "kron_pcg", "kron_mg", "gmres"])
    ap.add_argument("--theta", type=float, default=1.0,
                    help="semi-implicit pressure weight (p_t = 0 workloads only; 1 = fully implicit)")
    ap.add_argument("--dt", type=float, default=0.0, help="override the workload's time step (labelled)")
    ap.add_argument("--learned", action="store_true",
                    help="learned-preconditioner protocol: harvest + train on early steps, evaluate later steps")
    ap.add_argument("--learned-n", type=int, default=32, help="hexahedra per direction of the protocol's mesh")
    ap.add_argument("--learned-dt", type=float, default=0.01)
    ap.add_argument("--train-steps", type=int, default=100)
    ap.add_argument("--eval-steps", type=int, default=100)
    ap.add_argument("--learned-pairs", type=int, default=48)
    ap.add_argument("--learned-epochs", type=int, default=200)
    ap.add_argument("--graph-batch", type=int, default=8,
                    help="Krylov iterations per captured CUDA graph (1: no graphs, e.g. for kernel-level profiling)")
    ap.add_argument("--peak-probe", action="store_true",
                    help="measure the binary64 / binary32 FMA throughput of the device (stdg_fma_probe) and exit")
    ap.add_argument("--op-only", type=int, default=0,
                    help="only build the workload and apply the pressure operator this many times (profiling)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.dt > 0:
        w["dt"] = args.dt
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, w, world, rank)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_1601_07384_gb300.build import build
        build()
    if world > 1:
        dist.barrier()
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh

    if args.learned:
        return learned_protocol(args, g, torch)
    if args.peak_probe:
        with ClockSampler(local) as clk:
            f64, f32 = g.fma_probe()
        print(json.dumps({"fma_probe": {"fp64_tflops": f64, "fp32_tflops": f32,
                                        "pair_fp64_equiv_tflops": f32 / DF_OPS_PER_TERM,
                                        "nominal_fp64_tflops": FP64_PEAK_TFLOPS, "clocks": clk.summary()}}))
        return
    t_setup = time.perf_counter()
    v, t = kuhn_mesh(w["n"], seed=0)
    mesh = g.Mesh(v, t)
    ref = g.Reference(w["p"], w["pt"])
    solver = g.Solver(mesh, ref, w["dt"], precision=args.precision, restart=w["restart"], max_iters=200000,
                      graph_batch=args.graph_batch)
    if args.op_only > 0:
        ms = operator_alone_ms(solver, args.precision.startswith("mixed"), args.op_only)
        print(json.dumps({"op_only": args.op_only, "precision": args.precision, "workload": workload_name(w),
                          "avg_launch_ms": ms}))
        return
    set_data(solver, g, w)
    if args.theta != 1.0:
        solver.set_theta(args.theta)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    stream = solver.stream
    # At dt = 0.005 on the 24^3 mesh (convective CFL of the DG scheme about 2) the time stepping is
    # unstable: it stays bounded to t = 0.04 and diverges from step 9 on.  There the configured dt is
    # kept and the run restarts from the initial state every restart_every steps (a device-to-device
    # state copy, inside the timed region when it falls there), so any --steps/--warmup stay in range.
    every = w["restart_every"] if args.dt <= 0 else 0
    S0 = solver.get_state() if every else None
    since = [0]

    def advance():
        if every and since[0] == every:
            solver.set_state(*S0)
            since[0] = 0
        since[0] += 1
        return solver.step(w["nu"], w["npic"], method=args.solver, tol=w["tol"])

    for _ in range(args.warmup):
        advance()
    Pw, Vw, tw = solver.get_state()          # the timed steps' starting state (reused end to end)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K steps with the chosen solver, inputs resident in HBM
    solver.profile(True)
    stats = []
    with ClockSampler(local) as clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(advance())
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    prof = solver.profile_read()
    solver.profile(False)
    # whole job: replicas each run K steps of the same workload; s/step over all steps of all ranks
    ms, s_per_step = job_seconds_per_step(ms, args.steps, world)

    # ---- end to end through the C ABI with host buffers: every step copies its input state from
    # pinned host memory and its result back; each repeats the first timed step (same input state)
    ne2e = args.e2e_steps or w["e2e_steps"] or args.steps
    P0, V0, t0 = solver.get_state()
    Pin = torch.empty(Pw.numel(), dtype=torch.float64).pin_memory(); Pin.copy_(Pw)
    Vin = torch.empty(Vw.numel(), dtype=torch.float64).pin_memory(); Vin.copy_(Vw)
    Ph = torch.empty(P0.numel(), dtype=torch.float64).pin_memory()
    Vh = torch.empty(V0.numel(), dtype=torch.float64).pin_memory()
    del P0, V0
    lib = g._lib.load()
    import ctypes as C
    tcur = C.c_double(tw)
    # one untimed end-to-end iteration first (as the device-timed steps have their warm-up): the
    # first copies from freshly allocated pinned buffers and the first synchronising calls are not
    # steady state
    g._lib.check(lib.stdg_set_state(solver._h, C.c_void_p(Pin.data_ptr()), C.c_void_p(Vin.data_ptr()), 0, tw))
    solver.step(w["nu"], w["npic"], method=args.solver, tol=w["tol"])
    g._lib.check(lib.stdg_get_state(solver._h, C.c_void_p(Ph.data_ptr()), C.c_void_p(Vh.data_ptr()), 0,
                                    C.byref(tcur)))
    barrier()
    te0 = time.perf_counter()
    t_h2d = t_d2h = 0.0                           # the state copies, to separate them from the steps
    for _ in range(ne2e):
        tc0 = time.perf_counter()
        g._lib.check(lib.stdg_set_state(solver._h, C.c_void_p(Pin.data_ptr()), C.c_void_p(Vin.data_ptr()), 0, tw))
        tc1 = time.perf_counter()
        solver.step(w["nu"], w["npic"], method=args.solver, tol=w["tol"])
        tc2 = time.perf_counter()
        g._lib.check(lib.stdg_get_state(solver._h, C.c_void_p(Ph.data_ptr()), C.c_void_p(Vh.data_ptr()), 0,
                                        C.byref(tcur)))
        t_h2d += tc1 - tc0
        t_d2h += time.perf_counter() - tc2
    barrier()
    e2e = (time.perf_counter() - te0) / ne2e

    # ---- roofline of the dominant operator kernel (CUDA-event time of its launches in the timed region)
    kinds = ["fp64 blocks (k_apply)", "binary32-pair blocks (k_apply_warp<WDF>)", "binary32 blocks (k_apply_warp<WF32>)",
             "bfloat16 blocks (k_apply_warp<WBF16>)"]
    kbest = int(np.argmax(prof["kind_ms"]))
    nlaunch_k = max(prof["kind_launches"][kbest], 1)
    op_launch_ms = prof["kind_ms"][kbest] / nlaunch_k
    bytes_alg, flops = operator_cost(w, entry_bytes=[8, 8, 4, 2][kbest], vec_bytes=[8, 8, 4, 4][kbest])
    tflops = flops / (op_launch_ms * 1e-3) / 1e12
    gbs = bytes_alg / (op_launch_ms * 1e-3) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ops_per_step = prof["operator_launches"] / args.steps
    traffic = None
    tf = os.path.join(ROOT, "profiles", "operator_traffic.json")
    if os.path.exists(tf):
        traffic = json.load(open(tf)).get(f"{workload_name(w)}|{kinds[kbest]}")
    if kbest == 0:
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS,
                "peak_note": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz (probe measured 1.20 TFLOP/s)"}
    elif kbest == 1:
        roof = {"bound": "alu", "achieved": tflops, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / DF_PEAK_TFLOPS,
                "peak_note": f"FP64-accurate flops from binary32 pairs: 152 SMs x 128 FP32 lanes x 2070 MHz / "
                             f"{DF_OPS_PER_TERM} lane operations per multiply-add term x 2 flop"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "peak_note": f"HBM copy bandwidth, {hbm_src} (MEASURED_PEAKS.json hbm_gbs); of measured"}
    alone = operator_alone_ms(solver, kbest >= 2, 20)
    roof.update({"traffic": traffic, "kernel": kinds[kbest], "avg_launch_ms": op_launch_ms,
                 "alone_avg_launch_ms": alone,
                 "launches_timed": int(nlaunch_k), "algorithmic_bytes_per_launch": bytes_alg,
                 "flops_per_launch": flops, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                 "fp64_equiv_tflops": tflops})
    mem = {"solver_device_bytes": solver.alloc_stats()[0], "max_allocated_bytes": torch.cuda.max_memory_allocated(),
           "allocator": "PyTorch caching allocator (stdg_solver_create_alloc)"}

    out = {
        "metric": METRIC, "value": s_per_step * 1.0, "unit": "s/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": s_per_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "df32": "f64 (products from fp32 pairs)",
                                       "mixed_f32": "f64 outer (pair products) / f32 inner", "mixed_bf16": "f64 outer (pair products) / bf16 inner"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name(w) + (f", theta={args.theta}" if args.theta != 1.0 else "")
                   + (f" (dt overridden to {w['dt']})" if args.dt > 0 else ""),
                   "steps": (f"restarted from the initial state every {every} steps (t <= {every * w['dt']:g}): at "
                             f"this dt the scheme diverges from step 9; restarts keep every timed step bounded")
                   if every else "consecutive time steps",
                   "solver": args.solver, "precision": args.precision,
                   "parallelism": f"replicas only: {world} independent copies" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (operator blocks + Q per step >> 129 MB)"},
        "roofline": roof,
        "e2e": {"value": e2e, "unit": "s/step", "h2d_bytes_per_step": int(Pin.numel() + Vin.numel()) * 8,
                "d2h_bytes_per_step": int(Ph.numel() + Vh.numel()) * 8, "steps": ne2e, "warmup": 1,
                "h2d_s_per_step": t_h2d / ne2e, "d2h_s_per_step": t_d2h / ne2e},
        "gpu_launches": int(prof["kernel_launches"]),
        "operator_applications_per_step": ops_per_step,
        "press_iters": [s["press_iters"] for s in stats],
        "press_residual_max_per_step": [max(s["press_residual"]) for s in stats],
        "visc_iters": [s["visc_iters"] for s in stats],
        "max_divergence": max(s["max_divergence"] for s in stats),
        "matvecs_per_s": ops_per_step / (ms / 1e3 / args.steps),
        "pressure_dof_updates_per_s": ops_per_step / (ms / 1e3 / args.steps) * solver.ne * solver.Nst,
        "time_breakdown": {"phases_s_per_step": dict(zip(["slab setup", "averaging + Lambda", "convection", "viscous solves",
                                                            "goback + pressure rhs", "pressure solve", "updates"],
                                                           [v / 1e3 / args.steps for v in prof["phase_ms"][:7]])),
                           "operator_s_per_step": prof["operator_ms"] / 1e3 / args.steps,
                           "rest_s_per_step": ms / 1e3 / args.steps - prof["operator_ms"] / 1e3 / args.steps,
                           "operator_kinds": {kinds[k]: {"launches_per_step": prof["kind_launches"][k] / args.steps,
                                                         "ms_per_launch": prof["kind_ms"][k] / max(prof["kind_launches"][k], 1)}
                                              for k in range(4) if prof["kind_launches"][k] > 0}},
        "memory": mem,
        "setup_s": setup_s,
        "clocks": clk.summary(),
    }
    del solver
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # ---- FP64 comparison arms on a binary64 solver (created after the main one is freed: at the largest
    # configuration two solvers do not fit side by side), all from the timed steps' starting state
    if not args.no_compare:
        gcap = args.gmres_max_iters or w["gmres_cap"]
        ccap = args.plain_cg_max_iters or w["plain_cg_cap"]
        f64 = g.Solver(mesh, ref, w["dt"], precision="fp64", restart=w["restart"], max_iters=200000)
        set_data(f64, g, w)
        if args.theta != 1.0:
            f64.set_theta(args.theta)
        cmp = {}

        def run_step(method, cap):
            f64.set_state(Pw, Vw, tw)
            f64.set_max_iters(cap)
            torch.cuda.synchronize()
            a = time.perf_counter()
            try:
                st = f64.step(w["nu"], w["npic"], method=method, tol=w["tol"])
                ok = True
            except g.StdgError as exc:
                st, ok = {"error": str(exc)[:200]}, False
            torch.cuda.synchronize()
            return st, ok, time.perf_counter() - a

        if args.precision.startswith("mixed"):
            # the mixed step's error against a binary64 step from the same state (same solver method)
            st, ok, secs = run_step(args.solver, 200000)
            P64, V64, _ = f64.get_state()
            Pm, Vm = Ph.to("cuda"), Vh.to("cuda")
            cmp["mixed_vs_fp64_step"] = {
                "method": args.solver, "fp64_s_per_step": secs, "converged": ok,
                "p_rel_l2": float(torch.linalg.norm(Pm - P64) / torch.linalg.norm(P64)),
                "v_rel_l2": float(torch.linalg.norm(Vm - V64) / torch.linalg.norm(V64)),
                "note": "one step from the timed steps' starting state; relative L2 norm of the coefficient vectors "
                        "(orthonormal bases); the end-to-end arm's mixed result against the binary64 solver's"}
            del Pm, Vm, P64, V64
        # the paper's plain FP64 solver: GMRES(50) (CG when p_t = 0), capped: a lower bound if it stops
        plain = "cg" if w["pt"] == 0 else "gmres"
        st, ok, secs = run_step(plain, gcap)
        cmp["plain_paper_solver"] = {"method": plain, "max_iters_per_solve": gcap, "converged": ok,
                                     "s_per_step" if ok else "s_until_stopped": secs,
                                     "press_iters": st.get("press_iters"), "stopped": st.get("error")}
        if ok:
            cmp["plain_paper_solver"]["press_residual_max"] = max(st["press_residual"])
        # plain FP64 Kronecker CG (no preconditioner) on the same systems
        if plain != "cg":
            st, ok, secs = run_step("kron_cg", ccap)
            cmp["plain_fp64_kron_cg"] = {"max_iters_per_solve": ccap, "converged": ok,
                                         "s_per_step" if ok else "s_until_stopped": secs,
                                         "press_iters": st.get("press_iters"), "stopped": st.get("error")}
            if ok:
                cmp["plain_fp64_kron_cg"]["press_residual_max"] = max(st["press_residual"])
        out["fp64_comparisons"] = cmp
        del f64
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_cpu_baseline:
        host = OracleOnHostCores(w)
        out["cpu_baseline"] = cpu_baseline_line(host, w, ops_per_step)
        host.close()
    if rank == 0:
        if args.counts_out:                      # the operator count the reference arm scales by
            path = os.path.abspath(args.counts_out)
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cur = json.load(open(path)) if os.path.exists(path) else {}
            if not isinstance(cur, dict) or "workload" in cur:
                cur = {}
            cur[workload_name(w)] = {"operator_applications_per_step": ops_per_step}
            with open(path, "w") as f:
                json.dump(cur, f, indent=1)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
