"""One time step of the staggered space-time pressure-correction scheme (Sec. 2.6).

Step 0: p^{n+1,0} = 0, v^{n+1,0}(x, tau) = v^n(x, tau = 1) (reading R14).
For k = 0 .. n_picard-1 (reading R18):
  1. vbar = average(v^{n+1,k}) (Eq. average), Lambda(p^{n+1,k}) (Eq. prevpress)
  2. Upsilon^c(vbar) (Eq. convdg)
  3. solve Eq. A1_mod for vbar^{n+1,k+1/2}, each velocity component
  4. F = goback(vbar^{n+1,k+1/2}) (Eq. goback)
  5. solve Eq. A2_mod for dp = p^{n+1,k+1} - p^{n+1,k}
  6. v^{n+1,k+1} from Eq. A3_mod
The right-hand side of Eq. A1_mod uses Mbar_i^- vbar_i^n with vbar^n the average of the
previous slab's velocity (reading R15).

Semi-implicit theta variant for p_t = 0 (Sec. 2.7, Eqs. CS_15_theta / CS_16_theta): the momentum
equation of each dual cell sees the pressure only as p^{n+theta} = theta p^{n+1} + (1-theta) p^n,
theta in [1/2, 1].  In the pressure-correction iteration this means (reading R27): Lambda of
step 1 is taken of theta p^{n+1,k} + (1-theta) p^n; the system of step 5 is Eq. A2_mod for the
increment of p^{n+theta} (the same operator and right-hand side), so p^{n+1} grows by dp / theta;
the velocity update of step 6 is unchanged.  theta = 1 is the scheme above.
"""
from dataclasses import dataclass, field

import numpy as np

from . import operators as ops
from .blocks import SpaceTimeDG
from .krylov import cg, gmres


@dataclass
class State:
    V: np.ndarray          # (nf, 3, Nst) velocity of the last slab
    P: np.ndarray          # (ne, Nst) pressure of the last slab
    t: float = 0.0
    stats: list = field(default_factory=list)


def initial_state(disc: SpaceTimeDG, v0):
    return State(V=ops.project_initial(disc, v0), P=np.zeros((disc.mesh.ne, disc.Nst)), t=0.0)


def solve_pressure(disc, b, tol, restart=50, maxit=100000, method="krylov"):
    """Pinned pressure system: CG on -A when p_t = 0 (Cor. 1-2, reading R1), else GMRES;
    ``method="direct"`` uses a sparse LU of the assembled matrix instead (small meshes)."""
    n = b.size
    if method == "direct":
        from scipy.sparse.linalg import spsolve
        x = spsolve(ops.pressure_sparse(disc).tocsc(), b.ravel())
        return x.reshape(b.shape), 0, 0.0
    if disc.pt == 0:
        x, it, res = cg(lambda v: -ops.pressure_apply(disc, v).ravel(), -b.ravel(), np.zeros(n), tol, maxit)
    else:
        x, it, res = gmres(lambda v: ops.pressure_apply(disc, v).ravel(), b.ravel(), np.zeros(n), tol,
                           restart, maxit)
    return x.reshape(b.shape), it, res


def solve_viscous(disc, rhs, x0, nu, tol, restart=50, maxit=100000, method="krylov"):
    """Eq. A1_mod per component: CG when p_t = 0 (symmetric positive definite, Cor. 3-4), else
    GMRES; ``method="direct"`` uses a sparse LU of the assembled matrix instead."""
    out = np.empty_like(rhs)
    its = []
    if method == "direct":
        from scipy.sparse.linalg import splu
        lu = splu(ops.viscous_sparse(disc, nu).tocsc())
        for c in range(3):
            out[:, c] = lu.solve(np.ascontiguousarray(rhs[:, c].ravel())).reshape(rhs[:, c].shape)
        return out, [0, 0, 0]
    for c in range(3):
        f = lambda v: ops.viscous_apply(disc, v.reshape(rhs[:, c].shape), nu).ravel()
        if disc.pt == 0:
            x, it, _ = cg(f, rhs[:, c].ravel(), x0[:, c].ravel(), tol, maxit)
        else:
            x, it, _ = gmres(f, rhs[:, c].ravel(), x0[:, c].ravel(), tol, restart, maxit)
        out[:, c] = x.reshape(rhs[:, c].shape)
        its.append(it)
    return out, its


def time_step(disc: SpaceTimeDG, state: State, nu, n_picard, vbc, tol=1e-12, restart=50,
              method="krylov", theta=1.0):
    m, N, Ng = disc.mesh, disc.N, disc.Ng
    if theta != 1.0 and (disc.pt != 0 or not 0.5 <= theta <= 1.0):
        raise ValueError("the theta method needs p_t = 0 and 1/2 <= theta <= 1")
    t0 = state.t
    vbar_n = ops.average(disc, state.V)
    Vbc, G = ops.boundary_data(disc, t0, vbc)
    # step 0
    trace = np.einsum("a,jcak->jck", disc.g1, state.V.reshape(m.nf, 3, Ng, N))
    V = np.zeros_like(state.V)
    V[:, :, :N] = trace
    V[~m.interior] = Vbc[~m.interior]
    P = np.zeros((m.ne, disc.Nst))
    bd_rhs = ops.viscous_boundary_rhs(disc, G, nu)
    Mm = np.array([disc.tet_blocks(i)["Mbar_minus"] for i in range(m.ne)])
    Mb = np.array([disc.tet_blocks(i)["Mbar"] for i in range(m.ne)])
    rec = []
    for k in range(n_picard):
        vbar = ops.average(disc, V)                                          # step 1
        Lam = ops.prev_pressure(disc, theta * P + (1.0 - theta) * state.P)
        Ups = ops.convection(disc, vbar, t0, vbc)                            # step 2
        rhs = (np.einsum("ikl,icl->ick", Mm, vbar_n) - Ups
               - np.einsum("ikl,icl->ick", Mb, Lam) + bd_rhs)
        vhalf, vits = solve_viscous(disc, rhs, vbar, nu, tol, restart, method=method)       # step 3
        F = ops.goback(disc, vhalf, Vbc)                                     # step 4
        b = ops.pressure_rhs(disc, F)                                        # step 5
        dp, pits, pres = solve_pressure(disc, b, tol, restart, method=method)
        P = P + dp / theta
        V = ops.velocity_update(disc, F, dp, Vbc)                            # step 6
        rec.append({"visc_its": vits, "press_its": pits, "press_res": pres})
    return State(V=V, P=P, t=t0 + disc.dt, stats=state.stats + [rec])
