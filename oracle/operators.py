"""Operators of the staggered pressure-correction scheme, applied face by face from the
literal space-time blocks of ``blocks.py``.

Arrays: pressure-like fields (ne, Nst); velocity on dual cells (nf, 3, Nst); averaged
velocity on the main grid (ne, 3, Nst).  Index a*N + k as in blocks.py.
"""
import numpy as np

from .blocks import SpaceTimeDG, map_tet, map_tri, st_table


def pin_index(disc: SpaceTimeDG):
    """Pinned pressure entries (reading R3): constant Dubiner mode of tet 0, every time function."""
    return np.array([a * disc.N for a in range(disc.Ng)])


# ---------------------------------------------------------------------------- pressure
def pressure_apply(disc: SpaceTimeDG, x, pinned=True):
    """y = A x with A_i = Sum_{j in S_i, interior} D_ij M_j^-1 (Q_ij x_i + Q_{p(i,j),j} x_p)
    (Eq. CS_19 / A2_mod left-hand side).  Boundary dual cells carry prescribed velocity and
    add nothing to A (reading R2).  With ``pinned``: x at the pins is treated as 0 and
    y at the pins is -x (symmetric elimination keeping -A positive definite)."""
    m = disc.mesh
    xin = np.array(x, dtype=np.float64).reshape(m.ne, disc.Nst)
    xe = xin.copy()
    pins = pin_index(disc)
    if pinned:
        xe[0, pins] = 0.0
    y = np.zeros_like(xe)
    for j in np.nonzero(m.interior)[0]:
        fb = disc.face_blocks(j)
        (l, r) = fb["sides"]
        for c in range(3):
            g = np.linalg.solve(fb["M"], fb["Q"][0][c] @ xe[l] + fb["Q"][1][c] @ xe[r])
            y[l] += fb["D"][0][c] @ g
            y[r] += fb["D"][1][c] @ g
    if pinned:
        y[0, pins] = -xin[0, pins]
    return y


def pressure_dense(disc: SpaceTimeDG, pinned=True):
    """Explicitly assembled A (tiny meshes only)."""
    n = disc.mesh.ne * disc.Nst
    A = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n); e[col] = 1.0
        A[:, col] = pressure_apply(disc, e, pinned).ravel()
    return A


def pressure_rhs(disc: SpaceTimeDG, F, pinned=True):
    """b_i = Sum_{j in S_i} D_ij F_j over all faces of tet i (Eq. A2_mod right-hand side)."""
    m = disc.mesh
    b = np.zeros((m.ne, disc.Nst))
    for j in range(m.nf):
        fb = disc.face_blocks(j)
        for s, i in enumerate(fb["sides"]):
            for c in range(3):
                b[i] += fb["D"][s][c] @ F[j, c]
    if pinned:
        b[0, pin_index(disc)] = 0.0
    return b


def velocity_update(disc: SpaceTimeDG, F, dp, Vbc):
    """v_j = F_j - M_j^-1 (Q_rj dp_r + Q_lj dp_l) on interior faces (Eq. A3_mod);
    boundary dual cells keep their prescribed data."""
    m = disc.mesh
    V = np.array(F, dtype=np.float64, copy=True)
    for j in range(m.nf):
        if not m.interior[j]:
            V[j] = Vbc[j]
            continue
        fb = disc.face_blocks(j)
        (l, r) = fb["sides"]
        for c in range(3):
            V[j, c] = F[j, c] - np.linalg.solve(fb["M"], fb["Q"][1][c] @ dp[r] + fb["Q"][0][c] @ dp[l])
    return V


def divergence(disc: SpaceTimeDG, V):
    """Sum_{j in S_i} D_ij v_j (Eq. CS_15 left-hand side), per tet."""
    return pressure_rhs(disc, V, pinned=False)


# ---------------------------------------------------------------------------- averaging
def average(disc: SpaceTimeDG, V):
    """vbar_i = M_i^-1 Sum_{j in S_i} M_ij v_j (Eq. vis1 / average)."""
    m = disc.mesh
    acc = np.zeros((m.ne, 3, disc.Nst))
    for j in range(m.nf):
        fb = disc.face_blocks(j)
        for s, i in enumerate(fb["sides"]):
            acc[i] += (fb["Mij"][s] @ V[j].T).T
    out = np.empty_like(acc)
    for i in range(m.ne):
        out[i] = np.linalg.solve(disc.tet_blocks(i)["Mi"], acc[i].T).T
    return out


def prev_pressure(disc: SpaceTimeDG, P):
    """Lambda_i = M_i^-1 Sum_{j in S_i} M_ij M_j^-1 (Q_rj p_r + Q_lj p_l) (Eq. prevpress).
    Boundary faces contribute M_j^-1 Qvol_ij p_i: the one-sided volume term (reading R13)."""
    m = disc.mesh
    acc = np.zeros((m.ne, 3, disc.Nst))
    for j in range(m.nf):
        fb = disc.face_blocks(j)
        g = np.zeros((3, disc.Nst))
        for c in range(3):
            if m.interior[j]:
                (l, r) = fb["sides"]
                g[c] = np.linalg.solve(fb["M"], fb["Q"][1][c] @ P[r] + fb["Q"][0][c] @ P[l])
            else:
                i = fb["sides"][0]
                g[c] = np.linalg.solve(fb["M"], fb["Qvol"][0][c] @ P[i])
        for s, i in enumerate(fb["sides"]):
            acc[i] += (fb["Mij"][s] @ g.T).T
    out = np.empty_like(acc)
    for i in range(m.ne):
        out[i] = np.linalg.solve(disc.tet_blocks(i)["Mi"], acc[i].T).T
    return out


def goback(disc: SpaceTimeDG, vbar, Vbc):
    """F_j = Mbar_j^-1 (M_lj^T vbar_l + M_rj^T vbar_r) on interior faces (Eq. goback);
    boundary dual cells take the prescribed data (reading R2)."""
    m = disc.mesh
    F = np.zeros((m.nf, 3, disc.Nst))
    for j in range(m.nf):
        if not m.interior[j]:
            F[j] = Vbc[j]
            continue
        fb = disc.face_blocks(j)
        acc = np.zeros((3, disc.Nst))
        for s, i in enumerate(fb["sides"]):
            acc += (fb["Mij"][s].T @ vbar[i].T).T
        F[j] = np.linalg.solve(fb["Mbar"], acc.T).T
    return F


# ---------------------------------------------------------------------------- viscous
def viscous_apply(disc: SpaceTimeDG, X, nu):
    """Left-hand side of Eq. A1_mod for one velocity component X (ne, Nst):
    Mbar_i X_i - nu Sum_{j in S_i} D_ij Mbar_j^-1 (Q_ij X_i + Q_{p(i,j),j} X_p).
    On a boundary face the neighbour is the Dirichlet ghost (reading R25): its known part
    goes to the right-hand side (``viscous_boundary_rhs``)."""
    m = disc.mesh
    y = np.zeros_like(X)
    for i in range(m.ne):
        y[i] = disc.tet_blocks(i)["Mbar"] @ X[i]
    for j in range(m.nf):
        fb = disc.face_blocks(j)
        sides = fb["sides"]
        for c in range(3):
            q = sum(fb["Q"][s][c] @ X[i] for s, i in enumerate(sides))
            g = np.linalg.solve(fb["Mbar"], q)
            for s, i in enumerate(sides):
                y[i] -= nu * fb["D"][s][c] @ g
    return y


def viscous_boundary_rhs(disc: SpaceTimeDG, G, nu):
    """+nu D_ij Mbar_j^-1 G_j for boundary faces; G (nf, 3 mom, 3 dir, Nst) from boundary_data."""
    m = disc.mesh
    out = np.zeros((m.ne, 3, disc.Nst))
    for j in np.nonzero(~m.interior)[0]:
        fb = disc.face_blocks(j)
        i = fb["sides"][0]
        for mm in range(3):
            for c in range(3):
                out[i, mm] += nu * fb["D"][0][c] @ np.linalg.solve(fb["Mbar"], G[j, mm, c])
    return out


# ---------------------------------------------------------------------------- convection
def rusanov(vm, vp, n):
    """F_c^RS(v-, v+) . n of the paper's Rusanov flux, s_max = 2 max(|v+|, |v-|) pointwise
    (reading R12).  vm, vp (q, 3); n (3,) outward from the '-' side."""
    fm = vm * (vm @ n)[:, None]
    fp = vp * (vp @ n)[:, None]
    smax = 2.0 * np.maximum(np.linalg.norm(vp, axis=1), np.linalg.norm(vm, axis=1))
    return 0.5 * (fp + fm) - 0.5 * smax[:, None] * (vp - vm)


def convection(disc: SpaceTimeDG, vbar, t0, vbc):
    """Upsilon^c_i of Eq. convdg, per tet and momentum component: (ne, 3, Nst).

    Face integrals use the canonical point set of each face (identical for both sides);
    at a boundary face v+ = v_bc (reading R12).  ``vbc(x, t) -> (m, 3)``."""
    m, dt = disc.mesh, disc.dt
    tau, wt = disc.time_nl
    gv, _ = disc.gamma(tau)
    out = np.zeros((m.ne, 3, disc.Nst))
    fref = disc.tri_nl
    for i in range(m.ne):
        x, w = map_tet(m.tet_coords(i), *disc.tet_nl)
        ph, dph = disc.phi(i, x)
        Fst = st_table(ph, gv)
        W = np.kron(w, wt) * dt
        v = np.stack([Fst @ vbar[i, c] for c in range(3)], axis=1)      # (q, 3)
        for c in range(3):
            for d in range(3):
                out[i, c] -= st_table(dph[:, :, d], gv).T @ (W * v[:, c] * v[:, d])
        for f in range(4):
            j = m.t2f[i, f]
            fx, fw = map_tri(m.face_coords(j), *fref)
            n_out = m.normal[j] * m.sigma(i, j)
            phf, _ = disc.phi(i, fx)
            Ff = st_table(phf, gv)
            Wf = np.kron(fw, wt) * dt
            vm = np.stack([Ff @ vbar[i, c] for c in range(3)], axis=1)
            nb = m.t2n[i, f]
            if nb >= 0:
                phn, _ = disc.phi(nb, fx)
                Fn = st_table(phn, gv)
                vp = np.stack([Fn @ vbar[nb, c] for c in range(3)], axis=1)
            else:
                xq = np.repeat(fx, len(tau), axis=0)
                tq = np.tile(t0 + tau * dt, len(fx))
                vp = vbc(xq, tq)
            flux = rusanov(vm, vp, n_out)
            for c in range(3):
                out[i, c] += Ff.T @ (Wf * flux[:, c])
    return out


# ---------------------------------------------------------------------------- data
def project_initial(disc: SpaceTimeDG, v0):
    """Spatial L2 projection of v0(x) onto each dual cell, as a constant-in-time space-time
    vector (the coefficient of gamma_0 = 1): (nf, 3, Nst)."""
    m = disc.mesh
    V = np.zeros((m.nf, 3, disc.Nst))
    for j in range(m.nf):
        rhs = np.zeros((disc.N, 3))
        mass = np.zeros((disc.N, disc.N))
        for _, Vt in m.dual_subtets(j):
            x, w = map_tet(Vt, *disc.tet_nl)
            ps = disc.psi(j, x)
            rhs += (ps * w[:, None]).T @ v0(x)
            xl, wl = map_tet(Vt, *disc.tet_lin)
            pl = disc.psi(j, xl)
            mass += (pl * wl[:, None]).T @ pl
        s = np.linalg.solve(mass, rhs)                    # (N, 3)
        V[j, :, :disc.N] = s.T                            # gamma_0 = 1
    return V


def boundary_data(disc: SpaceTimeDG, t0, vbc):
    """For every boundary face j of tet i on the slab [t0, t0+dt]:
    Vbc_j = Mbar_j^-1 int psi~ v_bc (space-time L2 projection on T_ij, reading R2) and
    G_j[m, c] = int_{Gamma_j^st} psi~ v_bc,m n_c (viscous Dirichlet ghost, reading R25)."""
    m, dt = disc.mesh, disc.dt
    tau, wt = disc.time_nl
    gv, _ = disc.gamma(tau)
    Vbc = np.zeros((m.nf, 3, disc.Nst))
    G = np.zeros((m.nf, 3, 3, disc.Nst))
    for j in np.nonzero(~m.interior)[0]:
        fb = disc.face_blocks(j)
        i = fb["sides"][0]
        x, w = map_tet(m.subtet(i, j), *disc.tet_nl)
        Pst = st_table(disc.psi(j, x), gv)
        W = np.kron(w, wt) * dt
        vq = vbc(np.repeat(x, len(tau), axis=0), np.tile(t0 + tau * dt, len(x)))
        Vbc[j] = np.linalg.solve(fb["Mbar"], (Pst * W[:, None]).T @ vq).T
        fx, fw = map_tri(m.face_coords(j), *disc.tri_nl)
        Pf = st_table(disc.psi(j, fx), gv)
        Wf = np.kron(fw, wt) * dt
        vf = vbc(np.repeat(fx, len(tau), axis=0), np.tile(t0 + tau * dt, len(fx)))
        n = m.normal[j]
        for mm in range(3):
            for c in range(3):
                G[j, mm, c] = Pf.T @ (Wf * vf[:, mm] * n[c])
    return Vbc, G


# ---------------------------------------------------------------------------- assembled
def pressure_sparse(disc: SpaceTimeDG, pinned=True):
    """The matrix of ``pressure_apply`` assembled block by block (scipy CSR)."""
    import scipy.sparse as spm
    m, Nst = disc.mesh, disc.Nst
    rows, cols, vals = [], [], []
    ii, kk = np.meshgrid(np.arange(Nst), np.arange(Nst), indexing="ij")
    for j in np.nonzero(m.interior)[0]:
        fb = disc.face_blocks(j)
        for s, i in enumerate(fb["sides"]):
            for s2, i2 in enumerate(fb["sides"]):
                blk = sum(fb["D"][s][c] @ np.linalg.solve(fb["M"], fb["Q"][s2][c]) for c in range(3))
                rows.append((i * Nst + ii).ravel()); cols.append((i2 * Nst + kk).ravel())
                vals.append(blk.ravel())
    n = m.ne * Nst
    A = spm.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n, n)).tocsr()
    if pinned:
        pins = pin_index(disc)
        keep = np.ones(n); keep[pins] = 0.0
        Dk = spm.diags(keep)
        A = (Dk @ A @ Dk - spm.diags(1.0 - keep)).tocsr()
    return A


def viscous_sparse(disc: SpaceTimeDG, nu):
    """The matrix of ``viscous_apply`` assembled block by block (scipy CSR)."""
    import scipy.sparse as spm
    m, Nst = disc.mesh, disc.Nst
    rows, cols, vals = [], [], []
    ii, kk = np.meshgrid(np.arange(Nst), np.arange(Nst), indexing="ij")
    for i in range(m.ne):
        rows.append((i * Nst + ii).ravel()); cols.append((i * Nst + kk).ravel())
        vals.append(disc.tet_blocks(i)["Mbar"].ravel())
    for j in range(m.nf):
        fb = disc.face_blocks(j)
        for s, i in enumerate(fb["sides"]):
            for s2, i2 in enumerate(fb["sides"]):
                blk = -nu * sum(fb["D"][s][c] @ np.linalg.solve(fb["Mbar"], fb["Q"][s2][c])
                                for c in range(3))
                rows.append((i * Nst + ii).ravel()); cols.append((i2 * Nst + kk).ravel())
                vals.append(blk.ravel())
    n = m.ne * Nst
    return spm.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n)).tocsr()
