"""Space-time coefficient matrices, assembled literally by space-time quadrature.

Index convention for space-time coefficient vectors (reading R22): entry a*N + k holds the
coefficient of gamma_a(tau) * phi_k (or psi_k), a = time index, k = space index.

All blocks follow the paper's definitions with dt = Delta t * dtau, t = t^n + tau Delta t:
  D_{i,j}   Eq. MD_3    Q_{i,j}  Eq. MD_6 (sigma of Eq. SD_1)   M_j = M_j^+ - M_j^o  Eqs. MD_2, MD_2_2
  M_i, M_{i,j}  Eq. vis3      Mbar_j  Eq. mj      Mbar_i^{+,-,o}  Eqs. vis11_1, vis11_2, vis11
Dual basis: the Taylor monomials of Eq. bf_2, orthonormalised on each dual cell by
Gram-Schmidt in the multi-index order (reading R6; same span as the paper's basis).
For a boundary face the dual cell is T_{i,j} (reading R2), i takes the role of l(j)
(sigma = +1, n_ij = n_j outward), and Qvol is the volume part of Q alone (reading R13).
"""
from functools import lru_cache

import numpy as np

from .basis import dubiner, legendre01, nbasis, taylor
from .mesh import Mesh
from .quadrature import line_rule, n_linear, n_nonlinear, tet_rule, tri_rule


def st_table(space_vals, time_vals):
    """(m, N) x (mt, Ng) -> (m*mt, Ng*N) table of gamma_a(tau_t) * f_k(x_q), row q*mt + t."""
    m, N = space_vals.shape
    mt, Ng = time_vals.shape
    out = time_vals[None, :, :, None] * space_vals[:, None, None, :]     # (m, mt, Ng, N)
    return out.reshape(m * mt, Ng * N)


def map_tet(V, ref_pts, ref_wts):
    """Physical points / weights of a reference tet rule on the tetrahedron with vertices V."""
    Jm = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], axis=-1)
    return V[0] + ref_pts @ Jm.T, ref_wts * abs(np.linalg.det(Jm))


def map_tri(V, ref_pts, ref_wts):
    """Physical points / weights of a reference triangle rule on the triangle V (3,3)."""
    x = V[0] + ref_pts[:, :1] * (V[1] - V[0]) + ref_pts[:, 1:2] * (V[2] - V[0])
    area = 0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
    return x, ref_wts * 2.0 * area


class SpaceTimeDG:
    def __init__(self, mesh: Mesh, p: int, pt: int, dt: float):
        self.mesh, self.p, self.pt, self.dt = mesh, p, pt, float(dt)
        self.N = nbasis(p)
        self.Ng = pt + 1
        self.Nst = self.N * self.Ng
        self.tet_lin = tet_rule(n_linear(p))
        self.tri_lin = tri_rule(n_linear(p))
        self.time_lin = line_rule(n_linear(pt))
        self.tet_nl = tet_rule(n_nonlinear(p))
        self.tri_nl = tri_rule(n_nonlinear(p))
        self.time_nl = line_rule(n_nonlinear(pt))
        self.g0 = legendre01(pt, 0.0)[0][0]
        self.g1 = legendre01(pt, 1.0)[0][0]
        self._face = {}
        self._tet = {}

    # ---- bases at physical points -----------------------------------------------------
    def phi(self, i, x):
        """phi^(i) values (m,N) and physical gradients (m,N,3) at physical points x."""
        v, g = dubiner(self.p, self.mesh.to_ref(i, x))
        return v, g @ self.mesh.Jinv[i]          # grad_x = J^-T grad_xi  (row-vector form)

    @lru_cache(maxsize=None)
    def dual_basis(self, j):
        """(x0, h, C): psi_hat(x) = C @ taylor(x), orthonormal on the dual cell.

        Gram-Schmidt of the Taylor monomials in the fixed multi-index order, computed as two
        Cholesky passes (the second restores orthonormality lost to the Gram matrix's
        conditioning, which reaches ~1e9 at p = 4 on these cells)."""
        x0, h = self.mesh.dual_center_scale(j)
        pts, wts = [], []
        for _, V in self.mesh.dual_subtets(j):
            x, w = map_tet(V, *self.tet_lin)
            pts.append(x); wts.append(w)
        x = np.vstack(pts); w = np.concatenate(wts)
        T = taylor(self.p, x, x0, h)
        C = np.linalg.inv(np.linalg.cholesky((T * w[:, None]).T @ T))
        P = T @ C.T
        C = np.linalg.inv(np.linalg.cholesky((P * w[:, None]).T @ P)) @ C
        return x0, h, C

    def psi(self, j, x):
        x0, h, C = self.dual_basis(j)
        return taylor(self.p, x, x0, h) @ C.T

    def gamma(self, tau):
        return legendre01(self.pt, tau)

    # ---- per-face blocks (literal space-time) ----------------------------------------
    def face_blocks(self, j):
        if j in self._face:
            return self._face[j]
        m, dt, N, Nst = self.mesh, self.dt, self.N, self.Nst
        tau, wt = self.time_lin
        gv, gd = self.gamma(tau)
        n_j = m.normal[j]
        fx, fw = map_tri(m.face_coords(j), *self.tri_lin)
        out = {"sides": [], "Q": [], "D": [], "Mij": [], "Qvol": []}
        Mp = np.zeros((Nst, Nst)); Mo = np.zeros((Nst, Nst)); Mbar = np.zeros((Nst, Nst))
        for i, V in m.dual_subtets(j):
            x, w = map_tet(V, *self.tet_lin)
            ps = self.psi(j, x)
            ph, dph = self.phi(i, x)
            W = np.kron(w, wt) * dt                                   # space-time weights
            Pst = st_table(ps, gv)
            Fst = st_table(ph, gv)
            sig = m.sigma(i, j)
            # face part, same canonical face points for every side
            psf = self.psi(j, fx)
            phf, _ = self.phi(i, fx)
            Wf = np.kron(fw, wt) * dt
            Psf = st_table(psf, gv)
            Fsf = st_table(phf, gv)
            Q, D, Qv = [], [], []
            for c in range(3):
                dFst = st_table(dph[:, :, c], gv)
                vol = (Pst * W[:, None]).T @ dFst                     # int psi~_k d_c phi~_l
                fac = (Psf * Wf[:, None]).T @ Fsf                     # int_face psi~_k phi~_l
                Q.append(vol - fac * sig * n_j[c])                    # Eq. MD_6
                Qv.append(vol)
                D.append(((Fsf * Wf[:, None]).T @ Psf) * sig * n_j[c]
                         - (dFst * W[:, None]).T @ Pst)              # Eq. MD_3, n_ij = sigma n_j
            out["sides"].append(i)
            out["Q"].append(np.array(Q))
            out["D"].append(np.array(D))
            out["Qvol"].append(np.array(Qv))
            out["Mij"].append((Fst * W[:, None]).T @ Pst)             # Eq. vis3, M_{i,j}
            # dual-cell masses accumulate over the sub-tetrahedra of H_j
            P1 = st_table(ps, self.g1[None, :])
            Mp += (P1 * w[:, None]).T @ P1                            # Eq. MD_2
            dPst = st_table(ps, gd) / dt                              # d/dt psi~ = (1/dt) d/dtau
            Mo += (dPst * W[:, None]).T @ Pst                         # Eq. MD_2_2
            Mbar += (Pst * W[:, None]).T @ Pst                        # Eq. mj
        out["M"] = Mp - Mo
        out["Mbar"] = Mbar
        self._face[j] = out
        return out

    def side_index(self, j, i):
        return self.face_blocks(j)["sides"].index(i)

    # ---- per-tet blocks ----------------------------------------------------------------
    def tet_blocks(self, i):
        if i in self._tet:
            return self._tet[i]
        m, dt = self.mesh, self.dt
        tau, wt = self.time_lin
        gv, gd = self.gamma(tau)
        x, w = map_tet(m.tet_coords(i), *self.tet_lin)
        ph, _ = self.phi(i, x)
        W = np.kron(w, wt) * dt
        Fst = st_table(ph, gv)
        F1 = st_table(ph, self.g1[None, :])
        F0 = st_table(ph, self.g0[None, :])
        dF = st_table(ph, gd) / dt
        out = {
            "Mi": (Fst * W[:, None]).T @ Fst,                                # Eq. vis3
            "Mbar_plus": (F1 * w[:, None]).T @ F1,                           # Eq. vis11_1
            "Mbar_minus": (F0 * w[:, None]).T @ F1,                          # Eq. vis11_2 (R9)
            "Mbar_o": (dF * W[:, None]).T @ Fst,                             # Eq. vis11
        }
        out["Mbar"] = out["Mbar_plus"] - out["Mbar_o"]
        self._tet[i] = out
        return out
