"""Primary tetrahedral mesh, faces and the face-based dual grid (Sec. 2.2).

* S_i: the four faces of tet i; local face f of a tet is the face opposite its local vertex f.
* l(j), r(j): left / right tet of interior face j; the paper assigns them arbitrarily, here
  l = lower tet id (reading R5).  n_j is the unit normal pointing from l(j) to r(j).
* Faces are numbered in increasing (l(j), local face index in l(j)) order.
* Dual cell of interior face j: H_j = T_{l,j} U T_{r,j}, T_{i,j} = tetrahedron spanned by
  face j and the barycentre of T_i.  A boundary face's dual cell is T_{i,j} (reading R2).
* The canonical vertex order (A, B, C) of face j is l(j)'s local order.
* Periodic meshes (period given): vertex ids are the lattice points of the periodic box, a
  tetrahedron's geometry is its vertices' periodic images nearest to its first vertex, faces
  are matched by vertex ids (so every face is interior), and face geometry is taken in l(j)'s
  frame.  Points are mapped into a tetrahedron's reference coordinates through the periodic
  image nearest to it, so basis functions of r(j) can be evaluated at points given in l(j)'s
  frame.
"""
import numpy as np


class Mesh:
    def __init__(self, verts, tets, period=None):
        self.X = np.asarray(verts, dtype=np.float64)
        self.T = np.asarray(tets, dtype=np.int64)
        self.period = None if period is None else np.asarray(period, dtype=np.float64)
        ne = self.T.shape[0]
        P = self.X[self.T]                                   # (ne, 4, 3)
        if self.period is not None:                          # nearest images to the first vertex
            P = P[:, :1] + self.min_image(P - P[:, :1])
        self.P = P
        self.J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=-1)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0):
            raise ValueError("inverted or degenerate tetrahedron")
        self.Jinv = np.linalg.inv(self.J)
        self.bary = P.mean(axis=1)
        self.ne = ne

        faces = {}
        for i in range(ne):
            for f in range(4):
                key = tuple(sorted(int(v) for k, v in enumerate(self.T[i]) if k != f))
                faces.setdefault(key, []).append((i, f))
        recs = []
        for key, lst in faces.items():
            if len(lst) > 2:
                raise ValueError("non-manifold face")
            lst = sorted(lst)
            (l, fl) = lst[0]
            (r, fr) = lst[1] if len(lst) == 2 else (-1, -1)
            recs.append((l, fl, r, fr))
        recs.sort()
        self.nf = len(recs)
        self.left = np.array([r[0] for r in recs])
        self.fl = np.array([r[1] for r in recs])
        self.right = np.array([r[2] for r in recs])
        self.fr = np.array([r[3] for r in recs])
        self.interior = self.right >= 0
        self.t2f = np.full((ne, 4), -1, dtype=np.int64)
        self.t2n = np.full((ne, 4), -1, dtype=np.int64)
        for j, (l, fl, r, fr) in enumerate(recs):
            self.t2f[l, fl] = j
            self.t2n[l, fl] = r
            if r >= 0:
                self.t2f[r, fr] = j
                self.t2n[r, fr] = l
        # canonical face vertices: l's local order, skipping local vertex fl (coordinates in l's frame)
        self.fverts = np.array([[self.T[l, k] for k in range(4) if k != fl]
                                for (l, fl, _, _) in recs])
        self.fcoords = np.array([[P[l, k] for k in range(4) if k != fl] for (l, fl, _, _) in recs])
        A, B, C = (self.fcoords[:, k] for k in range(3))
        cr = np.cross(B - A, C - A)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        n = cr / (2.0 * self.area[:, None])
        opp = P[self.left, self.fl]
        flip = np.einsum("jd,jd->j", n, opp - A) > 0      # must point away from l's opposite vertex
        n[flip] *= -1.0
        self.normal = n

    def min_image(self, d):
        """Displacements d (..., 3) replaced by their periodic images nearest to 0 (identity for a
        non-periodic mesh)."""
        d = np.asarray(d, dtype=np.float64)
        return d if self.period is None else d - self.period * np.round(d / self.period)

    def tet_coords(self, i):
        """Vertex coordinates (4,3) of tet i (its own frame)."""
        return self.P[i]

    def face_coords(self, j):
        """Canonical vertex coordinates (3,3) of face j, in l(j)'s frame."""
        return self.fcoords[j]

    # ---- dual grid -------------------------------------------------------------------
    def subtet(self, i, j):
        """Vertices (4,3) of T_{i,j}: canonical face vertices of j, then barycentre of i (for a
        periodic face, r(j)'s barycentre is taken at its image next to the face)."""
        F = self.fcoords[j]
        b = F[0] + self.min_image(self.bary[i] - F[0])
        return np.vstack([F, b[None, :]])

    def dual_subtets(self, j):
        """[(side tet id, vertices)] making up the dual cell of face j."""
        out = [(int(self.left[j]), self.subtet(self.left[j], j))]
        if self.interior[j]:
            out.append((int(self.right[j]), self.subtet(self.right[j], j)))
        return out

    def dual_center_scale(self, j):
        """x0 = volume centroid of the dual cell, h = max over its vertices of |v - x0|_inf
        (reading R6; the orthonormalised basis does not depend on either in exact arithmetic)."""
        vols, cents, verts = [], [], []
        for _, V in self.dual_subtets(j):
            vols.append(abs(np.linalg.det((V[1:] - V[0]).T)) / 6.0)
            cents.append(V.mean(axis=0))
            verts.append(V)
        vols = np.array(vols)
        x0 = (vols[:, None] * np.array(cents)).sum(axis=0) / vols.sum()
        h = np.abs(np.vstack(verts) - x0).max()
        return x0, h

    def sigma(self, i, j):
        """sigma_{i,j} of Eq. SD_1: +1 for i = l(j), -1 for i = r(j) (reading R20)."""
        return 1.0 if i == self.left[j] else -1.0

    def to_ref(self, i, x):
        """Reference coordinates of physical points x (m,3) in tet i (through their periodic
        images nearest to tet i on a periodic mesh)."""
        return self.min_image(np.asarray(x) - self.P[i, 0]) @ self.Jinv[i].T
