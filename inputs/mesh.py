"""Jittered Kuhn meshes of the unit cube: n^3 hexahedra, each split into 6 tetrahedra.

The paper's convergence meshes have N_e = 6 n^3 elements (Sec. 3.2, Tables 1-2), i.e.
the same hexahedron-split family; the split pattern and the jitter used here are
the workload recipe of this project, not the paper's.

Vertex id of lattice point (i, j, k) is i + (n+1) (j + (n+1) k).  Tet id of the
tetrahedron with permutation index s in hexahedron (i, j, k) is 6 (i + n (j + n k)) + s.
For permutation pi of the axes (lexicographic order), the tetrahedron is
v0 = c, v1 = v0 + h e_pi0, v2 = v1 + h e_pi1, v3 = c + h (1,1,1), with v2 and v3 swapped
when the (unjittered) orientation is negative, so every tetrahedron is positively oriented.
Interior vertices get independent U(-a h, a h) offsets per coordinate, drawn from
splitmix64(seed) as 53-bit doubles in vertex-id order, x then y then z.
"""
from itertools import permutations

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64_doubles(seed: int, count: int) -> np.ndarray:
    """`count` doubles in [0, 1) from Vigna's splitmix64 stream (top 53 bits of each output)."""
    out = np.empty(count, dtype=np.float64)
    state = seed & _MASK
    for t in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        z ^= z >> 31
        out[t] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def kuhn_mesh(n: int, seed: int = 0, jitter: float = 0.1):
    """Return (verts[(n+1)^3, 3] float64, tets[6 n^3, 4] int64) for the unit cube."""
    h = 1.0 / n
    m = n + 1
    g = np.arange(m, dtype=np.float64) * h
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()          # vertex id order: i fastest
    verts = np.stack([g[ii], g[jj], g[kk]], axis=1)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
    nint = int(interior.sum())
    if jitter != 0.0 and nint > 0:
        u = splitmix64_doubles(seed, 3 * nint).reshape(nint, 3)
        verts[interior] += (2.0 * u - 1.0) * (jitter * h)

    perms = list(permutations(range(3)))                    # lexicographic order
    local = []                                              # per permutation: 4 lattice offsets
    for pi in perms:
        o0 = np.zeros(3, dtype=np.int64)
        o1 = o0.copy(); o1[pi[0]] += 1
        o2 = o1.copy(); o2[pi[1]] += 1
        o3 = np.ones(3, dtype=np.int64)
        det = np.linalg.det(np.stack([o1 - o0, o2 - o0, o3 - o0]).astype(np.float64))
        if det < 0:
            o2, o3 = o3, o2
        local.append((o0, o1, o2, o3))

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # hexahedron linear index i + n (j + n k): order with i fastest
    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for s, offs in enumerate(local):
        for v, o in enumerate(offs):
            tets[:, s, v] = (hi + o[0]) + m * ((hj + o[1]) + m * (hk + o[2]))
    return verts, tets.reshape(-1, 4)


def kuhn_periodic_mesh(n: int, lo: float = -np.pi, length: float = 2.0 * np.pi):
    """Regular Kuhn mesh of the periodic box [lo, lo + length)^3 (the domain of the paper's
    convergence test, Sec. 3.2): n^3 hexahedra x 6 tetrahedra with the split and tet ids of
    kuhn_mesh, on the n^3 lattice points of the box, vertex id i + n (j + n k), lattice
    indices taken modulo n (the vertices on the far faces are the periodic images of those on
    the near faces).  Returns (verts[n^3, 3], tets[6 n^3, 4], period[3]); the geometry of a
    tetrahedron is its vertices' nearest periodic images to its first vertex.  n >= 3."""
    if n < 3:
        raise ValueError("a periodic Kuhn mesh needs n >= 3")
    h = length / n
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    verts = lo + h * np.stack([ii, jj, kk], axis=1).astype(np.float64)
    perms = list(permutations(range(3)))
    local = []
    for pi in perms:
        o0 = np.zeros(3, dtype=np.int64)
        o1 = o0.copy(); o1[pi[0]] += 1
        o2 = o1.copy(); o2[pi[1]] += 1
        o3 = np.ones(3, dtype=np.int64)
        det = np.linalg.det(np.stack([o1 - o0, o2 - o0, o3 - o0]).astype(np.float64))
        if det < 0:
            o2, o3 = o3, o2
        local.append((o0, o1, o2, o3))
    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for s, offs in enumerate(local):
        for v, o in enumerate(offs):
            tets[:, s, v] = (hi + o[0]) % n + n * (((hj + o[1]) % n) + n * ((hk + o[2]) % n))
    return verts, tets.reshape(-1, 4), np.full(3, length)

