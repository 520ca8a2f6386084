"""Pins for the seeded mesh generator and the oracle's connectivity / dual grid (Sec. 2.2)."""
import numpy as np
import pytest

from inputs import kuhn_mesh, splitmix64_doubles
from oracle.mesh import Mesh


def test_splitmix64_reference_values():
    # first outputs of splitmix64 seeded with 0 (Vigna's reference stream), as 53-bit doubles
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = splitmix64_doubles(0, 3)
    assert np.array_equal(got, np.array([(r >> 11) / 2.0 ** 53 for r in ref]))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_counts_and_volumes(n):
    v, t = kuhn_mesh(n, seed=0)
    m = Mesh(v, t)
    nb = int((~m.interior).sum())
    assert m.ne == 6 * n ** 3 and nb == 12 * n * n and m.interior.sum() == (4 * m.ne - nb) // 2
    assert abs(m.detJ.sum() / 6.0 - 1.0) < 1e-13          # tets tile the unit cube
    # dual cells tile the cube too; every sub-tet T_ij has a quarter of T_i's volume
    vol = 0.0
    for j in range(m.nf):
        for i, V in m.dual_subtets(j):
            vij = abs(np.linalg.det((V[1:] - V[0]).T)) / 6.0
            assert abs(vij - m.detJ[i] / 24.0) < 1e-15
            vol += vij
    assert abs(vol - 1.0) < 1e-13


def test_orientation_and_closure():
    v, t = kuhn_mesh(3, seed=5)
    m = Mesh(v, t)
    s = np.zeros((m.ne, 3))
    for j in range(m.nf):
        l, r = m.left[j], m.right[j]
        assert l < r or r < 0
        s[l] += m.area[j] * m.normal[j]
        if r >= 0:
            s[r] -= m.area[j] * m.normal[j]
            # n_j points from l to r
            assert m.normal[j] @ (m.bary[r] - m.bary[l]) > 0
        assert m.t2f[l, m.fl[j]] == j
    assert np.abs(s).max() < 1e-15
    assert (m.t2f >= 0).all()
    # boundary faces lie on the cube surface with outward normals
    for j in np.nonzero(~m.interior)[0]:
        c = m.X[m.fverts[j]].mean(0)
        assert np.isclose(np.abs(m.normal[j]).max(), 1.0)
        assert np.min(np.minimum(c, 1 - c)) < 1e-12


def test_jitter_bounds_and_boundary_untouched():
    n = 4
    v0, _ = kuhn_mesh(n, seed=0, jitter=0.0)
    v1, _ = kuhn_mesh(n, seed=3)
    d = np.abs(v1 - v0)
    assert d.max() <= 0.1 / n + 1e-15 and d.max() > 0.05 / n
    onb = (np.isclose(v0, 0) | np.isclose(v0, 1)).any(axis=1)
    assert d[onb].max() == 0.0
