"""The C-ABI library builds, loads and exports every symbol include/stdg.h declares; host-side
calls (mesh, reference tables) agree with the oracle.  No GPU needed."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1601_07384_gb300.build import build
    path = build()
    import ctypes
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(stdg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1601_07384_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_host_mesh_matches_oracle(lib):
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh
    from oracle.mesh import Mesh
    v, t = kuhn_mesh(3, seed=2)
    m = g.Mesh(v, t)
    om = Mesh(v, t)
    l, r, fl, fr = m.faces()
    assert (m.ne, m.nf, m.ninterior, m.nboundary) == (162, 378, 270, 108)
    assert np.array_equal(l, om.left) and np.array_equal(r, om.right)
    assert np.array_equal(fl, om.fl) and np.array_equal(fr, om.fr)


def test_host_mesh_rejects_bad_input(lib):
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh
    v, t = kuhn_mesh(2, seed=0)
    with pytest.raises(g.StdgError, match="EMESH"):
        g.Mesh(v, t[:, [0, 2, 1, 3]])                     # inverted
    with pytest.raises(g.StdgError, match="EMESH"):
        g.Mesh(v, np.vstack([t, t[:1]]))                 # face shared by 3 tets
    with pytest.raises(g.StdgError, match="EUNSUPPORTED"):
        g.Reference(5, 0)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_host_basis_and_rules_match_oracle(lib, p):
    import paper_1601_07384_gb300 as g
    from oracle.basis import dubiner
    from oracle.quadrature import tet_rule
    x, w = g.tet_rule(p + 1)
    xo, wo = tet_rule(p + 1)
    assert np.abs(x - xo).max() < 1e-15 and np.abs(w - wo).max() < 1e-16
    xi = np.random.default_rng(p).random((30, 3)) / 3.0
    R = g.Reference(p, 0)
    ph, dph = R.eval(xi)
    pho, dpho = dubiner(p, xi)
    assert np.abs(ph - pho).max() < 1e-12 * max(1, np.abs(pho).max())
    assert np.abs(dph - dpho.transpose(0, 2, 1)).max() < 1e-12 * max(1, np.abs(dpho).max())


@pytest.mark.parametrize("pt", [0, 1, 2, 3])
def test_time_matrix_matches_oracle(lib, pt):
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh
    from oracle.blocks import SpaceTimeDG
    from oracle.mesh import Mesh
    v, t = kuhn_mesh(1, seed=0)
    d = SpaceTimeDG(Mesh(v, t), 1, pt, 0.1)
    Kor = d.face_blocks(0)["M"][::d.N, ::d.N]
    assert np.abs(g.Reference(1, pt).time_matrix() - Kor).max() < 1e-13


@pytest.mark.parametrize("pt", [0, 1, 2, 3, 4])
def test_time_blockdiag_of_the_time_matrix(lib, pt):
    """stdg_time_blockdiag (host logic of the time-decoupled viscous solve): K = W R W^-1 with R real
    block diagonal, whose blocks carry exactly the eigenvalues numpy finds for K."""
    import paper_1601_07384_gb300 as g
    K = g.Reference(1, pt).time_matrix()
    W, Wi, R, pair = g.time_blockdiag(K)
    n = pt + 1
    assert np.abs(K @ W - W @ R).max() <= 1e-12 * max(1.0, np.abs(K).max())
    assert np.abs(W @ Wi - np.eye(n)).max() <= 1e-12
    ev = []
    mask = np.zeros((n, n), dtype=bool)
    a = 0
    while a < n:
        if pair[a]:
            assert R[a, a] == R[a + 1, a + 1] and R[a, a + 1] == -R[a + 1, a] and R[a, a + 1] != 0
            ev += [complex(R[a, a], R[a, a + 1]), complex(R[a, a], -R[a, a + 1])]
            mask[a:a + 2, a:a + 2] = True
            a += 2
        else:
            ev.append(complex(R[a, a], 0.0))
            mask[a, a] = True
            a += 1
    assert np.all(R[~mask] == 0.0)
    ref = np.linalg.eigvals(K)
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert np.allclose(sorted(ev, key=key), sorted(ref, key=key), atol=1e-10)
    # K + K^T is positive semidefinite, so every eigenvalue has a nonnegative real part
    assert min(z.real for z in ev) >= -1e-12


def test_time_blockdiag_rotation_and_errors(lib):
    """A scaled rotation is its own block-diagonal form; bad arguments are rejected."""
    import paper_1601_07384_gb300 as g
    th = 0.7
    K = 2.0 * np.array([[np.cos(th), np.sin(th), 0.0], [-np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 0.5]])
    P = np.array([[1.0, 2.0, 0.0], [0.0, 1.0, 1.0], [1.0, 0.0, 3.0]])
    W, Wi, R, pair = g.time_blockdiag(P @ K @ np.linalg.inv(P))
    assert sorted(np.round(np.linalg.eigvals(R), 10), key=lambda z: (z.real, z.imag)) == \
        sorted(np.round(np.linalg.eigvals(K), 10), key=lambda z: (z.real, z.imag))
    assert int(pair.sum()) == 1
    with pytest.raises(g.StdgError):
        g.time_blockdiag(np.eye(6))


@pytest.mark.parametrize("n", [4, 9, 20])
def test_agglomerates_of_a_kuhn_mesh(lib, n):
    """stdg_mesh_agglomerate (host logic of the KRON_MG coarse correction): on the 6 n^3 jittered
    Kuhn tets the first level is exactly each hexahedron's 6 tets, every next level the 2 x 2 x 2
    blocks of the previous one (partly filled when n is odd), each level partitions the previous
    one, and the last is the first with at most 512 cells."""
    import paper_1601_07384_gb300 as g
    from inputs import kuhn_mesh
    v, t = kuhn_mesh(n, seed=0)
    cells, sizes = g.Mesh(v, t).agglomerate()
    ne = 6 * n ** 3
    hexid = np.arange(ne) // 6                       # tet id = 6 (i + n (j + n k)) + permutation
    hi, hj, hk = hexid % n, (hexid // n) % n, hexid // (n * n)
    assert sizes[0] == n ** 3
    assert len(set(zip(cells[0].tolist(), hexid.tolist()))) == n ** 3
    for lvl in range(1, len(sizes)):
        s = 2 ** lvl
        m = (n + s - 1) // s
        blk = (hi // s) + m * ((hj // s) + m * (hk // s))
        assert len(set(blk.tolist())) == sizes[lvl]
        assert len(set(zip(cells[lvl].tolist(), blk.tolist()))) == sizes[lvl]
        assert len(set(zip(cells[lvl - 1].tolist(), cells[lvl].tolist()))) == sizes[lvl - 1]
    assert sizes[-1] <= 512 and (len(sizes) == 1 or sizes[-2] > 512)
    assert list(sizes) == {4: [64], 9: [729, 125], 20: [8000, 1000, 125]}[n]


def test_periodic_mesh_matches_oracle(lib):
    """stdg_mesh_create_periodic: the same face table as the oracle's periodic mesh (every face
    interior), and without a GPU the solver creation fails with STDG_ECUDA (no host path); on a
    GPU it is accepted."""
    import ctypes as C
    import paper_1601_07384_gb300 as g
    from paper_1601_07384_gb300 import _lib
    from inputs import kuhn_periodic_mesh
    from oracle.mesh import Mesh as OMesh
    v, t, per = kuhn_periodic_mesh(3)
    gm = g.Mesh(v, t, period=per)
    om = OMesh(v, t, period=per)
    left, right, lf, rf = gm.faces()
    assert gm.nf == om.nf == 2 * len(t) and gm.nboundary == 0
    assert np.array_equal(left, om.left) and np.array_equal(right, om.right)
    assert np.array_equal(lf, om.fl) and np.array_equal(rf, om.fr)
    h = C.c_void_p()
    st = _lib.load().stdg_solver_create(gm._h, g.Reference(1, 0)._h, 0.01, None, None, C.byref(h))
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        assert st == -3                             # STDG_ECUDA
    else:
        assert st == 0
        _lib.load().stdg_solver_destroy(h)
    with pytest.raises(g.StdgError):
        g.Mesh(v, t, period=[0.0, 1.0, 1.0])
