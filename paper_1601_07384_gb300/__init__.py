"""GB300 (sm_103a) implementation of the staggered space-time DG pressure-correction path
(Tavelli & Dumbser, arXiv:1601.07384) behind the C ABI of include/stdg.h.

This module only marshals arguments: every step of the path runs in libstdg.so's CUDA kernels.
PyTorch supplies device memory and the CUDA stream.  There is no CPU fallback: if the library
or a GPU is missing, the calls raise.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import ALLOC_FN, FIELD, FREE_FN, PREC, SOLVER, VEL_FN, Field, SolveStats, SolverOptions, StdgError, StepStats

__all__ = ["Mesh", "Reference", "Solver", "StdgError", "beltrami", "constant", "zero", "curl_modes", "nbasis",
           "time_blockdiag"]


def nbasis(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def beltrami(a=np.pi / 4, d=np.pi / 2, nu=0.1):
    f = Field(); f.kind = FIELD["beltrami"]; f.a = a; f.d = d; f.nu = nu
    return f


def constant(u):
    f = Field(); f.kind = FIELD["constant"]
    for k in range(3):
        f.c[k] = float(u[k])
    return f


def zero():
    f = Field(); f.kind = FIELD["zero"]
    return f


def curl_modes(k, A, phi, scale=1.0):
    """STDG_FIELD_CURL_MODES: v = scale curl(b Psi), Psi = Sum_m A_m sin(2 pi k_m . x + phi_m),
    b = (64 x(1-x) y(1-y) z(1-z))^2 on the unit cube (zero with its gradient on the walls)."""
    k = np.asarray(k, dtype=np.float64).reshape(-1, 3)
    A = np.asarray(A, dtype=np.float64).reshape(-1, 3)
    phi = np.asarray(phi, dtype=np.float64).reshape(-1, 1)
    rows = np.ascontiguousarray(np.concatenate([k, A, phi], axis=1))
    f = Field(); f.kind = FIELD["curl_modes"]; f.c[0] = float(scale)
    f.nmodes = rows.shape[0]
    f.modes = rows.ctypes.data_as(_lib.DP)
    f._rows = rows                      # keeps the host table alive while the Field is
    return f


def time_blockdiag(K):
    """Real block-diagonal form K = W R W^-1 (stdg_time_blockdiag): returns W, Winv, R, pair."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    n = K.shape[0]
    W, Wi, R = np.empty((n, n)), np.empty((n, n)), np.empty((n, n))
    pair = (C.c_int * n)()
    _lib.check(_lib.load().stdg_time_blockdiag(K.ctypes.data_as(_lib.DP), n, W.ctypes.data_as(_lib.DP),
                                               Wi.ctypes.data_as(_lib.DP), R.ctypes.data_as(_lib.DP), pair))
    return W, Wi, R, np.array(pair[:], dtype=np.int64)


class Mesh:
    """Primary tetrahedral mesh and its face-based dual grid (stdg_mesh_create)."""

    def __init__(self, verts, tets, period=None):
        lib = _lib.load()
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tets, dtype=np.int64)
        h = C.c_void_p()
        if period is None:
            _lib.check(lib.stdg_mesh_create(v.ctypes.data_as(_lib.DP), v.shape[0], t.ctypes.data_as(_lib.I64P),
                                            t.shape[0], C.byref(h)))
        else:
            per = np.ascontiguousarray(period, dtype=np.float64)
            _lib.check(lib.stdg_mesh_create_periodic(v.ctypes.data_as(_lib.DP), v.shape[0],
                                                     t.ctypes.data_as(_lib.I64P), t.shape[0],
                                                     per.ctypes.data_as(_lib.DP), C.byref(h)))
        self._h = h
        ne, nf, ni, nb = (C.c_int64() for _ in range(4))
        _lib.check(lib.stdg_mesh_info(h, C.byref(ne), C.byref(nf), C.byref(ni), C.byref(nb)))
        self.ne, self.nf, self.ninterior, self.nboundary = ne.value, nf.value, ni.value, nb.value

    def faces(self):
        lib = _lib.load()
        l = np.empty(self.nf, np.int64); r = np.empty(self.nf, np.int64)
        fl = np.empty(self.nf, np.int32); fr = np.empty(self.nf, np.int32)
        _lib.check(lib.stdg_mesh_faces(self._h, l.ctypes.data_as(_lib.I64P), r.ctypes.data_as(_lib.I64P),
                                       fl.ctypes.data_as(_lib.I32P), fr.ctypes.data_as(_lib.I32P)))
        return l, r, fl, fr

    def __del__(self):
        if getattr(self, "_h", None) and _lib._lib is not None:
            _lib._lib.stdg_mesh_destroy(self._h)
            self._h = None


    def agglomerate(self, coarse_max=512, max_levels=16):
        """stdg_mesh_agglomerate: (cells [levels x ne], sizes [levels]) of the nested agglomerates."""
        lib = _lib.load()
        ne = self.ne
        cell = np.empty(max_levels * ne, dtype=np.int32)
        sizes = np.empty(max_levels, dtype=np.int64)
        lv = C.c_int()
        _lib.check(lib.stdg_mesh_agglomerate(self._h, int(coarse_max), int(max_levels),
                                             cell.ctypes.data_as(C.POINTER(C.c_int32)),
                                             sizes.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(lv)))
        L = lv.value
        return cell[:L * ne].reshape(L, ne), sizes[:L]

class Reference:
    """Reference quadrature / basis tables and the time matrix K (stdg_reference_matrices)."""

    def __init__(self, p, pt):
        lib = _lib.load()
        h = C.c_void_p()
        _lib.check(lib.stdg_reference_matrices(int(p), int(pt), C.byref(h)))
        self._h, self.p, self.pt = h, p, pt
        self.N, self.Ng = nbasis(p), pt + 1
        self.Nst = self.N * self.Ng

    def time_matrix(self):
        K = np.empty((self.Ng, self.Ng))
        _lib.check(_lib.load().stdg_ref_time_matrix(self._h, K.ctypes.data_as(_lib.DP)))
        return K

    def time_blockdiag(self):
        """stdg_time_blockdiag of this reference's K: (W, Winv, R, pair) with K = W R W^-1."""
        return time_blockdiag(self.time_matrix())

    def eval(self, xi):
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        phi = np.empty((len(xi), self.N)); dphi = np.empty((len(xi), 3, self.N))
        _lib.check(_lib.load().stdg_ref_eval(self._h, xi.ctypes.data_as(_lib.DP), len(xi),
                                             phi.ctypes.data_as(_lib.DP), dphi.ctypes.data_as(_lib.DP)))
        return phi, dphi

    def __del__(self):
        if getattr(self, "_h", None) and _lib._lib is not None:
            _lib._lib.stdg_ref_destroy(self._h)
            self._h = None


def tc_gemm_bf16(A, B):
    """D = A B^T on the tensor cores (stdg_tc_gemm_bf16): A (M, K), B (N, K) contiguous float32 CUDA
    tensors, rounded to bfloat16; binary32 sums; N <= 256."""
    torch = _torch()
    assert A.is_cuda and B.is_cuda and A.dtype == torch.float32 and B.dtype == torch.float32
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty(M, N, dtype=torch.float32, device=A.device)
    _lib.check(_lib.load().stdg_tc_gemm_bf16(_ptr(A), K, _ptr(B), K, _ptr(D), N, M, N, K,
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return D


def fma_probe():
    """(binary64, binary32) FMA throughput of the current device in TFLOP/s (stdg_fma_probe)."""
    torch = _torch()
    a, b = C.c_double(), C.c_double()
    _lib.check(_lib.load().stdg_fma_probe(C.byref(a), C.byref(b), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return a.value, b.value


def tet_rule(n):
    """Collapsed Gauss-Jacobi tetrahedron rule of the library (host code)."""
    xi = np.empty((n ** 3, 3)); w = np.empty(n ** 3)
    _lib.check(_lib.load().stdg_tet_rule(int(n), xi.ctypes.data_as(_lib.DP), w.ctypes.data_as(_lib.DP)))
    return xi, w


class Solver:
    """Device-resident discretisation: blocks, state and Krylov workspace (stdg_solver_create).

    allocator="torch" (default): every device array of the solver comes from PyTorch's caching
    allocator (stdg_solver_create_alloc with callbacks into torch.cuda.caching_allocator_alloc /
    caching_allocator_delete); allocator="cuda": the library calls cudaMalloc itself.  The callbacks
    count what they hand out: alloc_stats() gives the live bytes and the allocation count."""

    def __init__(self, mesh: Mesh, ref: Reference, dt, precision="fp64", restart=50, max_iters=200000,
                 stream=None, graph_batch=8, allocator="torch"):
        torch = _torch()
        lib = _lib.load()
        self.mesh, self.ref = mesh, ref
        self.N, self.Ng, self.Nst = ref.N, ref.Ng, ref.Nst
        self.ne, self.nf = mesh.ne, mesh.nf
        self.dt = float(dt)
        self._cb_error = None
        self._live = {}
        self._nalloc = [0]
        opts = SolverOptions(PREC[precision], int(restart), int(max_iters), int(graph_batch))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        if allocator == "torch":
            dev = torch.cuda.current_device()
            live, count = self._live, self._nalloc          # no reference to self: no cycle

            def _alloc(nbytes, stream, user):
                try:
                    p = torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=int(stream or 0))
                except Exception:                       # the library reports STDG_ENOMEM
                    return None
                live[int(p)] = int(nbytes)
                count[0] += 1
                return p

            def _free(ptr, nbytes, stream, user):
                try:
                    live.pop(int(ptr), None)
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:                       # interpreter shutdown: torch may be gone
                    pass

            self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
            _lib.check(lib.stdg_solver_create_alloc(mesh._h, ref._h, self.dt, C.byref(opts),
                                                    C.c_void_p(self.stream.cuda_stream), self._alloc_cb,
                                                    self._free_cb, None, C.byref(h)))
        elif allocator == "cuda":
            _lib.check(lib.stdg_solver_create(mesh._h, ref._h, self.dt, C.byref(opts),
                                              C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        else:
            raise ValueError(f"allocator must be 'torch' or 'cuda', not {allocator!r}")
        self._h = h

    def alloc_stats(self):
        """(live bytes, allocations so far) handed out through the allocator callbacks."""
        return sum(self._live.values()), self._nalloc[0]

    def _vel_callback(self, fn):
        """stdg_vel_fn around fn(x (n, 3), t (n,)) -> (n, 3); an exception is re-raised after the call."""
        def cb(xyzt, n, uvw, user):
            out = np.ctypeslib.as_array(uvw, shape=(n, 3))
            try:
                X = np.ctypeslib.as_array(xyzt, shape=(n, 4))
                out[:] = np.asarray(fn(X[:, :3].copy(), X[:, 3].copy()), dtype=np.float64).reshape(n, 3)
            except BaseException as exc:                # surfaced by _check_cb
                self._cb_error = exc
                out[:] = np.nan
        return VEL_FN(cb)

    def _check_cb(self, status):
        err, self._cb_error = self._cb_error, None
        if err is not None:
            raise err
        _lib.check(status)

    # ---------------------------------------------------------------- helpers
    def pressure_empty(self):
        torch = _torch()
        return torch.empty(self.ne * self.Nst, dtype=torch.float64, device="cuda")

    def velocity_empty(self):
        torch = _torch()
        return torch.empty(self.nf * 3 * self.Nst, dtype=torch.float64, device="cuda")

    @staticmethod
    def _dev(t):
        torch = _torch()
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "expect contiguous cuda float64"
        return t

    # ---------------------------------------------------------------- hot path
    def set_dt(self, dt):
        self.dt = float(dt)
        _lib.check(_lib.load().stdg_set_dt(self._h, self.dt))

    def set_max_iters(self, n):
        _lib.check(_lib.load().stdg_set_max_iters(self._h, int(n)))

    def pressure_apply(self, x, y=None, pinned=True):
        x = self._dev(x)
        y = self.pressure_empty() if y is None else self._dev(y)
        _lib.check(_lib.load().stdg_pressure_apply(self._h, _ptr(x), _ptr(y), int(bool(pinned))))
        return y

    def pressure_apply_factored(self, x, y=None, pinned=True):
        """Factored-form cross-check of the operator (gradient, M_j^-1, divergence per dual cell)."""
        x = self._dev(x)
        y = self.pressure_empty() if y is None else self._dev(y)
        _lib.check(_lib.load().stdg_pressure_apply_factored(self._h, _ptr(x), _ptr(y), int(bool(pinned))))
        return y

    def pressure_apply_f32(self, x, y=None, pinned=True):
        torch = _torch()
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        y = torch.empty_like(x) if y is None else y
        _lib.check(_lib.load().stdg_pressure_apply_f32(self._h, _ptr(x), _ptr(y), int(bool(pinned))))
        return y

    def pressure_rhs(self, F, b=None, pinned=True):
        F = self._dev(F)
        b = self.pressure_empty() if b is None else self._dev(b)
        _lib.check(_lib.load().stdg_pressure_rhs(self._h, _ptr(F), _ptr(b), int(bool(pinned))))
        return b

    def velocity_update(self, F, dp, V=None):
        F, dp = self._dev(F), self._dev(dp)
        V = self.velocity_empty() if V is None else self._dev(V)
        _lib.check(_lib.load().stdg_velocity_update(self._h, _ptr(F), _ptr(dp), _ptr(V)))
        return V

    def solve(self, b, tol=1e-10, method="kron_cg", x=None):
        b = self._dev(b)
        x = self.pressure_empty() if x is None else self._dev(x)
        st = SolveStats()
        _lib.check(_lib.load().stdg_solve(self._h, _ptr(b), _ptr(x), float(tol), SOLVER[method], C.byref(st)))
        return x, {"iterations": st.iterations, "restarts": st.restarts, "rel_residual": st.rel_residual,
                   "seconds": st.seconds, "fallback": st.fallback}

    def solve_noalloc(self, b, x, tol=1e-10):
        """stdg_solve_noalloc: the Kronecker-decoupled CG solve without any device allocation
        (the caller supplies x; work vectors live in a fixed array inside the library)."""
        st = SolveStats()
        _lib.check(_lib.load().stdg_solve_noalloc(self._h, _ptr(self._dev(b)), _ptr(self._dev(x)), float(tol),
                                                  C.byref(st)))
        return x, {"iterations": st.iterations, "restarts": st.restarts, "rel_residual": st.rel_residual,
                   "seconds": st.seconds}

    def velocity_moments(self, V, U=None):
        torch = _torch()
        V = self._dev(V)
        U = torch.empty(self.nf * 6 * self.Nst, dtype=torch.float64, device="cuda") if U is None else U
        _lib.check(_lib.load().stdg_velocity_moments(self._h, _ptr(V), _ptr(U)))
        return U

    def convection(self, vbar, ups=None):
        """The convective term of Eq. convdg for velocity averages vbar ([3][ne][Nst] on the device) on
        the slab starting at the current time, with the boundary field's Dirichlet data."""
        torch = _torch()
        vbar = self._dev(vbar)
        ups = torch.empty(3 * self.ne * self.Nst, dtype=torch.float64, device="cuda") if ups is None else ups
        _lib.check(_lib.load().stdg_convection(self._h, _ptr(vbar), _ptr(ups)))
        return ups

    # ---------------------------------------------------------------- time stepping
    def set_initial(self, field):
        """Initial velocity: a device field kind (Field), or a host callable fn(x (n, 3), t (n,)) -> (n, 3)
        evaluated at the projection's quadrature points (stdg_set_initial_fn)."""
        if callable(field):
            cb = self._vel_callback(field)
            self._check_cb(_lib.load().stdg_set_initial_fn(self._h, cb, None))
        else:
            _lib.check(_lib.load().stdg_set_initial(self._h, C.byref(field)))

    def set_boundary(self, field):
        """Dirichlet velocity: a device field kind, or a host callable evaluated at every step's boundary
        quadrature points (stdg_set_boundary_fn)."""
        if callable(field):
            self._bc_cb = self._vel_callback(field)          # called from every stdg_step
            self._check_cb(_lib.load().stdg_set_boundary_fn(self._h, self._bc_cb, None))
        else:
            _lib.check(_lib.load().stdg_set_boundary(self._h, C.byref(field)))
            self._bc_cb = None

    def step(self, nu, n_picard, method="kron_cg", tol=1e-10):
        st = StepStats()
        self._check_cb(_lib.load().stdg_step(self._h, float(nu), int(n_picard), SOLVER[method], float(tol),
                                             C.byref(st)))
        k = st.picard
        return {"picard": k, "press_iters": list(st.press_iters[:k]), "visc_iters": list(st.visc_iters[:k]),
                "press_residual": list(st.press_residual[:k]), "seconds": st.seconds,
                "max_divergence": st.max_divergence, "fallbacks": st.fallbacks}

    def set_theta(self, theta):
        """Semi-implicit pressure weight of the theta method (p_t = 0; 1 = fully implicit)."""
        _lib.check(_lib.load().stdg_set_theta(self._h, float(theta)))

    def get_state(self):
        torch = _torch()
        P, V = self.pressure_empty(), self.velocity_empty()
        t = C.c_double()
        _lib.check(_lib.load().stdg_get_state(self._h, _ptr(P), _ptr(V), 1, C.byref(t)))
        return P, V, t.value

    def set_state(self, P, V, t):
        _lib.check(_lib.load().stdg_set_state(self._h, _ptr(self._dev(P)), _ptr(self._dev(V)), 1, float(t)))

    # ---------------------------------------------------------------- learned preconditioner
    def gnn_init(self, hidden=64, layers=3, bf16=True, seed=0):
        _lib.check(_lib.load().stdg_gnn_init(self._h, int(hidden), int(layers), int(bool(bf16)), int(seed)))

    def gnn_layout(self):
        L = C.c_int(); H = C.c_int(); F = C.c_int()
        offs = (C.c_int64 * 64)()
        _lib.check(_lib.load().stdg_gnn_layout(self._h, offs, C.byref(H), C.byref(L), C.byref(F)))
        n = 2 + 3 * L.value + 2
        return {"offsets": list(offs[:n]), "hidden": H.value, "layers": L.value, "nfeat": F.value}

    def gnn_params(self, w_in=None):
        npar = C.c_int64()
        _lib.check(_lib.load().stdg_gnn_params(self._h, None, None, C.byref(npar)))
        out = np.empty(npar.value, dtype=np.float32)
        win = None
        if w_in is not None:
            win = np.ascontiguousarray(w_in, dtype=np.float32)
        _lib.check(_lib.load().stdg_gnn_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)),
                                               None if win is None else win.ctypes.data_as(C.POINTER(C.c_float)),
                                               C.byref(npar)))
        return out

    def gnn_apply(self, r, z=None):
        z = self.pressure_empty() if z is None else z
        _lib.check(_lib.load().stdg_gnn_apply(self._h, _ptr(self._dev(r)), _ptr(self._dev(z))))
        return z

    def gnn_loss_grad(self, R, T, npairs):
        npar = C.c_int64()
        _lib.check(_lib.load().stdg_gnn_params(self._h, None, None, C.byref(npar)))
        g = np.empty(npar.value, dtype=np.float32)
        loss = C.c_double()
        _lib.check(_lib.load().stdg_gnn_loss_grad(self._h, _ptr(self._dev(R)), _ptr(self._dev(T)), int(npairs),
                                                  C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def gnn_harvest(self, b, nsnap=10, every=20, max_pairs=64):
        tot = C.c_int()
        _lib.check(_lib.load().stdg_gnn_harvest(self._h, _ptr(self._dev(b)), int(nsnap), int(every), int(max_pairs),
                                                C.byref(tot)))
        return tot.value

    def gnn_autoharvest(self, nsnap=8, every=50, max_pairs=64):
        _lib.check(_lib.load().stdg_gnn_autoharvest(self._h, int(nsnap), int(every), int(max_pairs)))

    def gnn_autoharvest_mg(self, nsnap=8, max_pairs=64):
        """Harvest (residual, missed error) pairs from the outer iterations of the mixed KRON_MG solves."""
        _lib.check(_lib.load().stdg_gnn_autoharvest_mg(self._h, int(nsnap), int(max_pairs)))

    def gnn_train(self, epochs=50, lr=1e-3, batch=4):
        a = C.c_double(); b = C.c_double()
        _lib.check(_lib.load().stdg_gnn_train(self._h, int(epochs), float(lr), int(batch), C.byref(a), C.byref(b)))
        return a.value, b.value

    def profile(self, enable=True):
        _lib.check(_lib.load().stdg_profile(self._h, int(bool(enable))))

    def profile_read(self):
        st = _lib.ProfileStats()
        _lib.check(_lib.load().stdg_profile_read(self._h, C.byref(st)))
        return {"kernel_launches": st.kernel_launches, "operator_launches": st.operator_launches,
                "operator_ms": st.operator_ms, "kind_launches": list(st.kind_launches), "kind_ms": list(st.kind_ms),
                "phase_ms": list(st.phase_ms)}

    def blocks(self):
        N, nf, ne = self.N, self.nf, self.ne
        Q = np.empty((nf, 2, 3, N, N)); Mij = np.empty((nf, 2, N, N))
        A = np.empty((nf, N, N)); B = np.empty((ne, N, N))
        _lib.check(_lib.load().stdg_get_blocks(self._h, Q.ctypes.data_as(_lib.DP), Mij.ctypes.data_as(_lib.DP),
                                               A.ctypes.data_as(_lib.DP), B.ctypes.data_as(_lib.DP)))
        return {"Q": Q, "Mij": Mij, "Aoff": A, "Bdiag": B}

    def __del__(self):
        if getattr(self, "_h", None) and _lib._lib is not None:
            _lib._lib.stdg_solver_destroy(self._h)
            self._h = None
