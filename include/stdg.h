/*
 * stdg.h -- C ABI of the GB300 (sm_103a) implementation of the staggered semi-implicit
 * space-time DG pressure-correction scheme for the 3D incompressible Navier-Stokes
 * equations on tetrahedral meshes (Tavelli & Dumbser, arXiv:1601.07384).
 *
 * Conventions shared by every call
 *  - All floating point data is IEEE binary64 unless a call says otherwise.
 *  - Pointers named *_dev are raw CUDA device pointers on the solver's device; pointers
 *    named *_host are host pointers.  The caller owns every buffer it passes; the library
 *    reads inputs during the call (stream-ordered for device buffers) and never keeps them.
 *  - The library owns the objects it returns and the device arrays inside them; free them
 *    with the matching *_destroy call.
 *  - Device work is issued on the CUDA stream given to stdg_solver_create, in order.
 *  - Nothing aborts or throws across this boundary: every call returns a stdg_status; on a
 *    negative status stdg_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread).  There is no CPU fallback: a missing GPU is STDG_ECUDA.
 *  - Index conventions (Sec. 2.2-2.3 of the paper):
 *      N  = (p+1)(p+2)(p+3)/6 spatial basis functions, Ng = p_t + 1 time functions,
 *      Nst = N * Ng; a space-time coefficient (time a, space k) sits at a*N + k.
 *      Tet basis: orthonormal Dubiner on {xi,eta,zeta >= 0, xi+eta+zeta <= 1}; multi-index
 *      order "for n=0..p, i=0..n, j=0..n-i: (i, j, n-i-j)".  Time basis: orthonormal
 *      Legendre on [0,1].  Dual basis: the paper's scaled Taylor monomials (Eq. bf_2),
 *      Gram-Schmidt orthonormalised on each dual cell in the same multi-index order.
 *      Faces are numbered by increasing (l(j), local face of l(j)), l(j) = lower tet id;
 *      local face f of a tet is the face opposite its local vertex f.
 *  - Array layouts:  pressure  P[ne][Ng][N];  velocity on dual cells V[nf][3][Ng][N];
 *      averaged velocity on tets Vbar[ne][3][Ng][N].
 */
#ifndef STDG_H
#define STDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stdg_mesh stdg_mesh;
typedef struct stdg_ref stdg_ref;
typedef struct stdg_solver stdg_solver;

typedef enum {
  STDG_OK = 0,
  STDG_EINVAL = -1,       /* bad argument                                              */
  STDG_ENOMEM = -2,       /* host or device allocation failed                          */
  STDG_ECUDA = -3,        /* a CUDA runtime call failed (including: no usable GPU)     */
  STDG_ENOCONV = -4,      /* Krylov iteration cap reached; stats are filled in         */
  STDG_EMESH = -5,        /* inverted / degenerate tet or non-manifold face            */
  STDG_ENAN = -6,         /* a non-finite value appeared in a solve                    */
  STDG_ETIMEOUT = -7,     /* reserved: a bounded device wait gave up                   */
  STDG_EUNSUPPORTED = -8  /* degree or option outside what this build supports         */
} stdg_status;

/* Krylov methods for stdg_solve.
 *  STDG_SOLVER_GMRES : restarted GMRES(m) on the full space-time pressure operator with
 *                      classical Gram-Schmidt applied twice, as the paper's matrix-free,
 *                      unpreconditioned GMRES (abstract; Sec. 2.4, 2.7).
 *  STDG_SOLVER_CG    : conjugate gradients on -A; only for p_t = 0 (Sec. 2.7, Cor. 1-2).
 *  STDG_SOLVER_KRON_CG: the same pinned system solved exactly as Ng decoupled symmetric
 *                      positive definite systems: with the orthonormal bases used here the
 *                      operator of Eq. CS_19 factors as A = A_sp (x) dt^2 K^-1, so
 *                      A x = b  <=>  A_sp X = B K^T / dt^2 column by column (block CG, all
 *                      columns share each operator launch).  The stopping test is on the
 *                      residual of the full system, as for the other methods.
 *  STDG_SOLVER_KRON_PCG: STDG_SOLVER_KRON_CG preconditioned by block Jacobi: the exact inverse
 *                      of each tet's N x N diagonal block of the pinned -A_sp (built on first
 *                      use, Cholesky on the device).  The paper uses no preconditioner; this
 *                      changes only the iteration, not the system or its stopping test.
 *  STDG_SOLVER_KRON_MG: STDG_SOLVER_KRON_PCG with an additive coarse correction on the
 *                      constant mode of every tet: z = Binv r + R^T V (R r), R the constant-mode
 *                      coefficients (pinned one excluded), V one symmetric V-cycle (a damped
 *                      Jacobi sweep before and after, exact dense solve on the coarsest level)
 *                      over nested agglomerates of tets (centroids binned into cubes of the mean
 *                      hexahedron size, doubled per level) with Galerkin coarse matrices.  The
 *                      hierarchy is built on first use (host setup, a few device arrays).
 *                      Same system and stopping test; O(1) iterations in h where block Jacobi
 *                      needs O(1/h).  With the MIXED precisions it preconditions the inner
 *                      binary32 iterations.                                                  */
/*  STDG_SOLVER_FGMRES_BJ / STDG_SOLVER_FGMRES_GNN : flexible GMRES(m) on the full operator,
 *                      right-preconditioned by block Jacobi of the full operator
 *                      (A_ii^-1 = B_i^-1 (x) (dt^2 K^-1)^-1) alone, or, for FGMRES_GNN, with
 *                      the first direction of every restart cycle (the normalised residual)
 *                      preconditioned by block Jacobi plus the learned network correction
 *                      (stdg_gnn_*); later Arnoldi vectors use block Jacobi.  Needs
 *                      stdg_gnn_init.                                                      */
/*  STDG_SOLVER_KRON_MG_GNN : STDG_SOLVER_KRON_MG in a mixed precision in which every inner-solve step
 *                      of the binary64 flexible outer iteration is followed by a step along the learned
 *                      network's direction z = RMS(r) net(r / RMS(r)), S-orthogonalised against the
 *                      stored directions like any other: the error it leaves is the energy minimum over
 *                      the enlarged search space, so the network can save inner-solve steps but never
 *                      make a step worse; each network step costs one binary64-accurate operator
 *                      application.  The network is trained on (residual, error) pairs from the outer
 *                      iterations of earlier solves (stdg_gnn_autoharvest_mg).  A network step whose
 *                      output is not finite or vanishes is skipped; stdg_solve_stats.fallback counts
 *                      them.  stdg_solve_stats.restarts counts all outer steps.  Needs stdg_gnn_init.  */
enum { STDG_SOLVER_GMRES = 0, STDG_SOLVER_CG = 1, STDG_SOLVER_KRON_CG = 2, STDG_SOLVER_KRON_PCG = 3,
       STDG_SOLVER_FGMRES_BJ = 4, STDG_SOLVER_FGMRES_GNN = 5, STDG_SOLVER_KRON_MG = 6, STDG_SOLVER_KRON_MG_GNN = 7 };

/* Precision of the operator blocks used inside the Krylov iteration (stdg_solver_options).
 *  STDG_PREC_FP64   : blocks and arithmetic in binary64.
 *  STDG_PREC_DF32   : binary64 blocks and vectors, products formed in pairs of binary32
 *                     ("double-float", ~48-bit significand) because sm_103a's binary64
 *                     pipe is 1/64 of its binary32 rate; results agree with STDG_PREC_FP64
 *                     to ~1e-14 relative per operator application.  Used for the pressure
 *                     and the viscous operators inside the solves.  Where that kernel would
 *                     run fewer than 6 warps per SM (its shared memory per warp grows as N^2:
 *                     p >= 4), the binary64 kernel serves instead; the results are the same.
 *  STDG_PREC_MIXED_F32 / STDG_PREC_MIXED_BF16 : the Kronecker CG methods run as an inner-outer
 *                     iteration: flexible CG in binary64 (operator as in STDG_PREC_DF32)
 *                     preconditioned by a fixed number of block-Jacobi CG iterations whose
 *                     operator blocks are binary32 / bfloat16 (vectors and accumulation
 *                     binary32).  Residual recurrence, scalars and stopping test are binary64,
 *                     so the returned x meets the same FP64 residual tolerance.  With
 *                     STDG_SOLVER_KRON_MG the inner iterations add the coarse correction.
 *                     With STDG_PREC_MIXED_F32 the viscous solves of stdg_step are a binary64
 *                     refinement (residual with the STDG_PREC_DF32 operator) around binary32
 *                     inner solves; with STDG_PREC_MIXED_BF16 they use the STDG_PREC_DF32
 *                     operator.  stdg_solve_stats.iterations counts the binary32 iterations
 *                     and .restarts the outer ones.                                          */
enum { STDG_PREC_FP64 = 0, STDG_PREC_DF32 = 1, STDG_PREC_MIXED_F32 = 2, STDG_PREC_MIXED_BF16 = 3 };

typedef struct {
  int iterations;          /* Krylov iterations (operator applications in the loop)   */
  int restarts;            /* GMRES restarts                                          */
  double rel_residual;     /* ||b - A x|| / ||b|| of the returned x                   */
  double seconds;          /* wall time of the call                                   */
  int fallback;            /* 1 if FGMRES with the learned preconditioner failed (stall /
                              non-finite value) and plain GMRES produced the result          */
} stdg_solve_stats;

typedef struct {
  int picard;              /* Picard iterations done                                  */
  int press_iters[8];      /* pressure Krylov iterations per Picard iteration         */
  int visc_iters[8];       /* viscous Krylov iterations (sum over 3 components)       */
  double press_residual[8];/* final relative residual of each pressure solve          */
  double seconds;          /* wall time of the step                                   */
  double max_divergence;   /* max_i |Sum_j D_ij v_j| over unpinned tets after the step */
  int fallbacks;           /* pressure solves that fell back to plain GMRES               */
} stdg_step_stats;

/* Velocity data kinds for initial and Dirichlet boundary values (evaluated on the device; the data
 * of the problem statement, Sec. 2.4: initial velocity and prescribed boundary velocity).
 *  STDG_FIELD_ZERO     : v = 0 (no-slip walls).
 *  STDG_FIELD_CONSTANT : v = (c0, c1, c2).
 *  STDG_FIELD_BELTRAMI : Ethier-Steinman unsteady solution, params (a, d, nu):
 *      u = -a [e^{ax} sin(ay+dz) + e^{az} cos(ax+dy)] e^{-nu d^2 t}, v, w by cyclic shift.
 *  STDG_FIELD_CURL_MODES : the steady solenoidal field v = c0 curl(b Psi) of the unit cube, with
 *      Psi(x) = Sum_m A_m sin(2 pi k_m . x + phi_m) and b = B^2, B = 64 x(1-x) y(1-y) z(1-z): b and
 *      grad b vanish on the walls, so v = 0 there (no-slip compatible) and div v = 0 exactly.
 *      `modes` points to nmodes host rows (k_m[3], A_m[3], phi_m) of 7 doubles (1 <= nmodes <= 256);
 *      the call that receives the field copies them.
 * Data that none of these kinds covers comes through a host callback (stdg_vel_fn below). */
enum { STDG_FIELD_ZERO = 0, STDG_FIELD_CONSTANT = 1, STDG_FIELD_BELTRAMI = 2, STDG_FIELD_CURL_MODES = 3 };
typedef struct { int kind; double c[3]; double a, d, nu; int nmodes; const double* modes; } stdg_field;

/* Host velocity callback: fill uvw_host[n][3] with the velocity at the n space-time points
 * xyzt_host[n][4] = (x, y, z, t).  Both arrays are host memory owned by the library and valid only
 * during the call; `user` is passed through unchanged.  The callback must not call back into the
 * library. */
typedef void (*stdg_vel_fn)(const double* xyzt_host, int64_t n, double* uvw_host, void* user);

/* Device allocator callbacks (stdg_solver_create_alloc): return `bytes` of device memory on the
 * solver's device, usable on `stream` (the solver's stream), aligned to at least 256 bytes, or NULL
 * on failure; free a pointer that alloc returned (with its size and the same stream).  Lets the
 * caller's allocator own every device array of the solver, e.g. PyTorch's caching allocator. */
typedef void* (*stdg_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*stdg_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* ---------------------------------------------------------------- mesh (Sec. 2.2) */
/* Build the primary mesh and its face-based dual grid: faces from sorted vertex triples,
 * l(j) = lower tet id, r(j) = higher (-1 on the boundary), unit normals n_j from l to r,
 * sub-tetrahedra T_{i,j} (face j + barycentre of T_i).  verts_host[nv][3], tets_host[ne][4]
 * (0-based vertex ids, any orientation: a negative orientation is rejected as STDG_EMESH,
 * as are zero volumes and faces shared by more than two tets).  Host-only; no GPU needed. */
stdg_status stdg_mesh_create(const double* verts_host, int64_t nv, const int64_t* tets_host,
                             int64_t ne, stdg_mesh** out);
/* The same for a periodic box (the convergence test of Sec. 3.2): verts_host are the nv lattice
 * points of the box, tets_host index them (a vertex on a far face is the periodic image of one
 * on the near face), period_host[3] > 0 the box lengths.  A tet's geometry is its vertices'
 * periodic images nearest to its first vertex; faces are matched by vertex ids, so every face is
 * interior; face geometry is taken in l(j)'s frame, and every point of r(j) that meets face j (its
 * barycentre, the quadrature points of T_{r,j}) is moved into that frame by a period vector.  Host-only;
 * stdg_solver_create accepts the result like any mesh (no boundary faces: no Dirichlet data). */
stdg_status stdg_mesh_create_periodic(const double* verts_host, int64_t nv, const int64_t* tets_host,
                                      int64_t ne, const double* period_host, stdg_mesh** out);
void stdg_mesh_destroy(stdg_mesh* mesh);
stdg_status stdg_mesh_info(const stdg_mesh* mesh, int64_t* ne, int64_t* nfaces,
                           int64_t* ninterior, int64_t* nboundary);
/* Face table in face order: left[nf], right[nf] (-1 = boundary), lface[nf], rface[nf]
 * (local face indices, -1 on the boundary).  Any output pointer may be NULL. */
stdg_status stdg_mesh_faces(const stdg_mesh* mesh, int64_t* left_host, int64_t* right_host,
                            int32_t* lface_host, int32_t* rface_host);

/* Nested agglomerates of the mesh's tets: the coarse levels of STDG_SOLVER_KRON_MG.  Tet centroids
 * are binned into cubes of edge h = cbrt(mean |det J_i|) (6 x the mean tet volume: the hexahedron
 * edge of a Kuhn mesh) anchored at the lower corner of the vertices' bounding box, then into cubes
 * of edge 2h, 4h, ...; a size that merges no bins is skipped; it stops at the first level with at
 * most coarse_max cells, or after max_levels levels.  Out (caller-owned host arrays):
 * cell_host[l * ne + i] = cell of tet i on level l + 1 (cells numbered 0, 1, ... in bin order),
 * sizes_host[l] = cells on level l + 1, for l < *levels (arrays of max_levels * ne and max_levels
 * entries).  STDG_EINVAL on a NULL pointer or a limit < 1; STDG_EUNSUPPORTED (outputs filled) if
 * max_levels levels still leave more than coarse_max cells.  Host-only. */
stdg_status stdg_mesh_agglomerate(const stdg_mesh* mesh, int coarse_max, int max_levels, int32_t* cell_host,
                                  int64_t* sizes_host, int* levels);

/* ------------------------------------------------ reference matrices (Sec. 2.3-2.4) */
/* Quadrature rules, Dubiner / Legendre tables and the time matrices
 * K_ab = gamma_a(1) gamma_b(1) - int_0^1 gamma_a' gamma_b (from Eqs. MD_2, MD_2_2).
 * Supported: 0 <= p <= 4, 0 <= p_t <= 4 (STDG_EUNSUPPORTED otherwise).  Host-only. */
stdg_status stdg_reference_matrices(int p, int p_t, stdg_ref** out);
void stdg_ref_destroy(stdg_ref* ref);
/* K into K_host[Ng*Ng] (row a, column b). */
stdg_status stdg_ref_time_matrix(const stdg_ref* ref, double* K_host);
/* Real block-diagonal form of an Ng x Ng real matrix (1 <= Ng <= 5), K = W R W^-1, used to
 * decouple the viscous systems of Eq. A1_mod in time: R has a 2 x 2 block [[a, b], [-b, a]] for
 * every complex eigenvalue pair a +- ib (the columns of W are the real and imaginary parts of the
 * eigenvector of a + ib) and a 1 x 1 block for every real eigenvalue; pair_host[c] = 1 marks the
 * first column of a 2 x 2 block, 0 otherwise.  All arrays row-major, caller-owned, host memory:
 * K_host[Ng*Ng] in; W_host, Winv_host, R_host [Ng*Ng] and pair_host[Ng] out.  STDG_EINVAL on a
 * NULL pointer or Ng out of range; STDG_EUNSUPPORTED if the decomposition fails its own check
 * (||K W - W R|| <= 1e-10 max(||K W||, 1), infinity-norm condition number of W <= 1e6), e.g.
 * for a defective K.  Host-only. */
stdg_status stdg_time_blockdiag(const double* K_host, int Ng, double* W_host, double* Winv_host,
                                double* R_host, int* pair_host);
/* Evaluate the reference tet basis (Sec. 2.3) at n points xi_host[n][3] of the reference
 * tetrahedron: phi_host[n][N] and reference gradients dphi_host[n][3][N] (either may be NULL).
 * Points on the edge eta + zeta = 1 or at zeta = 1 are outside the collapsed map: EINVAL. */
stdg_status stdg_ref_eval(const stdg_ref* ref, const double* xi_host, int64_t n, double* phi_host,
                          double* dphi_host);
/* The tetrahedron quadrature rule with `npts1d` points per direction (collapsed Gauss-Jacobi
 * product, exact to total degree 2*npts1d-1): xi_host[npts1d^3][3], w_host[npts1d^3], weights
 * summing to 1/6.  Host-only. */
stdg_status stdg_tet_rule(int npts1d, double* xi_host, double* w_host);

/* ------------------------------------------------------------------ solver objects */
typedef struct {
  int precision;           /* STDG_PREC_FP64 (default) or STDG_PREC_DF32              */
  int restart;             /* GMRES restart length m (default 50)                     */
  int max_iters;           /* cap on Krylov iterations per solve (default 200000)     */
  int graph_batch;         /* CG iterations per CUDA-graph launch (default 8; 1 = no graphs,
                              one host check per iteration).  With B > 1 up to B-1 iterations
                              may run past convergence; they are counted in the stats.       */
} stdg_solver_options;

/* Upload mesh and reference tables to the current CUDA device and build every per-face
 * and per-tet coefficient block on it (the paper's preprocessing step, Sec. 4):
 * orthonormal dual basis, Q_{i,j} (Eq. MD_6, spatial part), M_{i,j} (Eq. vis3), and the
 * assembled five-point spatial blocks B_i and A_{l r} of Sum_j D M^-1 Q (Eq. CS_19).
 * cuda_stream may be NULL (default stream).  opts may be NULL (defaults).
 * Device memory: ~ (ne + nf) * N^2 * 8 * 4 bytes + nf * N^2 * 8 * 9 bytes. */
stdg_status stdg_solver_create(const stdg_mesh* mesh, const stdg_ref* ref, double dt,
                               const stdg_solver_options* opts, void* cuda_stream,
                               stdg_solver** out);
/* The same, with every device array of the solver (blocks, state, Krylov and step workspace, the
 * lazily built copies and hierarchies) obtained from alloc_fn(bytes, cuda_stream, user) and returned
 * through free_fn by stdg_solver_destroy, after the solver's stream has been synchronised.  alloc_fn
 * and free_fn must both be given (else STDG_EINVAL); a NULL return from alloc_fn is STDG_ENOMEM.
 * Allocation happens in this call and lazily in the first call that needs an array (stdg_step,
 * stdg_solve, ...), never during the library's own CUDA-graph captures.  Host pinned buffers, CUDA
 * events and graphs stay with the CUDA runtime; stdg_solve_noalloc never allocates. */
stdg_status stdg_solver_create_alloc(const stdg_mesh* mesh, const stdg_ref* ref, double dt,
                                     const stdg_solver_options* opts, void* cuda_stream, stdg_alloc_fn alloc_fn,
                                     stdg_free_fn free_fn, void* user, stdg_solver** out);
void stdg_solver_destroy(stdg_solver* s);
/* Change the time step (rebuilds only the Ng x Ng time factor dt^2 K^-1). */
stdg_status stdg_set_dt(stdg_solver* s, double dt);
/* Change the cap on Krylov iterations per solve (stdg_solver_options.max_iters); STDG_EINVAL if < 1. */
stdg_status stdg_set_max_iters(stdg_solver* s, int max_iters);

/* ---------------------------------------------------------------- hot-path kernels */
/* y = A x, the five-point block pressure operator of Eq. CS_19 / A2_mod (left-hand side):
 * (A x)_i = Sum_{j in S_i, interior} D_ij M_j^-1 (Q_ij x_i + Q_{p(i,j),j} x_{p(i,j)}).
 * Boundary dual cells carry prescribed velocity and add nothing to A.  pinned != 0:
 * the pressure is fixed at one point (abstract, Sec. 2.7) by eliminating the constant
 * Dubiner mode of tet 0 for every time function: x there is read as 0 and y there = -x.
 * x_dev, y_dev: P layout, ne*Nst doubles each, must not overlap. */
stdg_status stdg_pressure_apply(stdg_solver* s, const double* x_dev, double* y_dev, int pinned);

/* The same operator with binary32 vectors x_dev, y_dev (P layout, ne*Nst floats) and the
 * solver's low-precision blocks (binary32 or bfloat16 per its precision option, built on first
 * use; needs STDG_PREC_MIXED_F32 or STDG_PREC_MIXED_BF16, else STDG_EINVAL).  Accumulation is
 * binary32; each warp stages its tet's blocks into shared memory with TMA bulk copies. */
stdg_status stdg_pressure_apply_f32(stdg_solver* s, const float* x_dev, float* y_dev, int pinned);

/* The same operator (same pinning) applied in the factored form of Eq. CS_19 / A2_mod, as a
 * cross-check of the assembled blocks: for every interior dual cell j the gradient blocks of
 * its two tets, then M_j^-1 (v_j = -M_j^-1 (Q_lj x_l + Q_rj x_r)), then the divergence blocks back
 * into each tet (y_i = -Sum_j D_ij v_j).  It reads the stored Q_ij instead of B_i and A_lr
 * (about 4.6x the bytes of stdg_pressure_apply at N = 20), so it is not the production path.
 * x_dev, y_dev: P layout, distinct.  The first call allocates an internal P-layout and a
 * V-layout vector. */
stdg_status stdg_pressure_apply_factored(stdg_solver* s, const double* x_dev, double* y_dev, int pinned);

/* b = Sum_{j in S_i} D_ij F_j over all four faces of each tet (Eq. A2_mod right-hand side,
 * Eq. CS_15 left-hand side), with D_ij = -Q_ij^T.  F_dev: V layout (nf*3*Nst), b_dev: P
 * layout.  pinned != 0 zeroes b at the pinned entries. */
stdg_status stdg_pressure_rhs(stdg_solver* s, const double* F_dev, double* b_dev, int pinned);

/* Velocity update of Eq. A3_mod: v_j = F_j - M_j^-1 (Q_rj dp_r + Q_lj dp_l) on interior
 * faces; boundary dual cells copy F_j.  F_dev, V_dev: V layout; dp_dev: P layout.
 * V_dev may equal F_dev (in place). */
stdg_status stdg_velocity_update(stdg_solver* s, const double* F_dev, const double* dp_dev,
                                 double* V_dev);

/* Solve the pinned pressure system A x = b (Eq. A2_mod) to ||b - A x|| <= tol ||b||,
 * starting from x = 0, with `method` (STDG_SOLVER_*).  b_dev, x_dev: P layout.
 * Returns STDG_ENOCONV when max_iters is reached (x holds the last iterate). */
stdg_status stdg_solve(stdg_solver* s, const double* b_dev, double* x_dev, double tol,
                       int method, stdg_solve_stats* stats);

/* Allocation-free variant of stdg_solve(..., STDG_SOLVER_KRON_CG, ...).  The paper has no
 * counterpart: this exists for callers that may not allocate device memory once they are
 * running -- for example code whose device memory is entirely owned by another allocator (a
 * framework's caching pool that has reserved the device), or latency-critical loops where the
 * implicit synchronisation and unpredictable latency of cudaMalloc/cudaFree are not acceptable.
 * stdg_solve allocates its Krylov vectors on first use; this call allocates nothing: its work
 * vectors live in one fixed device array compiled into the library (8.5 MB, held on every GPU
 * that loads the library until the process exits).
 *  - Size limit: ne * Nst <= 262144 pressure unknowns; larger systems return STDG_EINVAL with a
 *    message (use stdg_solve for them).
 *  - The first call on each device looks up that array's device address (cudaGetSymbolAddress)
 *    with the device current; make that first call before any stream capture.
 *  - All calls share the one array, which keeps whatever the last call left in it (x is set to
 *    zero before the iteration; everything else is written before it is read).  Calls whose
 *    device work overlaps -- on different streams or from different threads -- race on it.
 *  - It always runs the Kronecker-decoupled CG on the binary64-accurate operator (binary64 blocks,
 *    or their binary32-pair form when the solver was created with another precision option), one
 *    host check per iteration: never the mixed-precision inner-outer iteration that stdg_solve runs
 *    for STDG_SOLVER_KRON_CG under STDG_PREC_MIXED_*.  Its iterates then differ from that call's at
 *    rounding level and its iteration count from that call's.
 *  - b_dev, x_dev, tol and stats are as for stdg_solve; a non-finite b is STDG_ENAN. */
stdg_status stdg_solve_noalloc(stdg_solver* s, const double* b_dev, double* x_dev, double tol,
                               stdg_solve_stats* stats);

/* ---------------------------------------------------------------- time stepping */
/* Initial velocity: spatial L2 projection of `field` at t = 0 onto every dual cell
 * (constant in time), pressure 0, time t = 0. */
stdg_status stdg_set_initial(stdg_solver* s, const stdg_field* field);
/* Dirichlet velocity on the boundary (all boundary faces), evaluated each step. */
stdg_status stdg_set_boundary(stdg_solver* s, const stdg_field* field);
/* The same two, with the data from a host callback instead of a device field kind (the problem
 * statement of Sec. 2.4 allows any initial and boundary velocity).  The library computes the
 * quadrature points on the device with the kernels that consume the values, copies them to the host
 * and calls fn on them:
 *  - stdg_set_initial_fn calls fn once, at t = 0, with nf * 2 * nq points (nq: the nonlinear-degree
 *    tetrahedron rule, ceil((3p+2)/2)^3 points per sub-tetrahedron; unused slots of boundary faces
 *    carry the point (0, 0, 0, 0)), then projects as stdg_set_initial does.  Host and device memory
 *    of the call scale with nf * nq: meant for meshes up to ~10^5 faces; use a device kind beyond.
 *  - stdg_set_boundary_fn collects the space-time points of every boundary dual cell and boundary
 *    face once (nboundary * (nq + nqf) * nt points: sub-tetrahedron and face rules of the nonlinear
 *    degree times the time rule) and calls fn at the start of every stdg_step, t = t^n + tau dt.
 *    The same values serve the boundary projections (readings R2, R25) and the boundary flux of the
 *    convection (Eq. convdg, v+ = v_bc).
 * STDG_EINVAL on a NULL fn; a later stdg_set_boundary replaces the callback. */
stdg_status stdg_set_initial_fn(stdg_solver* s, stdg_vel_fn fn, void* user);
stdg_status stdg_set_boundary_fn(stdg_solver* s, stdg_vel_fn fn, void* user);
/* One time step t -> t + dt of the Picard pressure-correction algorithm (Sec. 2.6, steps
 * 0-6), n_picard Picard iterations, viscosity nu; pressure solves with `method` to `tol`,
 * viscous solves (Eq. A1_mod) to `tol`: decoupled in time with K = W R W^-1
 * (stdg_time_blockdiag) and solved by conjugate-orthogonal CG preconditioned by the exact
 * inverse of every tet's diagonal block, then confirmed on the original system (GMRES iterates
 * only if that residual is above `tol`).  STDG_VISC_SOLVER=gmres in the environment selects
 * the previous solvers (CG for p_t = 0, right-preconditioned GMRES(20) otherwise).  stats may
 * be NULL. */
stdg_status stdg_step(stdg_solver* s, double nu, int n_picard, int method, double tol,
                      stdg_step_stats* stats);
/* The convective term alone, step 2 of a Picard iteration (Sec. 2.5, Eq. convdg): for the
 * velocity averages vbar_dev on the main grid, layout [3][ne][Nst] (component, tet, time column
 * a, spatial index k at a N + k), writes ups_dev (same layout) with
 *   Ups^c_i = - int_{T_i x slab} grad(phi~_k) . v_c vbar + int_{dT_i x slab} phi~_k F^RS_c . n_i
 * on the slab [t, t + dt] that starts at the solver's current time, boundary faces taking the
 * Dirichlet data of the field set by stdg_set_boundary (Rusanov flux with v+ = v_bc).  Device
 * buffers owned by the caller; synchronises the solver's stream.  STDG_EUNSUPPORTED when the
 * boundary data come from a host callback (stdg_set_boundary_fn: evaluated per step only),
 * STDG_EINVAL on a NULL argument.  STDG_CONV_KERNEL=generic in the environment (read when the
 * solver is created) selects the runtime-degree kernel at every degree. */
stdg_status stdg_convection(stdg_solver* s, const double* vbar_dev, double* ups_dev);
/* Semi-implicit theta variant for p_t = 0 (Sec. 2.7, Eqs. CS_15_theta / CS_16_theta): the
 * momentum of every dual cell sees the pressure as p^{n+theta} = theta p^{n+1} + (1-theta) p^n.
 * stdg_step then takes Lambda (Eq. prevpress) of theta p^{n+1,k} + (1-theta) p^n, solves the
 * same system (Eq. A2_mod) for the increment of p^{n+theta} and adds increment / theta to p^{n+1};
 * theta = 1 (the default) is the scheme above.  theta = 1/2 is Crank-Nicolson.  STDG_EINVAL
 * unless 1/2 <= theta <= 1, and for theta != 1 unless p_t = 0.  The first step with theta != 1
 * allocates two pressure vectors. */
stdg_status stdg_set_theta(stdg_solver* s, double theta);
/* Copy the state out / in: P (ne*Nst) and V (nf*3*Nst), device or host pointers per
 * on_device; either pointer may be NULL.  t_out may be NULL. */
stdg_status stdg_get_state(const stdg_solver* s, double* P, double* V, int on_device, double* t_out);
stdg_status stdg_set_state(stdg_solver* s, const double* P, const double* V, int on_device, double t);
/* Basis-independent velocity moments U[nf][2][3][Ng][N]: for each face j and each side s
 * (l, then r; r slot zero on the boundary) U = int_{T_{s,j}^st} phi~^(s) v_h (the
 * M_{i,j} v_j product of Eq. vis3).  V_dev: V layout, U_dev: nf*2*3*Nst doubles. */
stdg_status stdg_velocity_moments(stdg_solver* s, const double* V_dev, double* U_dev);

/* ------------------------------------------------- learned preconditioner (FGMRES) */
/* The paper solves the pressure system without a preconditioner.  These calls build, train and
 * apply a small message-passing network over the tet-face adjacency that is added to block
 * Jacobi as the right preconditioner of flexible GMRES (STDG_SOLVER_FGMRES_GNN):
 *   x_i = [r_i / RMS(r), (|J_i|/mean|J|)^(1/3), boundary faces of i / 4]
 *   h0 = relu(We x + be); h^l = relu(Ws^l h^{l-1} + Wm^l Sum_{face neighbours} h^{l-1} + b^l)
 *   M(r) = BJ(r) + RMS(r) (Wd h^L + bd)
 * Weights: binary32 master copy, working copy in bfloat16 (bf16_weights != 0) or binary32;
 * products accumulate in binary32.  Training minimises the mean of ||net(r) - t||^2 / ||t||^2
 * over harvested pairs with Adam.  Parameters are one flat binary32 array whose layout is
 * given by stdg_gnn_layout (offsets of We, be, then Ws, Wm, b per layer, then Wd, bd). */
stdg_status stdg_gnn_init(stdg_solver* s, int hidden, int layers, int bf16_weights, uint64_t seed);
stdg_status stdg_gnn_layout(stdg_solver* s, int64_t* offsets, int* hidden, int* layers, int* nfeat);
/* Copy the binary32 master parameters out (w_out) and/or in (w_in, resets Adam); either may be NULL. */
stdg_status stdg_gnn_params(stdg_solver* s, float* w_out, const float* w_in, int64_t* nparams);
/* z = RMS(r) (Wd h^L + bd): the network alone (P layout, device). */
stdg_status stdg_gnn_apply(stdg_solver* s, const double* r_dev, double* z_dev);
/* Mean loss over npairs pairs (R_dev, T_dev: npairs consecutive P-layout vectors) and its gradient
 * with respect to the master parameters, copied to grad_host (may be NULL). */
stdg_status stdg_gnn_loss_grad(stdg_solver* s, const double* R_dev, const double* T_dev, int npairs,
                               double* loss, float* grad_host);
/* Solve A x = b with block-Jacobi Kronecker CG to 1e-12, keeping up to nsnap iterates x_k taken
 * every `every` iterations; store pairs (r_k = b - A x_k, t_k = (x - x_k) - BJ(r_k)) for training
 * (at most max_pairs in total, device memory sized on the first call). */
stdg_status stdg_gnn_harvest(stdg_solver* s, const double* b_dev, int nsnap, int every, int max_pairs,
                             int* total_pairs);
/* While nsnap > 0, every pressure system that stdg_step solves is first passed to
 * stdg_gnn_harvest(s, b, nsnap, every, max_pairs) (an extra solve per Picard iteration); nsnap = 0
 * stops harvesting. */
stdg_status stdg_gnn_autoharvest(stdg_solver* s, int nsnap, int every, int max_pairs);
/* While nsnap > 0, every mixed-precision coarse-corrected pressure solve (STDG_SOLVER_KRON_MG and
 * _KRON_MG_GNN) stores nsnap pairs from its outer iterations, with no extra solve: the residual r_k of
 * the decoupled system after k >= 1 inner-solve steps and the error x* - x_k there (x* the solve's final
 * x).  Storage for max_pairs pairs is allocated on the first call; harvesting stops when it is full.
 * nsnap = 0 stops harvesting. */
stdg_status stdg_gnn_autoharvest_mg(stdg_solver* s, int nsnap, int max_pairs);
/* `epochs` passes of Adam (learning rate lr, `batch` pairs per update) over the harvested pairs. */
stdg_status stdg_gnn_train(stdg_solver* s, int epochs, double lr, int batch, double* first_loss,
                           double* last_loss);

/* The product behind the network's dense layers when its weights are bfloat16 (the learned
 * preconditioner above; the paper has no counterpart): D[m * ldd + n] = Sum_k A[m * lda + k] B[n * ldb + k]
 * for m < M, n < N, k < K, with A and B (binary32, device) rounded to bfloat16 and the products summed
 * in binary32 on the tensor cores (tcgen05.mma, kind::f16, accumulator in tensor memory).
 * 1 <= N <= 256 (STDG_EINVAL otherwise); work on `stream`, synchronised before return; STDG_ETIMEOUT
 * if a bounded wait for the tensor cores gave up.  Allocates one word of device memory per call. */
stdg_status stdg_tc_gemm_bf16(const float* A_dev, int64_t lda, const float* B_dev, int64_t ldb, float* D_dev,
                              int64_t ldd, int M, int N, int K, void* stream);

/* Throughput of the current device's binary64 and binary32 FMA pipes in TFLOP/s (2 flops per FMA),
 * measured with independent FMA chains on every SM and CUDA events on `stream`: the peaks the
 * binary64 operator kernel and, divided by the 12 binary32 operations of one pair product, the
 * pair kernel are rated against.  A measurement helper (the paper has no counterpart); allocates
 * 16 bytes of device memory for the duration of the call. */
stdg_status stdg_fma_probe(double* tflops_fp64, double* tflops_fp32, void* stream);

/* ---------------------------------------------------------------- profiling */
typedef struct {
  int64_t kernel_launches;   /* CUDA kernels this library launched since stdg_profile      */
  int64_t operator_launches; /* five-point operator launches (pressure and viscous)        */
  double operator_ms;        /* summed CUDA-event time of the operator launches (enabled)  */
  int64_t kind_launches[4];  /* timed operator launches by kernel: [0] binary64 blocks,     */
  double kind_ms[4];         /* [1] binary32-pair blocks, [2] binary32, [3] bfloat16 blocks */
  double phase_ms[8];        /* stdg_step by phase (CUDA events, enabled): [0] slab setup
                                (averages, boundary data, trace), [1] averaging and Lambda,
                                [2] convection, [3] viscous solves, [4] goback and pressure
                                right-hand side, [5] pressure solve, [6] updates, [7] unused */
} stdg_profile_stats;
/* Reset the counters; enable != 0 also records a CUDA event pair around every operator
 * launch on the solver's stream (adds two event records per launch). */
stdg_status stdg_profile(stdg_solver* s, int enable);
/* Synchronise the solver's stream and read the counters. */
stdg_status stdg_profile_read(stdg_solver* s, stdg_profile_stats* out);

/* ---------------------------------------------------------------- inspection */
/* Copy per-face spatial blocks to host arrays (any may be NULL):
 *  Q_host[nf][2][3][N][N]: Q^sp_{s,j}[c][m][l] = int_{T_sj} psi_m d_c phi_l - sigma n_c int_{Gamma_j} psi_m phi_l
 *     (Eq. MD_6 without the time factor); on a boundary face slot 1 holds the volume part.
 *  Mij_host[nf][2][N][N]: int_{T_sj} phi_k psi_l.   Aoff_host[nf][N][N], Bdiag_host[ne][N][N]. */
stdg_status stdg_get_blocks(const stdg_solver* s, double* Q_host, double* Mij_host,
                            double* Aoff_host, double* Bdiag_host);

const char* stdg_last_error(void);
const char* stdg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STDG_H */
