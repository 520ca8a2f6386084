// The solver object behind the C ABI (internal).
#pragma once
#include <vector>

#include "dev.cuh"

namespace stdg {
struct MgState;                    // agglomeration coarse correction (mg.cu)
// State of the learned preconditioner (gnn.cu)
struct GnnState {
  int H = 64, L = 3, G = 2, F = 0, C = 0, bf16 = 1;
  int64_t np = 0;
  std::vector<int64_t> off;        // We, be, (Ws, Wm, b) x L, Wd, bd
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  void* wc = nullptr;              // working copy (bfloat16 or binary32)
  int adam_t = 0;
  float *geom = nullptr, *X = nullptr, *pre0 = nullptr, *out = nullptr, *dout = nullptr;
  float *dh = nullptr, *dpre = nullptr, *t1 = nullptr, *t2 = nullptr, *wpart = nullptr;
  std::vector<float*> h, mb, pre;
  double *sdev = nullptr, *part = nullptr, *loss = nullptr, *tpinv = nullptr;
  double *R = nullptr, *T = nullptr;   // harvested pairs (residual, target = error - BJ(residual))
  int npairs = 0, cap = 0;
};
}  // namespace stdg

struct stdg_solver {
  int device = 0;
  cudaStream_t stream = nullptr;
  stdg_solver_options opt{};
  int p = 0, pt = 0, N = 0, Ng = 0, Nst = 0;
  int64_t ne = 0, nf = 0, nint = 0, nbd = 0;
  double dt = 0.0;
  std::vector<double> K, Kinv, g0, g1;        // host copies of the time matrices
  stdg::TimeMats tm{};
  stdg::DevMesh dm;
  stdg::DevRef dr;
  int nq_lin = 0, nqf_lin = 0, nq_nl = 0, nqf_nl = 0, nt_nl = 0;
  std::vector<double> time_nl_tau, time_nl_w, time_nl_g;
  double *d_ttau = nullptr, *d_tw = nullptr, *d_tg = nullptr;   // device copies
  // per-face / per-tet blocks
  double *Q = nullptr, *Mij = nullptr, *C = nullptr, *x0h = nullptr;
  double *Aoff = nullptr, *Bdiag = nullptr, *Bvisc = nullptr;
  double *Binv = nullptr;                     // block-Jacobi: (-B_i)^-1, pinned (lazily built)
  double *kz = nullptr;                       // preconditioned residual
  // low-precision copies for the mixed-precision inner solve
  void *lpB = nullptr, *lpA = nullptr;        // blocks in binary32 or bfloat16, padded stride lpSB
  int lpSB = 0, lpkind = -1;
  void *dfB = nullptr, *dfA = nullptr;        // (hi, lo) binary32 pairs of the FP64 blocks
  int dfSB = 0;
  int tma_grid[16] = {0};                     // persistent grid size per block element size
  int *gface = nullptr, *gnbr = nullptr;      // per-tet gather tables (int4 each) for the TMA kernels
  void *wB = nullptr, *wA = nullptr;          // warp-kernel block copies (binary32 / bfloat16), padded rows
  void *wdB = nullptr, *wdA = nullptr;        // warp-kernel (hi, lo) binary32 planes of the FP64 blocks
  void *wdBv = nullptr;                       // same for the viscous diagonal blocks B_i - Bvisc_i
  void *wBv32 = nullptr;                      // the viscous diagonal blocks in binary32 (padded rows)
  int warp_grid[32] = {0}, warp_wpc[32] = {0};
  int op_warp = 1;                            // 1: warp-per-tet kernels, 0: block-staged TMA kernels
  int op_cta = 1;                             // with op_warp: several warps share each staged tet
  int mix_inner = 80;                         // binary32 CG iterations per outer step of the mixed solve
  int mix_inner_mg = 40;                      // the same with the coarse correction (converges faster)
  int mix_m = 16;                             // directions the outer flexible CG keeps
  int df_min_warps = 3;                       // the pair kernel serves where this many warps fit per SM
  bool visc_inner64 = false;                  // mixed viscous refinement: binary64-vector inner COCG
  bool conv_generic = false;                  // convection: the runtime-degree kernel at every degree
  double *fcgP = nullptr, *fcgQ = nullptr;    // their P_j and Q_j = S P_j
  double *opdot = nullptr;                    // per-block p.q partials of the binary32 operator launch
  float *lpBinv = nullptr;                    // block-Jacobi inverses in binary32
  float *fr = nullptr, *fp = nullptr, *fq = nullptr, *fz = nullptr, *fx = nullptr, *fb = nullptr;
  double* dmix = nullptr;                     // device copy of K (time mixing)
  int* derr = nullptr;                        // device error word (bounded waits)
  // state
  double *P = nullptr, *V = nullptr;
  double t = 0.0;
  stdg_field bc{};
  // Krylov workspace (allocated on first use)
  double *kb = nullptr, *kx = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr;
  double *basis = nullptr;                    // (restart+1) * n
  double *part = nullptr;                     // reduction partials
  double *scal = nullptr;                     // device scalars
  double *hostbuf = nullptr;                  // pinned host scalars
  int basis_cols = 0;
  // step workspace
  double *Vbar = nullptr, *Vbar_n = nullptr, *Lam = nullptr, *Ups = nullptr, *rhsv = nullptr;
  double *F = nullptr, *Vbc = nullptr, *Gbc = nullptr, *bvec = nullptr, *dp = nullptr, *vtmp = nullptr;
  double *wk1 = nullptr, *wk2 = nullptr;
  double *fac_x = nullptr, *fac_v = nullptr;   // factored-form cross-check operator (lazily allocated)
  double theta = 1.0;                          // semi-implicit pressure weight (p_t = 0 only)
  double *Pn = nullptr, *Pth = nullptr;        // p^n and theta p^{n+1,k} + (1 - theta) p^n (theta < 1)
  float2 *cphiP = nullptr, *cdphiP = nullptr, *cfphiP = nullptr;   // convection tables as (hi, lo) pairs
  float2 *cphiT = nullptr, *cfphiT = nullptr;                        // the value tables transposed
  float2 *ctgP = nullptr, *ctwP = nullptr;                            // time basis and weights, as pairs
  // device allocations: through the caller's allocator when one was given (stdg_solver_create_alloc),
  // else cudaMalloc; released in reverse order by stdg_solver_destroy
  struct Alloc { void* p; size_t bytes; };
  std::vector<Alloc> allocs;
  stdg_alloc_fn alloc_fn = nullptr;
  stdg_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  // initial / boundary data from a host callback (stdg_set_initial_fn, stdg_set_boundary_fn)
  stdg_vel_fn bc_fn = nullptr;
  void* bc_user = nullptr;
  int* bidx = nullptr;                        // compact boundary index of every face, -1 if interior
  double* bc_table = nullptr;                 // callback values at the boundary points [nbd][npt][3]
  double* bc_modes = nullptr;                 // device modes of a STDG_FIELD_CURL_MODES boundary field
  std::vector<double> bc_pts;                 // the boundary points [nbd * npt][4]: x, y, z, tau
  std::vector<double> bc_xyzt, bc_uvw;        // per-step callback arguments
  stdg::GnnState* gnn = nullptr;
  stdg::MgState* mg = nullptr;               // coarse correction of STDG_SOLVER_KRON_MG (built on first use)
  float *vpcU = nullptr, *vpcLam = nullptr;  // viscous block-Jacobi by fast diagonalisation (viscpc.cu)
  int vbd = -1;                               // K = W R W^-1 found (1), not available (0), not tried (-1)
  double vW[25], vWinv[25], vR[25];           // its factors (Ng x Ng, row-major)
  int vpair[5];                               // first column of each 2 x 2 block of R
  double* kzz = nullptr;                     // FGMRES preconditioned directions
  int snap_every = 0, snap_cap = 0, nsnap = 0;
  int ah_nsnap = 0, ah_every = 0, ah_max = 0;   // harvest pairs from the pressure systems of stdg_step
  int ah_mg = 0;                                // harvest from the first ah_mg outer iterations of each mixed solve
  double* snaps = nullptr;
  // CUDA-graph batching of Krylov iterations
  cudaStream_t cstream = nullptr;
  cudaEvent_t sync_ev[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> gev;
  bool capturing = false;
  // profiling: kernel launch count and CUDA-event timing of every operator launch
  int64_t nlaunch = 0, op_launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev;      // start/stop pairs
  int ev_used = 0;
  double op_ms = 0.0;
  double kind_ms[4] = {0, 0, 0, 0};           // by kernel kind: FP64, pair-FP32, FP32, BF16
  int64_t kind_n[4] = {0, 0, 0, 0};
  int ev_kind[4096];
  // stdg_step phase timing (profiling): event pool, the phase each recorded event closes, totals
  std::vector<cudaEvent_t> phase_ev;
  std::vector<int> phase_of;
  double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace stdg {
// binary32 Krylov kernels (lowprec.cu), exposed as launch functions
struct LpKernels {
  void (*coldot)(cudaStream_t, int64_t, int, int, const float*, const float*, double*);
  void (*update)(cudaStream_t, int64_t, int, int, const double*, float*, float*, const float*, const float*,
                 const double*, double*, int);
  void (*dir)(cudaStream_t, int64_t, int, int, const double*, const float*, float*);
  void (*bjacobi)(cudaStream_t, int, int, int, const float*, const float*, float*, double*);
  void (*from64)(cudaStream_t, int64_t, int, int, const double*, double, const double*, float*);
  void (*accum)(cudaStream_t, int64_t, double, const float*, double*);
  void (*f32)(cudaStream_t, int64_t, const double*, float*);
  void (*scale)(cudaStream_t, int64_t, float, float*);
  void (*f32s)(cudaStream_t, int64_t, double, const double*, float*);
};
LpKernels lp_kernels();
// x += alpha p; r -= alpha q; z = Binv r; partials of r.z per column (kLpBlocks partials)
void lp_update_bjacobi(cudaStream_t st, int ne, int N, int Ng, const double* alpha, float* x, float* r, const float* p,
                       const float* q, const float* Binv, float* z, double* part);
cudaError_t lp_build_blocks(stdg_solver* s, int kind);
cudaError_t launch_apply_lp(stdg_solver* s, const float* x, float* y, int pinned, int kron, float scale, float pin_diag,
                            double* dotpart = nullptr);
cudaError_t warp_prepare(stdg_solver* s, int precision);   // block copies + launch shape, outside capture
int warp_df_warps_per_sm(stdg_solver* s);                  // resident warps per SM of the pair kernel
cudaError_t launch_apply_warp_lp(stdg_solver* s, const float* x, float* y, int pinned, int kron, float scale,
                                 float pin_diag, double* dotpart = nullptr);
int warp_blocks_lp(stdg_solver* s);   // blocks of the binary32 operator launch (dot partials it writes)
cudaError_t warp_prepare_f32_visc(stdg_solver* s);        // binary32 viscous operator (mixed_f32 only)
cudaError_t warp_launch_f32_visc(stdg_solver* s, const float* x, float* y, double scale, double mass_coef,
                                 const double* Kmass);
cudaError_t launch_apply_warp_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                                 double pin_diag);
cudaError_t launch_apply_warp_df_visc(stdg_solver* s, const double* x, double* y, double scale, double mass_coef,
                                      const double* Kmass);
cudaError_t launch_apply_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                            double pin_diag);
cudaError_t df_build_blocks(stdg_solver* s);
stdg_status ensure_krylov(stdg_solver* s);
stdg_status apply_pressure(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                           double pin_diag);
stdg_status solve_pressure(stdg_solver* s, const double* b, double* x, double tol, int method,
                           stdg_solve_stats* st);
stdg_status solve_pressure_noalloc(stdg_solver* s, const double* b, double* x, double tol,
                                   stdg_solve_stats* st);
stdg_status gnn_precond(stdg_solver* s, const double* r, double* z, int use_gnn);
stdg_status gnn_correct(stdg_solver* s, const double* r, double* z, int* bad);
bool gnn_mg_harvest_room(stdg_solver* s, int k);
void gnn_mg_harvest_snap(stdg_solver* s, int k, const double* r, const double* x, const double* z);
void gnn_mg_harvest_finish(stdg_solver* s, int got, const double* x);
stdg_status solve_viscous(stdg_solver* s, const double* b, double* x, double nu, double tol, int* iters,
                          double* res);
stdg_status dev_alloc(stdg_solver* s, void** p, size_t bytes);
cudaError_t dev_alloc_cuda(stdg_solver* s, void** p, size_t bytes);   // the same, as a CUDA error code
void dev_free(stdg_solver* s, void* p);                                 // early release of one array
// Agglomeration coarse correction (mg.cu): z += R^T V (R r) on the constant modes of every tet, with
// partials of r.(R^T V R r) per column written to part[b * Ng + a], b < mg_partial_blocks().
stdg_status mg_ensure(stdg_solver* s);       // host + device setup, outside stream capture
void mg_apply_f32(stdg_solver* s, const float* r, float* z, double* part);
void mg_apply_f64(stdg_solver* s, const double* r, double* z, double* part);
int mg_launches(const stdg_solver* s);       // kernel launches per application
int mg_partial_blocks();
int mg_levels(const stdg_solver* s, int* sizes, int cap);
void mg_free(stdg_solver* s);
// Dense layer products on the tensor cores (tcgemm.cu): D (+)= A B^T with bfloat16 operands
struct TcGemmArgs {
  int M, N, K, ksplit;                       // CTA (x, z) covers rows [128 x, ...) and k in [z ksplit, ...)
  const float* A; int64_t sAm, sAk;          // A(m, k) = A[m sAm + k sAk]
  const void* B; int64_t sBn, sBk;           // B(n, k) = B[n sBn + k sBk]
  int b_bf16;                                // B elements are bfloat16 (else binary32)
  int b_ones_last;                           // B(N - 1, k) = 1 (a bias column of a weight gradient)
  float* D; int64_t ldd, dsplit;             // D(m, n) of K range z at D[z dsplit + m ldd + n]
  const float* bias;                         // + bias[n]
  int accumulate, relu;                      // D = (D +) A B^T (+ bias), then max(., 0)
  float* pre;                                // pre-activation (before ReLU), if not null
  int* err;                                  // set to 1 when a bounded wait gives up
};
cudaError_t launch_tc_gemm(TcGemmArgs a, cudaStream_t st);
// Viscous block Jacobi (viscpc.cu): eigenvectors / eigenvalues of every tet's spatial viscous block,
// then z = D^-1 r (accum: z += D^-1 r) with D the tet-diagonal blocks of the viscous operator.
stdg_status visc_pc_ensure(stdg_solver* s);
stdg_status visc_pc_apply(stdg_solver* s, double nu, const double* r, double* z, int accum,
                          const double* Kt = nullptr);
stdg_status visc_pc_apply32(stdg_solver* s, double nu, const float* r, float* z, const double* Kt);

// Binary32 vector kernels of the inner COCG solves (cocg32.cu).  Vectors are [tet][time column][N];
// the multipliers M (Ng x Ng, binary64 on the device) are block diagonal with blocks of size 1 or 2,
// so only M[a][a-1..a+1] is read.  mix holds an Ng x Ng matrix applied to every tet's time columns.
struct Mix32 { float v[kMaxNg * kMaxNg]; };
void c32_mix_to32(cudaStream_t st, int ne, int N, int Ng, const Mix32& M, const double* in, float* out);
void c32_mix_acc64(cudaStream_t st, int ne, int N, int Ng, const Mix32& M, const float* y, double* x);
void c32_cross(cudaStream_t st, int ne, int N, int Ng, const float* u, const float* v, double* part);
void c32_update(cudaStream_t st, int ne, int N, int Ng, const double* M, float* y, float* r, const float* p,
                const float* q, const Mix32& W, double* part, int want);
void c32_dir(cudaStream_t st, int ne, int N, int Ng, const double* M, const float* z, float* p);
bool time_blockdiag(const double* K, int Ng, double* W, double* Winv, double* R, int* pair);
void prof_fold(stdg_solver* s);
}  // namespace stdg
