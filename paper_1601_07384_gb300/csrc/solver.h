// The solver object behind the C ABI (internal).
#pragma once
#include <vector>

#include "dev.cuh"

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
  float* blk32 = nullptr;                     // double-float copies (hi, lo) of Bdiag / Aoff
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
  std::vector<void*> allocs;
  // profiling: kernel launch count and CUDA-event timing of every operator launch
  int64_t nlaunch = 0, op_launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev;      // start/stop pairs
  int ev_used = 0;
  double op_ms = 0.0;
};

namespace stdg {
stdg_status ensure_krylov(stdg_solver* s);
stdg_status apply_pressure(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                           double pin_diag);
stdg_status solve_pressure(stdg_solver* s, const double* b, double* x, double tol, int method,
                           stdg_solve_stats* st);
stdg_status solve_pressure_noalloc(stdg_solver* s, const double* b, double* x, double tol,
                                   stdg_solve_stats* st);
stdg_status solve_viscous(stdg_solver* s, const double* b, double* x, double nu, double tol, int* iters,
                          double* res);
stdg_status dev_alloc(stdg_solver* s, void** p, size_t bytes);
void prof_fold(stdg_solver* s);
}  // namespace stdg
