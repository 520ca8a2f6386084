// Device-side declarations shared by the stdg CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

#define STDG_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      stdg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                      __LINE__);                                                         \
      return STDG_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

#define STDG_LAUNCH_CHECK()                                                              \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) {                                                             \
      stdg::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),        \
                      __FILE__, __LINE__);                                               \
      return STDG_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

namespace stdg {

constexpr int kMaxN = 35;   // p <= 4
constexpr int kMaxNg = 5;   // p_t <= 4

// Multi-index exponents passed by value to kernels.
struct MultiIdx { unsigned char e[3 * kMaxN]; };

// Device copies of the mesh.
struct DevMesh {
  int ne = 0, nf = 0;
  int *left = nullptr, *right = nullptr, *fl = nullptr, *fr = nullptr;
  int *code_l = nullptr, *code_r = nullptr;
  int *t2f = nullptr, *t2n = nullptr, *t2code = nullptr;
  double *X0 = nullptr, *J = nullptr, *Jinv = nullptr, *detJ = nullptr, *bary = nullptr;
  double *fvx = nullptr, *normal = nullptr, *area = nullptr;
  double* fshift = nullptr;   // [nf][3]: r(j)'s frame -> l(j)'s frame (a period vector on periodic meshes)
};

// Device copies of the reference tables (layouts as in stdg_ref).
struct DevRef {
  double *sub_lin_xi = nullptr, *sub_lin_w = nullptr, *sub_lin_phi = nullptr, *sub_lin_dphi = nullptr;
  double *tri_lin_st = nullptr, *tri_lin_w = nullptr, *face_lin_phi = nullptr;
  double *sub_nl_xi = nullptr, *sub_nl_w = nullptr;
  double *tet_nl_xi = nullptr, *tet_nl_w = nullptr, *tet_nl_phi = nullptr, *tet_nl_dphi = nullptr;
  double *tri_nl_st = nullptr, *tri_nl_w = nullptr, *face_nl_phi = nullptr;
};

// Small time matrices passed by value.
struct TimeMats {
  double Tp[kMaxNg * kMaxNg];     // dt^2 K^-1
  double K[kMaxNg * kMaxNg];
  double Kinv[kMaxNg * kMaxNg];
  double g0[kMaxNg], g1[kMaxNg];
};

// Launchers (precompute.cu)
cudaError_t launch_face_blocks(const DevMesh& m, const DevRef& r, int p, int N, int nq, int nqf,
                               const MultiIdx& mi, double* Q, double* Mij, double* C, double* x0h,
                               cudaStream_t st);
cudaError_t launch_assemble(const DevMesh& m, int N, const double* Q, double* Aoff, double* Bdiag,
                            double* Bvisc, cudaStream_t st);
cudaError_t launch_block_inverse(int ne, int N, const double* Bdiag, double* Binv, cudaStream_t st);

}  // namespace stdg

namespace stdg {

// Generic five-point block operator on tets (pressure operator of Eq. CS_19, or the viscous
// operator of Eq. A1_mod which shares its spatial blocks):
//   acc_i = (Bdiag_i + extra_coef Bextra_i) x_i + Sum_{f: interior} A_{i,p(i,f)} x_p
//   y_i[a][k] = scale Sum_b Tacc[a][b] acc_i[b][k] + mass_coef detJ_i Sum_b Kmass[a][b] x_i[b][k]
// with Tacc = identity when tacc_identity.  pinned: x at (tet 0, mode 0, every a) read as 0,
// y there = pin_diag * x.
struct ApplyArgs {
  int ne, N, Ng;
  const int *t2f, *t2n, *left;
  const double *Bdiag, *Aoff, *Bextra, *detJ;
  double extra_coef, scale, mass_coef, pin_diag;
  int tacc_identity, pinned;
  double Tacc[kMaxNg * kMaxNg];
  double Kmass[kMaxNg * kMaxNg];
};
cudaError_t launch_apply(const ApplyArgs& a, const double* x, double* y, cudaStream_t st);

// b_i[a][l] = coef Sum_{f} Sum_c Sum_m Q^c_{s(i,j)}[m][l] F_j[c][a][m]   (D = -Q^T; coef = -dt)
cudaError_t launch_rhs(int ne, int N, int Ng, const int* t2f, const int* left, const double* Q,
                       const double* F, double coef, int pinned, double* b, cudaStream_t st);
// V_j = F_j - dt (I (x) K^-1) Sum_s Q_sj dp_s on interior faces, V_j = F_j on boundary faces.
cudaError_t launch_update(int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                          const double* F, const double* dp, double dt, const double* Kinv,
                          double* V, cudaStream_t st);
// The support steps in pair arithmetic at the compile-time degrees (support.cu); cudaErrorNotSupported
// at other (N, Ng), where the binary64 kernels serve.  support_fp64(): STDG_SUPPORT=fp64 in the
// environment (read once per process) keeps the binary64 kernels everywhere.
bool support_fp64();
cudaError_t sup_average(cudaStream_t st, int ne, int N, int Ng, const int* t2f, const int* left, const double* detJ,
                        const double* Mij, const double* in, double* out);
cudaError_t sup_face_grad(cudaStream_t st, int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                          const double* Pp, double dt, const double* Kinv, double* G);
cudaError_t sup_update(cudaStream_t st, int nf, int N, int Ng, const int* left, const int* right, const double* Q,
                       const double* F, const double* dp, double dt, const double* Kinv, double* V);
// U_j[s][c][a][k] = dt Sum_l Mij_s[k][l] V_j[c][a][l]
cudaError_t launch_moments(int nf, int N, int Ng, const double* Mij, const double* V, double dt,
                           double* U, cudaStream_t st);

}  // namespace stdg

namespace stdg {
// Velocity data evaluated on the device (stdg_field), plus two internal kinds for data from a host
// callback: kFieldTable reads the value the callback returned for point `pid`; kFieldCollect records
// the point (x, y, z, tau) at `pid` so that the host can evaluate the callback there, and yields 0.
constexpr int kFieldTable = 100;
constexpr int kFieldCollect = 101;
struct FieldArg {
  int kind; double c[3]; double a, d, nu;
  int nmodes; const double* modes;   // STDG_FIELD_CURL_MODES: per mode k (3), A (3), phi, 2 pi k x A (3)
  const double* table;               // kFieldTable: [pid][3]
  double* collect;                   // kFieldCollect: [pid][4]
};

__device__ inline void eval_field(const FieldArg& f, const double* x, double t, int64_t pid, double tau, double* v) {
  if (f.kind == STDG_FIELD_CONSTANT) { v[0] = f.c[0]; v[1] = f.c[1]; v[2] = f.c[2]; return; }
  if (f.kind == STDG_FIELD_BELTRAMI) {
    const double a = f.a, d = f.d, X = x[0], Y = x[1], Z = x[2];
    const double e = exp(-f.nu * d * d * t);
    v[0] = -a * (exp(a * X) * sin(a * Y + d * Z) + exp(a * Z) * cos(a * X + d * Y)) * e;
    v[1] = -a * (exp(a * Y) * sin(a * Z + d * X) + exp(a * X) * cos(a * Y + d * Z)) * e;
    v[2] = -a * (exp(a * Z) * sin(a * X + d * Y) + exp(a * Y) * cos(a * Z + d * X)) * e;
    return;
  }
  if (f.kind == STDG_FIELD_CURL_MODES) {
    // v = c0 curl(b Psi) = c0 (grad b x Psi + b curl Psi), b = B^2, B = 64 x(1-x) y(1-y) z(1-z)
    const double X = x[0], Y = x[1], Z = x[2];
    const double px = X * (1.0 - X), py = Y * (1.0 - Y), pz = Z * (1.0 - Z);
    const double B = 64.0 * px * py * pz;
    const double g0 = 2.0 * B * 64.0 * (1.0 - 2.0 * X) * py * pz;
    const double g1 = 2.0 * B * 64.0 * px * (1.0 - 2.0 * Y) * pz;
    const double g2 = 2.0 * B * 64.0 * px * py * (1.0 - 2.0 * Z);
    const double b = B * B;
    double ps0 = 0.0, ps1 = 0.0, ps2 = 0.0, cu0 = 0.0, cu1 = 0.0, cu2 = 0.0;
    for (int m = 0; m < f.nmodes; ++m) {
      const double* md = f.modes + 10 * m;
      const double th = 2.0 * 3.14159265358979323846 * (md[0] * X + md[1] * Y + md[2] * Z) + md[6];
      double sn, cs;
      sincos(th, &sn, &cs);
      ps0 = fma(md[3], sn, ps0); ps1 = fma(md[4], sn, ps1); ps2 = fma(md[5], sn, ps2);
      cu0 = fma(md[7], cs, cu0); cu1 = fma(md[8], cs, cu1); cu2 = fma(md[9], cs, cu2);
    }
    v[0] = f.c[0] * (g1 * ps2 - g2 * ps1 + b * cu0);
    v[1] = f.c[0] * (g2 * ps0 - g0 * ps2 + b * cu1);
    v[2] = f.c[0] * (g0 * ps1 - g1 * ps0 + b * cu2);
    return;
  }
  if (f.kind == kFieldTable) {
    v[0] = f.table[3 * pid]; v[1] = f.table[3 * pid + 1]; v[2] = f.table[3 * pid + 2];
    return;
  }
  if (f.kind == kFieldCollect) {
    f.collect[4 * pid] = x[0]; f.collect[4 * pid + 1] = x[1]; f.collect[4 * pid + 2] = x[2];
    f.collect[4 * pid + 3] = tau;
  }
  v[0] = v[1] = v[2] = 0.0;
}
}  // namespace stdg
