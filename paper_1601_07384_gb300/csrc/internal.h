// Internal declarations of the stdg library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stdg.h"

namespace stdg {

void set_error(const char* fmt, ...);
const char* last_error();

// Quadrature rule on a reference entity: x[n*dim], w[n].
struct Rule {
  int dim = 0, n = 0;
  std::vector<double> x, w;
};

// Gauss-Jacobi on [0,1] for the weight (1-x)^alpha (alpha integer >= 0).
void gauss_jacobi01(int n, int alpha, std::vector<double>& x, std::vector<double>& w);
Rule line_rule(int n);
Rule tri_rule(int n);   // reference triangle, weights sum to 1/2
Rule tet_rule(int n);   // reference tetrahedron, weights sum to 1/6

int nbasis(int p);
// Multi-indices (i, j, k) in the shared order: n = 0..p, i = 0..n, j = 0..n-i, k = n-i-j.
std::vector<int> multi_indices(int p);
// Orthonormal Dubiner values phi[N] and reference gradients dphi[3*N] (d-major) at xi.
void dubiner_eval(int p, const double* xi, double* phi, double* dphi);
// Orthonormal Legendre on [0,1]: g[Ng], dg[Ng].
void legendre01(int pt, double tau, double* g, double* dg);

// Ordered triple code of three distinct local vertices (a, b, c) of a tetrahedron.
inline int tri_code(int a, int b, int c) { return a * 16 + b * 4 + c; }
constexpr int kTriCodes = 64;

}  // namespace stdg

struct stdg_mesh {
  int64_t nv = 0, ne = 0, nf = 0, nint = 0, nbd = 0;
  std::vector<double> X;                 // nv*3
  std::vector<int64_t> T;                // ne*4
  std::vector<double> J, Jinv, detJ, bary;  // ne*9 (row-major, columns = edges), ne*9, ne, ne*3
  std::vector<int64_t> left, right;      // nf
  std::vector<int32_t> fl, fr;           // nf
  std::vector<int64_t> fverts;           // nf*3, canonical order = l's local order
  std::vector<int32_t> code_l, code_r;   // nf, ordered-triple codes of the canonical vertices in l / r
  std::vector<double> normal, area;      // nf*3, nf
  std::vector<int64_t> t2f, t2n;         // ne*4
  std::vector<int32_t> t2code;           // ne*4: code of face t2f[i][f]'s canonical vertices in tet i
  bool periodic = false;                 // periodic box: vertex ids are lattice points of the box
  double period[3] = {0, 0, 0};
  std::vector<double> fcoords;           // nf*9: canonical face vertex coordinates in l(j)'s frame
  std::vector<double> fshift;            // nf*3: a point of r(j) in l(j)'s frame = in r(j)'s frame + fshift
                                         //       (a period vector on a periodic mesh, else 0)
};

struct stdg_ref {
  int p = 0, pt = 0, N = 0, Ng = 0, Nst = 0;
  int nq_lin = 0, nqf_lin = 0, nt_lin = 0, nq_nl = 0, nqf_nl = 0, nt_nl = 0;
  std::vector<double> K, Kinv, g0, g1;   // Ng*Ng, Ng*Ng, Ng, Ng
  // linear-degree rules (products of two degree-p functions): sub-tets S_f, faces, time
  std::vector<double> sub_lin_xi, sub_lin_w, sub_lin_phi, sub_lin_dphi;   // [4][nq][3], [4][nq], [4][nq][N], [4][nq][3][N]
  std::vector<double> tri_lin_st, tri_lin_w, face_lin_phi;               // [nqf][2], [nqf], [64][nqf][N]
  std::vector<double> time_lin_tau, time_lin_w, time_lin_g, time_lin_dg; // [nt], [nt], [nt][Ng], [nt][Ng]
  // nonlinear-degree rules (cubic integrands and non-polynomial data)
  std::vector<double> sub_nl_xi, sub_nl_w;                                // [4][nq][3], [4][nq]
  std::vector<double> tet_nl_xi, tet_nl_w, tet_nl_phi, tet_nl_dphi;      // [nq][3], [nq], [nq][N], [nq][3][N]
  std::vector<double> tri_nl_st, tri_nl_w, face_nl_phi;                  // [nqf][2], [nqf], [64][nqf][N]
  std::vector<double> time_nl_tau, time_nl_w, time_nl_g;                 // [nt], [nt], [nt][Ng]
};
