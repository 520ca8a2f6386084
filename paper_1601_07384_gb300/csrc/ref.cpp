// Reference quadrature, bases and tables (Sec. 2.3; rules are this library's choice since
// the paper does not fix them).  Host code, built from the definitions:
//  * Gauss-Jacobi nodes: roots of P_n^(alpha,0) on (-1,1), bracketed on a fine grid and
//    polished by Newton; weights 2^(alpha+1) / ((1 - x^2) P_n'(x)^2).
//  * Collapsed (conical product) rules for the triangle and the tetrahedron.
//  * Dubiner basis via collapsed coordinates u = xi/(1-eta-zeta), v = eta/(1-zeta), w = zeta:
//    c P_i(2u-1) (1-v)^i P_j^(2i+1,0)(2v-1) (1-w)^(i+j) P_k^(2i+2j+2,0)(2w-1),
//    c = sqrt((2i+1)(2i+2j+2)(2i+2j+2k+3)); gradients by the chain rule.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace stdg {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

// P_n^(a,b)(x) and its derivative by the three-term recurrence.
static void jacobi(int n, double a, double b, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a + b;
    double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
    double a2 = (c - 1.0) * (a * a - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
    double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  // d/dx P_n^(a,b) = (n + a + b + 1)/2 P_{n-1}^(a+1,b+1)
  if (n == 1) { *dP = 0.5 * (a + b + 2.0); return; }
  double q, dq;
  jacobi(n - 1, a + 1.0, b + 1.0, x, &q, &dq);
  *dP = 0.5 * (n + a + b + 1.0) * q;
}

void gauss_jacobi01(int n, int alpha, std::vector<double>& x, std::vector<double>& w) {
  x.clear(); w.clear();
  const int grid = 20000;
  double prev_x = -1.0, prev_v, d;
  jacobi(n, alpha, 0.0, -1.0 + 1e-15, &prev_v, &d);
  std::vector<double> roots;
  for (int g = 1; g <= grid; ++g) {
    double xx = -1.0 + 2.0 * g / grid;
    if (g == grid) xx = 1.0 - 1e-15;
    double v;
    jacobi(n, alpha, 0.0, xx, &v, &d);
    if ((v < 0) != (prev_v < 0)) {
      double lo = prev_x, hi = xx, flo = prev_v;
      for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        double mid = 0.5 * (lo + hi), fm;
        jacobi(n, alpha, 0.0, mid, &fm, &d);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      double r = 0.5 * (lo + hi);
      for (int it = 0; it < 3; ++it) {
        double f, df;
        jacobi(n, alpha, 0.0, r, &f, &df);
        if (df != 0.0) r -= f / df;
      }
      roots.push_back(r);
    }
    prev_x = xx; prev_v = v;
  }
  for (double r : roots) {
    double f, df;
    jacobi(n, alpha, 0.0, r, &f, &df);
    double wt = std::pow(2.0, alpha + 1.0) / ((1.0 - r * r) * df * df);
    // map to [0,1]: weight (1-x)^alpha dx -> 2^(alpha+1) (1-t)^alpha dt
    x.push_back(0.5 * (r + 1.0));
    w.push_back(wt / std::pow(2.0, alpha + 1.0));
  }
}

Rule line_rule(int n) {
  Rule r; r.dim = 1; r.n = n;
  gauss_jacobi01(n, 0, r.x, r.w);
  return r;
}

Rule tri_rule(int n) {
  std::vector<double> u, wu, v, wv;
  gauss_jacobi01(n, 0, u, wu);
  gauss_jacobi01(n, 1, v, wv);
  Rule r; r.dim = 2; r.n = n * n;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      r.x.push_back(u[a] * (1.0 - v[b]));
      r.x.push_back(v[b]);
      r.w.push_back(wu[a] * wv[b]);
    }
  return r;
}

Rule tet_rule(int n) {
  std::vector<double> u, wu, v, wv, s, ws;
  gauss_jacobi01(n, 0, u, wu);
  gauss_jacobi01(n, 1, v, wv);
  gauss_jacobi01(n, 2, s, ws);
  Rule r; r.dim = 3; r.n = n * n * n;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        r.x.push_back(u[a] * (1.0 - v[b]) * (1.0 - s[c]));
        r.x.push_back(v[b] * (1.0 - s[c]));
        r.x.push_back(s[c]);
        r.w.push_back(wu[a] * wv[b] * ws[c]);
      }
  return r;
}

int nbasis(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

std::vector<int> multi_indices(int p) {
  std::vector<int> out;
  for (int n = 0; n <= p; ++n)
    for (int i = 0; i <= n; ++i)
      for (int j = 0; j <= n - i; ++j) {
        out.push_back(i); out.push_back(j); out.push_back(n - i - j);
      }
  return out;
}

void dubiner_eval(int p, const double* xi, double* phi, double* dphi) {
  const double X = xi[0], Y = xi[1], Z = xi[2];
  const double s = 1.0 - Y - Z;      // (1-v)(1-w)
  const double t = 1.0 - Z;          // 1-w
  const double u = X / s, v = Y / t, w = Z;
  std::vector<int> mi = multi_indices(p);
  const int N = nbasis(p);
  for (int m = 0; m < N; ++m) {
    int i = mi[3 * m], j = mi[3 * m + 1], k = mi[3 * m + 2];
    double c = std::sqrt((2.0 * i + 1) * (2.0 * i + 2 * j + 2) * (2.0 * i + 2 * j + 2 * k + 3));
    double A, dA, Bj, dBj, Ck, dCk;
    jacobi(i, 0.0, 0.0, 2 * u - 1, &A, &dA);
    jacobi(j, 2.0 * i + 1, 0.0, 2 * v - 1, &Bj, &dBj);
    jacobi(k, 2.0 * i + 2 * j + 2, 0.0, 2 * w - 1, &Ck, &dCk);
    double omv_i = std::pow(1.0 - v, i), omw_ij = std::pow(1.0 - w, i + j);
    double B = omv_i * Bj;
    double C = omw_ij * Ck;
    double Au = 2.0 * dA;                                            // dA/du
    double Bv = 2.0 * omv_i * dBj - (i > 0 ? i * std::pow(1.0 - v, i - 1) * Bj : 0.0);
    double Cw = 2.0 * omw_ij * dCk - (i + j > 0 ? (i + j) * std::pow(1.0 - w, i + j - 1) * Ck : 0.0);
    phi[m] = c * A * B * C;
    // chain rule: du/dxi = 1/s, du/deta = u/s, du/dzeta = u/s; dv/deta = 1/t, dv/dzeta = v/t
    double gx = Au / s * B * C;
    double gy = Au * (u / s) * B * C + A * Bv / t * C;
    double gz = Au * (u / s) * B * C + A * Bv * (v / t) * C + A * B * Cw;
    dphi[0 * N + m] = c * gx;
    dphi[1 * N + m] = c * gy;
    dphi[2 * N + m] = c * gz;
  }
}

void legendre01(int pt, double tau, double* g, double* dg) {
  for (int a = 0; a <= pt; ++a) {
    double P, dP;
    jacobi(a, 0.0, 0.0, 2 * tau - 1, &P, &dP);
    g[a] = std::sqrt(2.0 * a + 1) * P;
    dg[a] = 2.0 * std::sqrt(2.0 * a + 1) * dP;
  }
}

static void invert_small(int n, const std::vector<double>& A, std::vector<double>& Ai) {
  // Gauss-Jordan with partial pivoting (n <= 5)
  std::vector<double> M(A);
  Ai.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Ai[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > std::fabs(M[piv * n + c])) piv = r;
    for (int k = 0; k < n; ++k) { std::swap(M[c * n + k], M[piv * n + k]); std::swap(Ai[c * n + k], Ai[piv * n + k]); }
    double d = M[c * n + c];
    for (int k = 0; k < n; ++k) { M[c * n + k] /= d; Ai[c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      for (int k = 0; k < n; ++k) { M[r * n + k] -= f * M[c * n + k]; Ai[r * n + k] -= f * Ai[c * n + k]; }
    }
  }
}

}  // namespace stdg

using namespace stdg;

static const double kRefV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// Map a unit-tet rule onto the reference sub-tet S_f (face f's vertices in increasing local
// order, then the centroid); weights scaled by |det| = 1/4.
static void sub_rule(const Rule& r, int f, std::vector<double>& xi, std::vector<double>& w) {
  int vs[3], c = 0;
  for (int k = 0; k < 4; ++k) if (k != f) vs[c++] = k;
  double P[4][3];
  for (int d = 0; d < 3; ++d) {
    P[0][d] = kRefV[vs[0]][d]; P[1][d] = kRefV[vs[1]][d]; P[2][d] = kRefV[vs[2]][d]; P[3][d] = 0.25;
  }
  for (int q = 0; q < r.n; ++q) {
    const double* s = &r.x[3 * q];
    for (int d = 0; d < 3; ++d)
      xi.push_back(P[0][d] + s[0] * (P[1][d] - P[0][d]) + s[1] * (P[2][d] - P[0][d]) + s[2] * (P[3][d] - P[0][d]));
    w.push_back(r.w[q] * 0.25);
  }
}

// phi at the face points (s,t) of a triangle rule laid on local vertices (a, b, c).
static void face_phi(int p, const Rule& tr, std::vector<double>& out) {
  const int N = nbasis(p);
  out.assign((size_t)kTriCodes * tr.n * N, 0.0);
  std::vector<double> phi(N), dphi(3 * N);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        if (a == b || b == c || a == c) continue;
        int code = tri_code(a, b, c);
        for (int q = 0; q < tr.n; ++q) {
          double s = tr.x[2 * q], t = tr.x[2 * q + 1], xi[3];
          for (int d = 0; d < 3; ++d) xi[d] = kRefV[a][d] + s * (kRefV[b][d] - kRefV[a][d]) + t * (kRefV[c][d] - kRefV[a][d]);
          dubiner_eval(p, xi, phi.data(), dphi.data());
          std::memcpy(&out[((size_t)code * tr.n + q) * N], phi.data(), N * sizeof(double));
        }
      }
}

extern "C" stdg_status stdg_reference_matrices(int p, int pt, stdg_ref** out) {
  if (!out) { set_error("stdg_reference_matrices: out is NULL"); return STDG_EINVAL; }
  *out = nullptr;
  if (p < 0 || p > 4 || pt < 0 || pt > 4) {
    set_error("stdg_reference_matrices: supported 0 <= p <= 4, 0 <= p_t <= 4 (got %d, %d)", p, pt);
    return STDG_EUNSUPPORTED;
  }
  stdg_ref* R = new (std::nothrow) stdg_ref;
  if (!R) { set_error("out of host memory"); return STDG_ENOMEM; }
  R->p = p; R->pt = pt; R->N = nbasis(p); R->Ng = pt + 1; R->Nst = R->N * R->Ng;
  const int N = R->N, Ng = R->Ng;
  const int nlin = p + 1, nnl = (3 * p + 2 + 1) / 2, ntl = pt + 1, ntn = (3 * pt + 2 + 1) / 2;
  // time basis and K_ab = g_a(1) g_b(1) - int g_a' g_b
  std::vector<double> g(Ng), dg(Ng);
  R->g0.resize(Ng); R->g1.resize(Ng);
  legendre01(pt, 0.0, R->g0.data(), dg.data());
  legendre01(pt, 1.0, R->g1.data(), dg.data());
  Rule tl = line_rule(ntl), tn = line_rule(ntn);
  R->K.assign(Ng * Ng, 0.0);
  for (int a = 0; a < Ng; ++a)
    for (int b = 0; b < Ng; ++b) R->K[a * Ng + b] = R->g1[a] * R->g1[b];
  R->nt_lin = tl.n; R->nt_nl = tn.n;
  for (int q = 0; q < tl.n; ++q) {
    legendre01(pt, tl.x[q], g.data(), dg.data());
    R->time_lin_tau.push_back(tl.x[q]); R->time_lin_w.push_back(tl.w[q]);
    for (int a = 0; a < Ng; ++a) { R->time_lin_g.push_back(g[a]); R->time_lin_dg.push_back(dg[a]); }
    for (int a = 0; a < Ng; ++a)
      for (int b = 0; b < Ng; ++b) R->K[a * Ng + b] -= tl.w[q] * dg[a] * g[b];
  }
  invert_small(Ng, R->K, R->Kinv);
  for (int q = 0; q < tn.n; ++q) {
    legendre01(pt, tn.x[q], g.data(), dg.data());
    R->time_nl_tau.push_back(tn.x[q]); R->time_nl_w.push_back(tn.w[q]);
    for (int a = 0; a < Ng; ++a) R->time_nl_g.push_back(g[a]);
  }
  // spatial tables
  Rule tetl = tet_rule(nlin), tetn = tet_rule(nnl), tril = tri_rule(nlin), trin = tri_rule(nnl);
  R->nq_lin = tetl.n; R->nqf_lin = tril.n; R->nq_nl = tetn.n; R->nqf_nl = trin.n;
  std::vector<double> phi(N), dphi(3 * N);
  for (int f = 0; f < 4; ++f) {
    std::vector<double> xi, w;
    sub_rule(tetl, f, xi, w);
    for (int q = 0; q < tetl.n; ++q) {
      dubiner_eval(p, &xi[3 * q], phi.data(), dphi.data());
      R->sub_lin_phi.insert(R->sub_lin_phi.end(), phi.begin(), phi.end());
      R->sub_lin_dphi.insert(R->sub_lin_dphi.end(), dphi.begin(), dphi.end());
    }
    R->sub_lin_xi.insert(R->sub_lin_xi.end(), xi.begin(), xi.end());
    R->sub_lin_w.insert(R->sub_lin_w.end(), w.begin(), w.end());
    std::vector<double> xn, wn;
    sub_rule(tetn, f, xn, wn);
    R->sub_nl_xi.insert(R->sub_nl_xi.end(), xn.begin(), xn.end());
    R->sub_nl_w.insert(R->sub_nl_w.end(), wn.begin(), wn.end());
  }
  R->tri_lin_st = tril.x; R->tri_lin_w = tril.w;
  R->tri_nl_st = trin.x; R->tri_nl_w = trin.w;
  face_phi(p, tril, R->face_lin_phi);
  face_phi(p, trin, R->face_nl_phi);
  R->tet_nl_xi = tetn.x; R->tet_nl_w = tetn.w;
  for (int q = 0; q < tetn.n; ++q) {
    dubiner_eval(p, &tetn.x[3 * q], phi.data(), dphi.data());
    R->tet_nl_phi.insert(R->tet_nl_phi.end(), phi.begin(), phi.end());
    R->tet_nl_dphi.insert(R->tet_nl_dphi.end(), dphi.begin(), dphi.end());
  }
  *out = R;
  return STDG_OK;
}

extern "C" void stdg_ref_destroy(stdg_ref* r) { delete r; }

extern "C" stdg_status stdg_ref_time_matrix(const stdg_ref* r, double* K) {
  if (!r || !K) { set_error("stdg_ref_time_matrix: NULL argument"); return STDG_EINVAL; }
  std::memcpy(K, r->K.data(), r->K.size() * sizeof(double));
  return STDG_OK;
}

extern "C" stdg_status stdg_ref_eval(const stdg_ref* r, const double* xi, int64_t n, double* phi, double* dphi) {
  if (!r || (!xi && n > 0) || n < 0) { set_error("stdg_ref_eval: invalid argument"); return STDG_EINVAL; }
  const int N = r->N;
  std::vector<double> p(N), d(3 * N);
  for (int64_t q = 0; q < n; ++q) {
    const double* x = xi + 3 * q;
    if (!(1.0 - x[1] - x[2] > 0.0) || !(1.0 - x[2] > 0.0)) { set_error("stdg_ref_eval: point outside the collapsed map"); return STDG_EINVAL; }
    dubiner_eval(r->p, x, p.data(), d.data());
    if (phi) std::memcpy(phi + q * N, p.data(), N * sizeof(double));
    if (dphi) std::memcpy(dphi + q * 3 * N, d.data(), 3 * N * sizeof(double));
  }
  return STDG_OK;
}

extern "C" stdg_status stdg_tet_rule(int n, double* xi, double* w) {
  if (n < 1 || n > 32 || !xi || !w) { set_error("stdg_tet_rule: invalid argument"); return STDG_EINVAL; }
  Rule t = tet_rule(n);
  std::memcpy(xi, t.x.data(), t.x.size() * sizeof(double));
  std::memcpy(w, t.w.data(), t.w.size() * sizeof(double));
  return STDG_OK;
}

extern "C" const char* stdg_last_error(void) { return stdg::last_error(); }
extern "C" const char* stdg_version(void) { return "stdg-gb300 0.1 (sm_103a)"; }
