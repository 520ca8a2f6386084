// Primary mesh, faces and dual-grid geometry (Sec. 2.2).  Host code.
//  * face j of the paper: keyed by its sorted vertex triple; l(j) = lower tet id (the paper
//    assigns l/r arbitrarily), r(j) = the other tet or -1 on the boundary B(Omega);
//  * faces ordered by (l(j), local face of l(j)); local face f = face opposite local vertex f;
//  * n_j: unit normal pointing from l(j) to r(j) (outward on the boundary);
//  * canonical vertex order of face j = l(j)'s local order; code_l / code_r record where
//    those three vertices sit among the local vertices of l and r (ordered-triple code);
//  * periodic meshes: a tet's geometry is its vertices' periodic images nearest to its first
//    vertex, faces are matched by vertex ids (every face interior), face geometry is in l(j)'s
//    frame.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>

#include "internal.h"

using namespace stdg;

namespace {
struct Key {
  int64_t a, b, c;
  bool operator==(const Key& o) const { return a == o.a && b == o.b && c == o.c; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : {k.a, k.b, k.c}) { h ^= (uint64_t)v; h *= 1099511628211ull; }
    return (size_t)h;
  }
};
struct Rec { int64_t l; int fl; int64_t r; int fr; };
}  // namespace

static stdg_status mesh_build(const double* verts, int64_t nv, const int64_t* tets, int64_t ne,
                              const double* period, stdg_mesh** out) {
  if (!out || !verts || !tets || nv <= 0 || ne <= 0) {
    set_error("stdg_mesh_create: invalid argument");
    return STDG_EINVAL;
  }
  *out = nullptr;
  stdg_mesh* M = new (std::nothrow) stdg_mesh;
  if (!M) { set_error("out of host memory"); return STDG_ENOMEM; }
  M->nv = nv; M->ne = ne;
  M->X.assign(verts, verts + 3 * nv);
  M->T.assign(tets, tets + 4 * ne);
  if (period) {
    M->periodic = true;
    for (int d = 0; d < 3; ++d) M->period[d] = period[d];
  }
  // coordinate d of local vertex k of tet i (periodic: the image nearest to the tet's vertex 0)
  auto vc = [M](int64_t i, int k, int d) {
    const double v = M->X[3 * M->T[4 * i + k] + d];
    if (!M->periodic || k == 0) return v;
    const double v0 = M->X[3 * M->T[4 * i] + d], L = M->period[d];
    return v0 + (v - v0) - L * std::nearbyint((v - v0) / L);
  };
  M->J.resize(9 * ne); M->Jinv.resize(9 * ne); M->detJ.resize(ne); M->bary.resize(3 * ne);
  for (int64_t i = 0; i < ne; ++i) {
    const int64_t* t = &M->T[4 * i];
    for (int k = 0; k < 4; ++k)
      if (t[k] < 0 || t[k] >= nv) {
        delete M; set_error("stdg_mesh_create: tet %lld has vertex id out of range", (long long)i);
        return STDG_EMESH;
      }
    double* J = &M->J[9 * i];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) J[d * 3 + c] = vc(i, c + 1, d) - vc(i, 0, d);  // column c = edge c
    double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                 J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(det > 0.0)) {
      delete M; set_error("stdg_mesh_create: tet %lld inverted or degenerate (det %g)", (long long)i, det);
      return STDG_EMESH;
    }
    M->detJ[i] = det;
    double* Ji = &M->Jinv[9 * i];
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det; Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    for (int d = 0; d < 3; ++d) M->bary[3 * i + d] = 0.25 * (vc(i, 0, d) + vc(i, 1, d) + vc(i, 2, d) + vc(i, 3, d));
  }
  std::unordered_map<Key, int64_t, KeyHash> idx;
  idx.reserve((size_t)(2.2 * ne) + 16);
  std::vector<Rec> recs;
  recs.reserve((size_t)(2.2 * ne) + 16);
  for (int64_t i = 0; i < ne; ++i)
    for (int f = 0; f < 4; ++f) {
      std::array<int64_t, 3> v;
      int c = 0;
      for (int k = 0; k < 4; ++k) if (k != f) v[c++] = M->T[4 * i + k];
      std::sort(v.begin(), v.end());
      Key key{v[0], v[1], v[2]};
      auto it = idx.find(key);
      if (it == idx.end()) {
        idx.emplace(key, (int64_t)recs.size());
        recs.push_back({i, f, -1, -1});
      } else {
        Rec& r = recs[it->second];
        if (r.r >= 0) {
          delete M; set_error("stdg_mesh_create: face shared by more than two tets");
          return STDG_EMESH;
        }
        r.r = i; r.fr = f;  // i > r.l because tets are visited in increasing order
      }
    }
  std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    return a.l != b.l ? a.l < b.l : a.fl < b.fl;
  });
  const int64_t nf = (int64_t)recs.size();
  M->nf = nf;
  M->left.resize(nf); M->right.resize(nf); M->fl.resize(nf); M->fr.resize(nf);
  M->fverts.resize(3 * nf); M->code_l.resize(nf); M->code_r.resize(nf);
  M->normal.resize(3 * nf); M->area.resize(nf); M->fcoords.resize(9 * nf); M->fshift.assign(3 * nf, 0.0);
  M->t2f.assign(4 * ne, -1); M->t2n.assign(4 * ne, -1); M->t2code.assign(4 * ne, -1);
  for (int64_t j = 0; j < nf; ++j) {
    const Rec& r = recs[j];
    M->left[j] = r.l; M->right[j] = r.r; M->fl[j] = r.fl; M->fr[j] = r.fr;
    int lv[3], c = 0;
    for (int k = 0; k < 4; ++k) if (k != r.fl) lv[c++] = k;
    for (int k = 0; k < 3; ++k) M->fverts[3 * j + k] = M->T[4 * r.l + lv[k]];
    M->code_l[j] = tri_code(lv[0], lv[1], lv[2]);
    M->t2f[4 * r.l + r.fl] = j;
    M->t2n[4 * r.l + r.fl] = r.r;
    M->t2code[4 * r.l + r.fl] = M->code_l[j];
    if (r.r >= 0) {
      int rv[3];
      for (int k = 0; k < 3; ++k) {
        rv[k] = -1;
        for (int q = 0; q < 4; ++q) if (M->T[4 * r.r + q] == M->fverts[3 * j + k]) rv[k] = q;
      }
      M->code_r[j] = tri_code(rv[0], rv[1], rv[2]);
      M->t2f[4 * r.r + r.fr] = j;
      M->t2n[4 * r.r + r.fr] = r.l;
      M->t2code[4 * r.r + r.fr] = M->code_r[j];
      M->nint++;
    } else {
      M->code_r[j] = -1;
      M->nbd++;
    }
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) M->fcoords[9 * j + 3 * k + d] = vc(r.l, lv[k], d);
    if (r.r >= 0 && M->periodic) {
      // the shared vertex fverts[0] in r's frame against l's frame: a whole number of periods
      int q0 = -1;
      for (int q = 0; q < 4; ++q) if (M->T[4 * r.r + q] == M->fverts[3 * j]) q0 = q;
      for (int d = 0; d < 3; ++d) M->fshift[3 * j + d] = M->fcoords[9 * j + d] - vc(r.r, q0, d);
    }
    const double* A = &M->fcoords[9 * j];
    const double* B = &M->fcoords[9 * j + 3];
    const double* C = &M->fcoords[9 * j + 6];
    double e1[3], e2[3], n[3];
    for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = C[d] - A[d]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const double O[3] = {vc(r.l, r.fl, 0), vc(r.l, r.fl, 1), vc(r.l, r.fl, 2)};  // l's vertex opposite the face
    double s = (O[0] - A[0]) * n[0] + (O[1] - A[1]) * n[1] + (O[2] - A[2]) * n[2];
    double sg = s > 0 ? -1.0 : 1.0;
    for (int d = 0; d < 3; ++d) M->normal[3 * j + d] = sg * n[d] / len;
    M->area[j] = 0.5 * len;
  }
  *out = M;
  return STDG_OK;
}

extern "C" stdg_status stdg_mesh_create(const double* verts, int64_t nv, const int64_t* tets,
                                        int64_t ne, stdg_mesh** out) {
  return mesh_build(verts, nv, tets, ne, nullptr, out);
}

extern "C" stdg_status stdg_mesh_create_periodic(const double* verts, int64_t nv, const int64_t* tets,
                                                 int64_t ne, const double* period, stdg_mesh** out) {
  if (!period || !(period[0] > 0.0) || !(period[1] > 0.0) || !(period[2] > 0.0)) {
    set_error("stdg_mesh_create_periodic: the period must be positive in every direction");
    return STDG_EINVAL;
  }
  return mesh_build(verts, nv, tets, ne, period, out);
}

extern "C" void stdg_mesh_destroy(stdg_mesh* m) { delete m; }

extern "C" stdg_status stdg_mesh_info(const stdg_mesh* m, int64_t* ne, int64_t* nf, int64_t* ni, int64_t* nb) {
  if (!m) { set_error("stdg_mesh_info: NULL mesh"); return STDG_EINVAL; }
  if (ne) *ne = m->ne;
  if (nf) *nf = m->nf;
  if (ni) *ni = m->nint;
  if (nb) *nb = m->nbd;
  return STDG_OK;
}

extern "C" stdg_status stdg_mesh_faces(const stdg_mesh* m, int64_t* l, int64_t* r, int32_t* fl, int32_t* fr) {
  if (!m) { set_error("stdg_mesh_faces: NULL mesh"); return STDG_EINVAL; }
  if (l) std::memcpy(l, m->left.data(), m->nf * sizeof(int64_t));
  if (r) std::memcpy(r, m->right.data(), m->nf * sizeof(int64_t));
  if (fl) std::memcpy(fl, m->fl.data(), m->nf * sizeof(int32_t));
  if (fr) std::memcpy(fr, m->fr.data(), m->nf * sizeof(int32_t));
  return STDG_OK;
}
