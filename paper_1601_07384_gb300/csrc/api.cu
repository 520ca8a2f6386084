// C ABI entry points: solver construction (device preprocessing) and the hot-path calls.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "solver.h"

using namespace stdg;

namespace {

template <typename T>
stdg_status upload(stdg_solver* s, T** dst, const T* src, size_t count) {
  stdg_status e = dev_alloc(s, (void**)dst, count * sizeof(T));
  if (e != STDG_OK) return e;
  if (count && cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("cudaMemcpy upload failed");
    return STDG_ECUDA;
  }
  return STDG_OK;
}

stdg_status upload_i32(stdg_solver* s, int** dst, const int64_t* src, size_t count) {
  std::vector<int> tmp(count);
  for (size_t k = 0; k < count; ++k) tmp[k] = (int)src[k];
  return upload(s, dst, tmp.data(), count);
}

stdg_status upload_i32(stdg_solver* s, int** dst, const int32_t* src, size_t count) {
  return upload(s, dst, (const int*)src, count);
}

void set_time_mats(stdg_solver* s) {
  const int Ng = s->Ng;
  for (int q = 0; q < Ng * Ng; ++q) {
    s->tm.Tp[q] = s->dt * s->dt * s->Kinv[q];
    s->tm.K[q] = s->K[q];
    s->tm.Kinv[q] = s->Kinv[q];
  }
  for (int a = 0; a < Ng; ++a) { s->tm.g0[a] = s->g0[a]; s->tm.g1[a] = s->g1[a]; }
}

stdg_status check(stdg_solver* s) {
  if (!s) { set_error("NULL solver"); return STDG_EINVAL; }
  if (cudaSetDevice(s->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return STDG_ECUDA; }
  return STDG_OK;
}

}  // namespace

static stdg_status solver_create(const stdg_mesh* m, const stdg_ref* r, double dt, const stdg_solver_options* opts,
                                 void* stream, stdg_alloc_fn alloc_fn, stdg_free_fn free_fn, void* user,
                                 stdg_solver** out) {
  if (!m || !r || !out || !(dt > 0.0)) { set_error("stdg_solver_create: invalid argument"); return STDG_EINVAL; }
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("stdg_solver_create: no CUDA device available (this library has no CPU path)");
    return STDG_ECUDA;
  }
  if (m->ne >= (int64_t)1 << 31 || m->nf >= (int64_t)1 << 31) { set_error("mesh too large for int32 indices"); return STDG_EUNSUPPORTED; }
  stdg_solver* s = new (std::nothrow) stdg_solver;
  if (!s) { set_error("out of host memory"); return STDG_ENOMEM; }
  cudaGetDevice(&s->device);
  s->stream = (cudaStream_t)stream;
  s->alloc_fn = alloc_fn; s->free_fn = free_fn; s->alloc_user = user;
  s->opt.precision = STDG_PREC_FP64; s->opt.restart = 50; s->opt.max_iters = 200000; s->opt.graph_batch = 8;
  if (opts) {
    s->opt = *opts;
    if (s->opt.restart <= 0) s->opt.restart = 50;
    if (s->opt.restart > 60) { delete s; set_error("restart must be <= 60"); return STDG_EUNSUPPORTED; }
    if (s->opt.max_iters <= 0) s->opt.max_iters = 200000;
    if (s->opt.graph_batch <= 0) s->opt.graph_batch = 8;
    if (s->opt.graph_batch > 64) { delete s; set_error("graph_batch must be <= 64"); return STDG_EINVAL; }
    if (s->opt.precision < 0 || s->opt.precision > 3) { delete s; set_error("unknown precision %d", opts->precision); return STDG_EINVAL; }
  }
  {
    // "tma": block-staged TMA operator kernels; "warp": one warp per staged tet; default: CTAs of
    // several warps per staged tet
    const char* k = std::getenv("STDG_OP_KERNEL");
    s->op_warp = (k && std::strcmp(k, "tma") == 0) ? 0 : 1;
    s->op_cta = (k && std::strcmp(k, "warp") == 0) ? 0 : 1;
    const char* mi = std::getenv("STDG_MIXED_INNER");   // binary32 iterations per outer mixed step
    if (mi && std::atoi(mi) > 0 && std::atoi(mi) <= 1000) s->mix_inner = s->mix_inner_mg = std::atoi(mi);
    const char* mm = std::getenv("STDG_MIXED_M");       // directions kept by the outer flexible CG
    if (mm && std::atoi(mm) > 0 && std::atoi(mm) <= 16) s->mix_m = std::atoi(mm);
    const char* dw = std::getenv("STDG_DF_MIN_WARPS");  // pair kernel used when this many warps fit per SM
    if (dw && std::atoi(dw) > 0 && std::atoi(dw) <= 64) s->df_min_warps = std::atoi(dw);
    const char* vi = std::getenv("STDG_VISC_INNER64");
    s->visc_inner64 = vi && std::atoi(vi) == 1;
    const char* ck = std::getenv("STDG_CONV_KERNEL");  // "generic": no compile-time-degree convection kernel
    s->conv_generic = ck && std::strcmp(ck, "generic") == 0;
  }
  s->p = r->p; s->pt = r->pt; s->N = r->N; s->Ng = r->Ng; s->Nst = r->Nst;
  s->ne = m->ne; s->nf = m->nf; s->nint = m->nint; s->nbd = m->nbd;
  s->dt = dt;
  s->K = r->K; s->Kinv = r->Kinv; s->g0 = r->g0; s->g1 = r->g1;
  set_time_mats(s);
  s->nq_lin = r->nq_lin; s->nqf_lin = r->nqf_lin; s->nq_nl = r->nq_nl; s->nqf_nl = r->nqf_nl; s->nt_nl = r->nt_nl;
  s->time_nl_tau = r->time_nl_tau; s->time_nl_w = r->time_nl_w; s->time_nl_g = r->time_nl_g;
  stdg_status e = STDG_OK;
#define TRY(x) do { if ((e = (x)) != STDG_OK) { stdg_solver_destroy(s); return e; } } while (0)
  // mesh
  DevMesh& d = s->dm;
  d.ne = (int)m->ne; d.nf = (int)m->nf;
  TRY(upload_i32(s, &d.left, m->left.data(), m->nf));
  TRY(upload_i32(s, &d.right, m->right.data(), m->nf));
  TRY(upload_i32(s, &d.fl, m->fl.data(), m->nf));
  TRY(upload_i32(s, &d.fr, m->fr.data(), m->nf));
  TRY(upload_i32(s, &d.code_l, m->code_l.data(), m->nf));
  TRY(upload_i32(s, &d.code_r, m->code_r.data(), m->nf));
  TRY(upload_i32(s, &d.t2f, m->t2f.data(), 4 * m->ne));
  TRY(upload_i32(s, &d.t2n, m->t2n.data(), 4 * m->ne));
  TRY(upload_i32(s, &d.t2code, m->t2code.data(), 4 * m->ne));
  {
    // gather tables: per tet and local face, (face id << 1 | tet is r(j)) or -1 on the boundary
    std::vector<int> gf(4 * m->ne), gn(4 * m->ne);
    for (int64_t i = 0; i < m->ne; ++i)
      for (int f = 0; f < 4; ++f) {
        const int64_t j = m->t2f[4 * i + f], nb = m->t2n[4 * i + f];
        gf[4 * i + f] = nb >= 0 ? (int)((j << 1) | (m->left[j] == i ? 0 : 1)) : -1;
        gn[4 * i + f] = (int)nb;
      }
    TRY(upload(s, &s->gface, gf.data(), gf.size()));
    TRY(upload(s, &s->gnbr, gn.data(), gn.size()));
    // compact boundary index of every face (-1: interior), for data given at boundary points
    std::vector<int> bi(m->nf);
    int nb = 0;
    for (int64_t j = 0; j < m->nf; ++j) bi[j] = m->right[j] < 0 ? nb++ : -1;
    TRY(upload(s, &s->bidx, bi.data(), bi.size()));
  }
  std::vector<double> X0(3 * m->ne), fvx(9 * m->nf);
  for (int64_t i = 0; i < m->ne; ++i)
    for (int c = 0; c < 3; ++c) X0[3 * i + c] = m->X[3 * m->T[4 * i] + c];
  for (int64_t j = 0; j < m->nf; ++j)
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) fvx[9 * j + 3 * k + c] = m->fcoords[9 * j + 3 * k + c];
  TRY(upload(s, &d.X0, X0.data(), X0.size()));
  TRY(upload(s, &d.J, m->J.data(), m->J.size()));
  TRY(upload(s, &d.Jinv, m->Jinv.data(), m->Jinv.size()));
  TRY(upload(s, &d.detJ, m->detJ.data(), m->detJ.size()));
  TRY(upload(s, &d.bary, m->bary.data(), m->bary.size()));
  TRY(upload(s, &d.fvx, fvx.data(), fvx.size()));
  TRY(upload(s, &d.normal, m->normal.data(), m->normal.size()));
  TRY(upload(s, &d.area, m->area.data(), m->area.size()));
  TRY(upload(s, &d.fshift, m->fshift.data(), m->fshift.size()));
  // reference tables
  DevRef& t = s->dr;
  TRY(upload(s, &t.sub_lin_xi, r->sub_lin_xi.data(), r->sub_lin_xi.size()));
  TRY(upload(s, &t.sub_lin_w, r->sub_lin_w.data(), r->sub_lin_w.size()));
  TRY(upload(s, &t.sub_lin_phi, r->sub_lin_phi.data(), r->sub_lin_phi.size()));
  TRY(upload(s, &t.sub_lin_dphi, r->sub_lin_dphi.data(), r->sub_lin_dphi.size()));
  TRY(upload(s, &t.tri_lin_st, r->tri_lin_st.data(), r->tri_lin_st.size()));
  TRY(upload(s, &t.tri_lin_w, r->tri_lin_w.data(), r->tri_lin_w.size()));
  TRY(upload(s, &t.face_lin_phi, r->face_lin_phi.data(), r->face_lin_phi.size()));
  TRY(upload(s, &t.sub_nl_xi, r->sub_nl_xi.data(), r->sub_nl_xi.size()));
  TRY(upload(s, &t.sub_nl_w, r->sub_nl_w.data(), r->sub_nl_w.size()));
  TRY(upload(s, &t.tet_nl_xi, r->tet_nl_xi.data(), r->tet_nl_xi.size()));
  TRY(upload(s, &t.tet_nl_w, r->tet_nl_w.data(), r->tet_nl_w.size()));
  TRY(upload(s, &t.tet_nl_phi, r->tet_nl_phi.data(), r->tet_nl_phi.size()));
  TRY(upload(s, &t.tet_nl_dphi, r->tet_nl_dphi.data(), r->tet_nl_dphi.size()));
  TRY(upload(s, &t.tri_nl_st, r->tri_nl_st.data(), r->tri_nl_st.size()));
  TRY(upload(s, &t.tri_nl_w, r->tri_nl_w.data(), r->tri_nl_w.size()));
  TRY(upload(s, &t.face_nl_phi, r->face_nl_phi.data(), r->face_nl_phi.size()));
  TRY(upload(s, &s->d_ttau, r->time_nl_tau.data(), r->time_nl_tau.size()));
  TRY(upload(s, &s->d_tw, r->time_nl_w.data(), r->time_nl_w.size()));
  TRY(upload(s, &s->d_tg, r->time_nl_g.data(), r->time_nl_g.size()));
  // blocks
  const size_t NN = (size_t)s->N * s->N;
  TRY(dev_alloc(s, (void**)&s->Q, (size_t)m->nf * 6 * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->Mij, (size_t)m->nf * 2 * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->C, (size_t)m->nf * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->x0h, (size_t)m->nf * 4 * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->Aoff, (size_t)m->nf * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->Bdiag, (size_t)m->ne * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->Bvisc, (size_t)m->ne * NN * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->derr, sizeof(int)));
  cudaMemset(s->derr, 0, sizeof(int));
  TRY(dev_alloc(s, (void**)&s->P, (size_t)m->ne * s->Nst * sizeof(double)));
  TRY(dev_alloc(s, (void**)&s->V, (size_t)m->nf * 3 * s->Nst * sizeof(double)));
  cudaMemset(s->P, 0, (size_t)m->ne * s->Nst * sizeof(double));
  cudaMemset(s->V, 0, (size_t)m->nf * 3 * s->Nst * sizeof(double));
  MultiIdx mi{};
  std::vector<int> ex = multi_indices(s->p);
  for (size_t k = 0; k < ex.size(); ++k) mi.e[k] = (unsigned char)ex[k];
  cudaError_t ce = launch_face_blocks(d, t, s->p, s->N, r->nq_lin, r->nqf_lin, mi, s->Q, s->Mij, s->C, s->x0h, s->stream);
  if (ce == cudaSuccess) ce = launch_assemble(d, s->N, s->Q, s->Aoff, s->Bdiag, s->Bvisc, s->stream);
  // pair blocks (DF32, and the mixed modes' outer and viscous operators), unless the pair kernel would
  // run fewer than 6 warps per SM at this N, Ng: there the binary64 kernel is faster and serves instead
  if (ce == cudaSuccess && s->opt.precision != STDG_PREC_FP64 && (!s->op_warp || warp_df_warps_per_sm(s) >= s->df_min_warps))
    ce = s->op_warp ? warp_prepare(s, STDG_PREC_DF32) : df_build_blocks(s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) {
    set_error("device preprocessing failed: %s", cudaGetErrorString(ce));
    stdg_solver_destroy(s);
    return STDG_ECUDA;
  }
#undef TRY
  s->bc.kind = STDG_FIELD_ZERO;
  *out = s;
  return STDG_OK;
}

extern "C" stdg_status stdg_solver_create(const stdg_mesh* m, const stdg_ref* r, double dt,
                                          const stdg_solver_options* opts, void* stream, stdg_solver** out) {
  return solver_create(m, r, dt, opts, stream, nullptr, nullptr, nullptr, out);
}

extern "C" stdg_status stdg_solver_create_alloc(const stdg_mesh* m, const stdg_ref* r, double dt,
                                                const stdg_solver_options* opts, void* stream, stdg_alloc_fn alloc_fn,
                                                stdg_free_fn free_fn, void* user, stdg_solver** out) {
  if (!alloc_fn || !free_fn) { set_error("stdg_solver_create_alloc: alloc_fn and free_fn are both needed"); return STDG_EINVAL; }
  return solver_create(m, r, dt, opts, stream, alloc_fn, free_fn, user, out);
}

extern "C" void stdg_solver_destroy(stdg_solver* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream); else cudaDeviceSynchronize();
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : s->gev) cudaEventDestroy(e);
  for (cudaEvent_t e : s->sync_ev) if (e) cudaEventDestroy(e);
  if (s->cstream) cudaStreamDestroy(s->cstream);
  for (size_t k = s->allocs.size(); k-- > 0;) {
    if (s->free_fn) s->free_fn(s->allocs[k].p, s->allocs[k].bytes, (void*)s->stream, s->alloc_user);
    else cudaFree(s->allocs[k].p);
  }
  s->allocs.clear();
  if (s->hostbuf) cudaFreeHost(s->hostbuf);
  mg_free(s);
  delete s->gnn;
  delete s;
}

extern "C" stdg_status stdg_set_dt(stdg_solver* s, double dt) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!(dt > 0.0)) { set_error("dt must be positive"); return STDG_EINVAL; }
  s->dt = dt;
  set_time_mats(s);
  return STDG_OK;
}

extern "C" stdg_status stdg_set_max_iters(stdg_solver* s, int max_iters) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (max_iters < 1) { set_error("max_iters must be >= 1"); return STDG_EINVAL; }
  s->opt.max_iters = max_iters;
  return STDG_OK;
}

extern "C" stdg_status stdg_pressure_apply(stdg_solver* s, const double* x, double* y, int pinned) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!x || !y || x == y) { set_error("stdg_pressure_apply: x, y must be distinct device buffers"); return STDG_EINVAL; }
  return apply_pressure(s, x, y, pinned ? 1 : 0, 0, 1.0, -1.0);
}

extern "C" stdg_status stdg_pressure_apply_f32(stdg_solver* s, const float* x, float* y, int pinned) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!x || !y || (const void*)x == (const void*)y) { set_error("stdg_pressure_apply_f32: x, y must be distinct device buffers"); return STDG_EINVAL; }
  if (s->opt.precision != STDG_PREC_MIXED_F32 && s->opt.precision != STDG_PREC_MIXED_BF16) {
    set_error("stdg_pressure_apply_f32 needs a solver created with STDG_PREC_MIXED_F32 or _BF16");
    return STDG_EINVAL;
  }
  if (!s->lpB && !s->wB) {
    cudaError_t ce;
    if (s->op_warp) { s->lpkind = s->opt.precision; ce = warp_prepare(s, s->opt.precision); }
    else ce = lp_build_blocks(s, s->opt.precision);
    s->nlaunch += 2;
    if (ce != cudaSuccess) { set_error("low-precision block copies failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  }
  ++s->nlaunch;
  cudaError_t ce = launch_apply_lp(s, x, y, pinned ? 1 : 0, 0, 1.0f, -1.0f);
  if (ce != cudaSuccess) { set_error("low-precision operator launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

// y[a N] = d * x[a N] for the Ng pinned entries of tet 0
__global__ void k_pin_set(int N, int Ng, double d, const double* __restrict__ x, double* __restrict__ y) {
  const int a = threadIdx.x;
  if (a < Ng) y[a * N] = d * x[a * N];
}

extern "C" stdg_status stdg_pressure_apply_factored(stdg_solver* s, const double* x, double* y, int pinned) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!x || !y || x == y) { set_error("stdg_pressure_apply_factored: x, y must be distinct device buffers"); return STDG_EINVAL; }
  const size_t np = (size_t)s->ne * s->Nst, nv = (size_t)s->nf * 3 * s->Nst;
  if (!s->fac_x && (e = dev_alloc(s, (void**)&s->fac_x, np * sizeof(double))) != STDG_OK) return e;
  if (!s->fac_v && (e = dev_alloc(s, (void**)&s->fac_v, nv * sizeof(double))) != STDG_OK) return e;
  const double* xin = x;
  if (pinned) {                                   // x read as 0 at the pinned entries
    cudaMemcpyAsync(s->fac_x, x, np * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    k_pin_set<<<1, 32, 0, s->stream>>>(s->N, s->Ng, 0.0, x, s->fac_x);
    ++s->nlaunch;
    xin = s->fac_x;
  }
  // gradient and inverse momentum block per dual cell: v_j = -M_j^-1 (Q_lj x_l + Q_rj x_r) (boundary cells 0)
  cudaMemsetAsync(s->fac_v, 0, nv * sizeof(double), s->stream);
  cudaError_t ce = launch_update((int)s->nf, s->N, s->Ng, s->dm.left, s->dm.right, s->Q, s->fac_v, xin, s->dt,
                                 s->tm.Kinv, s->fac_v, s->stream);
  if (ce != cudaSuccess) { set_error("update launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  // divergence back into each tet: y_i = -Sum_j D_ij v_j = Sum_j D_ij M_j^-1 Q_j x
  ce = launch_rhs((int)s->ne, s->N, s->Ng, s->dm.t2f, s->dm.left, s->Q, s->fac_v, s->dt, pinned ? 1 : 0, y, s->stream);
  if (ce != cudaSuccess) { set_error("rhs launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  s->nlaunch += 2;
  if (pinned) {
    k_pin_set<<<1, 32, 0, s->stream>>>(s->N, s->Ng, -1.0, x, y);
    ++s->nlaunch;
  }
  return cudaGetLastError() == cudaSuccess ? STDG_OK : (set_error("pin launch failed"), STDG_ECUDA);
}

extern "C" stdg_status stdg_pressure_rhs(stdg_solver* s, const double* F, double* b, int pinned) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!F || !b) { set_error("stdg_pressure_rhs: NULL buffer"); return STDG_EINVAL; }
  ++s->nlaunch;
  cudaError_t ce = launch_rhs((int)s->ne, s->N, s->Ng, s->dm.t2f, s->dm.left, s->Q, F, -s->dt, pinned ? 1 : 0, b, s->stream);
  if (ce != cudaSuccess) { set_error("rhs launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

extern "C" stdg_status stdg_velocity_update(stdg_solver* s, const double* F, const double* dp, double* V) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!F || !dp || !V) { set_error("stdg_velocity_update: NULL buffer"); return STDG_EINVAL; }
  ++s->nlaunch;
  cudaError_t ce = launch_update((int)s->nf, s->N, s->Ng, s->dm.left, s->dm.right, s->Q, F, dp, s->dt,
                                 s->tm.Kinv, V, s->stream);
  if (ce != cudaSuccess) { set_error("update launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

extern "C" stdg_status stdg_solve(stdg_solver* s, const double* b, double* x, double tol, int method,
                                  stdg_solve_stats* st) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!b || !x || b == x || !(tol > 0.0)) { set_error("stdg_solve: invalid argument"); return STDG_EINVAL; }
  return solve_pressure(s, b, x, tol, method, st);
}

extern "C" stdg_status stdg_solve_noalloc(stdg_solver* s, const double* b, double* x, double tol,
                                          stdg_solve_stats* st) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!b || !x || b == x || !(tol > 0.0)) { set_error("stdg_solve_noalloc: invalid argument"); return STDG_EINVAL; }
  return solve_pressure_noalloc(s, b, x, tol, st);
}

extern "C" stdg_status stdg_velocity_moments(stdg_solver* s, const double* V, double* U) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  ++s->nlaunch;
  cudaError_t ce = launch_moments((int)s->nf, s->N, s->Ng, s->Mij, V, s->dt, U, s->stream);
  if (ce != cudaSuccess) { set_error("moments launch failed: %s", cudaGetErrorString(ce)); return STDG_ECUDA; }
  return STDG_OK;
}

extern "C" stdg_status stdg_get_blocks(const stdg_solver* s, double* Q, double* Mij, double* Aoff, double* Bdiag) {
  if (!s) { set_error("NULL solver"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  const size_t NN = (size_t)s->N * s->N;
  if (Q) STDG_CUDA(cudaMemcpy(Q, s->Q, s->nf * 6 * NN * sizeof(double), cudaMemcpyDeviceToHost));
  if (Mij) STDG_CUDA(cudaMemcpy(Mij, s->Mij, s->nf * 2 * NN * sizeof(double), cudaMemcpyDeviceToHost));
  if (Aoff) STDG_CUDA(cudaMemcpy(Aoff, s->Aoff, s->nf * NN * sizeof(double), cudaMemcpyDeviceToHost));
  if (Bdiag) STDG_CUDA(cudaMemcpy(Bdiag, s->Bdiag, s->ne * NN * sizeof(double), cudaMemcpyDeviceToHost));
  return STDG_OK;
}

extern "C" stdg_status stdg_get_state(const stdg_solver* s, double* P, double* V, int on_device, double* t) {
  if (!s) { set_error("NULL solver"); return STDG_EINVAL; }
  cudaSetDevice(s->device);
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // on the solver's stream, after its work, then wait: the caller reads the buffers on return
  if (P) STDG_CUDA(cudaMemcpyAsync(P, s->P, s->ne * s->Nst * sizeof(double), k, s->stream));
  if (V) STDG_CUDA(cudaMemcpyAsync(V, s->V, s->nf * 3 * s->Nst * sizeof(double), k, s->stream));
  STDG_CUDA(cudaStreamSynchronize(s->stream));
  if (t) *t = s->t;
  return STDG_OK;
}

extern "C" stdg_status stdg_set_state(stdg_solver* s, const double* P, const double* V, int on_device, double t) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // on the solver's stream, after its work, then wait: the caller may reuse the buffers on return
  if (P) STDG_CUDA(cudaMemcpyAsync(s->P, P, s->ne * s->Nst * sizeof(double), k, s->stream));
  if (V) STDG_CUDA(cudaMemcpyAsync(s->V, V, s->nf * 3 * s->Nst * sizeof(double), k, s->stream));
  STDG_CUDA(cudaStreamSynchronize(s->stream));
  s->t = t;
  return STDG_OK;
}


extern "C" stdg_status stdg_profile(stdg_solver* s, int enable) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (s->prof) prof_fold(s);
  if (enable && s->ev.empty()) {
    s->ev.resize(2 * 2048);
    for (auto& ev : s->ev) {
      if (cudaEventCreate(&ev) != cudaSuccess) { set_error("cudaEventCreate failed"); return STDG_ECUDA; }
    }
  }
  s->prof = enable != 0;
  s->ev_used = 0;
  s->op_ms = 0.0;
  s->op_launches = 0;
  s->nlaunch = 0;
  for (int q = 0; q < 4; ++q) { s->kind_ms[q] = 0.0; s->kind_n[q] = 0; }
  for (double& v : s->phase_ms) v = 0.0;
  return STDG_OK;
}

extern "C" stdg_status stdg_profile_read(stdg_solver* s, stdg_profile_stats* out) {
  stdg_status e = check(s);
  if (e != STDG_OK) return e;
  if (!out) { set_error("stdg_profile_read: NULL out"); return STDG_EINVAL; }
  if (s->prof) prof_fold(s);
  cudaStreamSynchronize(s->stream);
  out->kernel_launches = s->nlaunch;
  out->operator_launches = s->op_launches;
  out->operator_ms = s->op_ms;
  for (int q = 0; q < 4; ++q) { out->kind_launches[q] = s->kind_n[q]; out->kind_ms[q] = s->kind_ms[q]; }
  for (int q = 0; q < 8; ++q) out->phase_ms[q] = s->phase_ms[q];
  return STDG_OK;
}
