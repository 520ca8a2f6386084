// Dispatch of the warp-per-tet operator kernels (opwarp.cuh; one translation unit per block
// precision so that they compile in parallel).
#include "solver.h"

namespace stdg {

cudaError_t warp_prepare_f32(stdg_solver* s);
cudaError_t warp_prepare_bf16(stdg_solver* s);
cudaError_t warp_prepare_df(stdg_solver* s);
cudaError_t warp_launch_f32(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale, double pin_diag,
                            double* dotpart);
cudaError_t warp_launch_bf16(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale, double pin_diag,
                             double* dotpart);
int warp_blocks_f32(stdg_solver* s);
int warp_blocks_bf16(stdg_solver* s);
cudaError_t warp_launch_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale, double pin_diag);
cudaError_t warp_launch_df_visc(stdg_solver* s, const double* x, double* y, double scale, double mass_coef,
                                const double* Kmass);

cudaError_t warp_prepare(stdg_solver* s, int precision) {
  if (precision == STDG_PREC_DF32) return warp_prepare_df(s);
  if (precision == STDG_PREC_MIXED_BF16) return warp_prepare_bf16(s);
  return warp_prepare_f32(s);
}

cudaError_t launch_apply_warp_lp(stdg_solver* s, const float* x, float* y, int pinned, int kron, float scale,
                                 float pin_diag, double* dotpart) {
  cudaError_t e;
  if (!s->capturing && (e = warp_prepare(s, s->lpkind)) != cudaSuccess) return e;
  if (s->lpkind == STDG_PREC_MIXED_BF16) return warp_launch_bf16(s, x, y, pinned, kron, scale, pin_diag, dotpart);
  return warp_launch_f32(s, x, y, pinned, kron, scale, pin_diag, dotpart);
}

int warp_blocks_lp(stdg_solver* s) {
  return s->lpkind == STDG_PREC_MIXED_BF16 ? warp_blocks_bf16(s) : warp_blocks_f32(s);
}

cudaError_t launch_apply_warp_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                                 double pin_diag) {
  cudaError_t e;
  if (!s->capturing && (e = warp_prepare(s, STDG_PREC_DF32)) != cudaSuccess) return e;
  return warp_launch_df(s, x, y, pinned, kron, scale, pin_diag);
}

cudaError_t launch_apply_warp_df_visc(stdg_solver* s, const double* x, double* y, double scale, double mass_coef,
                                      const double* Kmass) {
  cudaError_t e;
  if (!s->capturing && (e = warp_prepare(s, STDG_PREC_DF32)) != cudaSuccess) return e;
  if (!s->wdBv) return cudaErrorNotReady;
  return warp_launch_df_visc(s, x, y, scale, mass_coef, Kmass);
}

}  // namespace stdg
