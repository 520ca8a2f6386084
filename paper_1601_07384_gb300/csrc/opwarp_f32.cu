// Warp-per-tet operator kernels, binary32 blocks.
#include "opwarp.cuh"

namespace stdg {

cudaError_t warp_prepare_f32(stdg_solver* s) { return warp_prepare_t<WF32>(s, &s->wB, &s->wA); }

cudaError_t warp_launch_f32(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale,
                             double pin_diag, double* dotpart) {
  return launch_warp<WF32>(s, s->wB, s->wA, x, y, pinned, kron, scale, pin_diag, 0.0, nullptr, dotpart);
}

// the viscous operator of Eq. A1_mod with binary32 blocks: scale (B_i - Bvisc_i, A_lr) x +
// mass_coef |J_i| (Kmass (x) I) x_i.  Prepare outside stream capture; launch inside or outside.
cudaError_t warp_prepare_f32_visc(stdg_solver* s) {
  cudaError_t e = warp_prepare_t<WF32>(s, &s->wB, &s->wA);
  return e == cudaSuccess ? ensure_warp_visc_diag<WF32>(s, &s->wBv32) : e;
}
cudaError_t warp_launch_f32_visc(stdg_solver* s, const float* x, float* y, double scale, double mass_coef,
                                 const double* Kmass) {
  if (!s->wBv32) return cudaErrorNotReady;
  return launch_warp<WF32>(s, s->wBv32, s->wA, x, y, 0, 1, scale, 0.0, mass_coef, Kmass);
}

// blocks of the launch: the number of dot partials it writes
int warp_blocks_f32(stdg_solver* s) { return s->warp_grid[warp_kind<WF32>() * 8 + s->Ng]; }

}  // namespace stdg
