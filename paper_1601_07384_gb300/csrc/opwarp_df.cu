// Warp-per-tet operator kernels, binary64-accurate products from binary32 (hi, lo) planes.
#include "opwarp.cuh"

namespace stdg {

cudaError_t warp_prepare_df(stdg_solver* s) {
  cudaError_t e = warp_prepare_t<WDF>(s, &s->wdB, &s->wdA);
  return e == cudaSuccess ? ensure_warp_visc_diag<WDF>(s, &s->wdBv) : e;
}

// the viscous operator of Eq. A1_mod: scale (B_i - Bvisc_i, A_lr) x + mass_coef |J_i| (K (x) I) x_i
cudaError_t warp_launch_df_visc(stdg_solver* s, const double* x, double* y, double scale, double mass_coef,
                                const double* Kmass) {
  return launch_warp<WDF>(s, s->wdBv, s->wdA, x, y, 0, 1, scale, 0.0, mass_coef, Kmass);
}

cudaError_t warp_launch_df(stdg_solver* s, const double* x, double* y, int pinned, int kron, double scale,
                             double pin_diag) {
  return launch_warp<WDF>(s, s->wdB, s->wdA, x, y, pinned, kron, scale, pin_diag);
}

}  // namespace stdg
