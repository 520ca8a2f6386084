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

// Warps per SM the pair kernel runs with at this solver's N and Ng (0 if it cannot run): its
// shared memory per warp grows as N^2 (blocks) and N Ng (x rows), and with too few warps per SM the
// binary64 kernel is faster.
int warp_df_warps_per_sm(stdg_solver* s) {
  cudaError_t e;
  switch (s->Ng) {
    case 1: e = warp_configure<WDF, 1>(s); break;
    case 2: e = warp_configure<WDF, 2>(s); break;
    case 3: e = warp_configure<WDF, 3>(s); break;
    case 4: e = warp_configure<WDF, 4>(s); break;
    default: e = warp_configure<WDF, 5>(s); break;
  }
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  const int kind = warp_kind<WDF>() * 8 + s->Ng;
  return s->warp_grid[kind] * s->warp_wpc[kind] / nsm;
}

}  // namespace stdg
