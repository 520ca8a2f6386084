// Warp-per-tet operator kernels, binary32 blocks.
#include "opwarp.cuh"

namespace stdg {

cudaError_t warp_prepare_f32(stdg_solver* s) { return warp_prepare_t<WF32>(s, &s->wB, &s->wA); }

cudaError_t warp_launch_f32(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale,
                             double pin_diag, double* dotpart) {
  return launch_warp<WF32>(s, s->wB, s->wA, x, y, pinned, kron, scale, pin_diag, 0.0, nullptr, dotpart);
}

// blocks of the launch: the number of dot partials it writes
int warp_blocks_f32(stdg_solver* s) { return s->warp_grid[warp_kind<WF32>() * 8 + s->Ng]; }

}  // namespace stdg
