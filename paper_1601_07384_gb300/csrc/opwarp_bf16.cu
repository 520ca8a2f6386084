// Warp-per-tet operator kernels, bfloat16 blocks.
#include "opwarp.cuh"

namespace stdg {

cudaError_t warp_prepare_bf16(stdg_solver* s) { return warp_prepare_t<WBF16>(s, &s->wB, &s->wA); }

cudaError_t warp_launch_bf16(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale,
                             double pin_diag, double* dotpart) {
  return launch_warp<WBF16>(s, s->wB, s->wA, x, y, pinned, kron, scale, pin_diag, 0.0, nullptr, dotpart);
}

// blocks of the launch: the number of dot partials it writes
int warp_blocks_bf16(stdg_solver* s) { return s->warp_grid[warp_kind<WBF16>() * 8 + s->Ng]; }

}  // namespace stdg
