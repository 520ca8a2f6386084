// Warp-per-tet operator kernels, bfloat16 blocks.
#include "opwarp.cuh"

namespace stdg {

cudaError_t warp_prepare_bf16(stdg_solver* s) { return warp_prepare_t<WBF16>(s, &s->wB, &s->wA); }

cudaError_t warp_launch_bf16(stdg_solver* s, const float* x, float* y, int pinned, int kron, double scale,
                             double pin_diag) {
  return launch_warp<WBF16>(s, s->wB, s->wA, x, y, pinned, kron, scale, pin_diag);
}

}  // namespace stdg
