// simt_wide32.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8 (128 threads,
// 16 x 8 fragments) with a 2-deep ring of 32-wide k-steps: the same shared
// memory as 4 stages of 16, half the per-stage synchronisation and slot
// refills, and the block checksums updated over 16 k-rows per warp side.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_wide32(int level, const SimtMaps& maps, const SimtParams& p, int split,
                               cudaStream_t st) {
  using T = SimtTile<128, 128, 32, 64, 64, 16, 8, 2>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
