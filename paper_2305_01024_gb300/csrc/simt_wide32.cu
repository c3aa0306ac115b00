// simt_wide32.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=128, n_tb=128, k_tb=32, m_w=64, n_w=64, m_t=16, n_t=8 (128 threads,
// 16 x 8 fragments) with a 3-deep ring of 32-wide k-steps: half the
// per-stage synchronisation and slot refills of 16-wide steps, 96 KB of
// operands in flight, and the block checksums updated over 16 k-rows per warp
// side.  At block level a CTA takes 112,640 bytes of shared memory, so two
// CTAs (the register budget's 2 x 128 threads at 255 registers) still fit in
// an SM's 228 KB.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_wide32(int level, const SimtMaps& maps, const SimtParams& p, int split,
                               cudaStream_t st) {
  using T = SimtTile<128, 128, 32, 64, 64, 16, 8, 3>;
  return launch_simt_level<T>(level, maps, p, split, st);
}

// The detector of the offline scheme (Section 5.5) on the same tile: column
// checksums only, one verification per split, no correction.
cudaError_t simt_launch_wide32_detect(const SimtMaps& maps, const SimtParams& p, int split, cudaStream_t st) {
  using T = SimtTile<128, 128, 32, 64, 64, 16, 8, 3>;
  return launch_simt<T, L_DETECT>(maps, p, split, st);
}
}  // namespace ftg
