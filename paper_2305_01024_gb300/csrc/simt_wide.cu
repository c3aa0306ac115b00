// simt_wide.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=128, n_tb=128, k_tb=16, m_w=64, n_w=64, m_t=16, n_t=8 (128 threads,
// 16 x 8 fragments) at every checksum level; not one of Table 1's tuples:
// its larger fragments leave room for the block checksum loads.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_wide(int level, const SimtMaps& maps, const SimtParams& p, int split,
                             cudaStream_t st) {
  using T = SimtTile<128, 128, 16, 64, 64, 16, 8>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
