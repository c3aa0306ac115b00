// simt_large.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=64, n_tb=64, k_tb=8, m_w=32, n_w=64, m_t=8, n_t=8 at every checksum level;
// Table 1's "large" tuple.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_large(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<64, 64, 8, 32, 64, 8, 8>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
