// simt_small.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=16, n_tb=16, k_tb=16, m_w=8, n_w=16, m_t=2, n_t=2 at every checksum level;
// Table 1's "small" tuple.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_small(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<16, 16, 16, 8, 16, 2, 2>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
