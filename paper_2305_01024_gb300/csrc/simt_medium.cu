// simt_medium.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=32, n_tb=32, k_tb=8, m_w=16, n_w=32, m_t=4, n_t=4 at every checksum level;
// Table 1's "medium" tuple.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_medium(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<32, 32, 8, 16, 32, 4, 4>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
