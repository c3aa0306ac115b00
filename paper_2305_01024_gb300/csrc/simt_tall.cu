// simt_tall.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=32, n_tb=128, k_tb=8, m_w=16, n_w=64, m_t=4, n_t=8 at every checksum level;
// Table 1's "tall and skinny" tuple.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_tall(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<32, 128, 8, 16, 64, 4, 8>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
