// simt_huge.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=128, n_tb=128, k_tb=8, m_w=32, n_w=64, m_t=8, n_t=8 at every checksum level;
// Table 1's "huge" tuple.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_huge(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<128, 128, 8, 32, 64, 8, 8>;
  return launch_simt_level<T>(level, maps, p, split, st);
}
}  // namespace ftg
