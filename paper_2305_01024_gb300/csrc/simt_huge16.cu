// simt_huge16.cu -- instantiates the fused-ABFT SGEMM for the tile tuple
// m_tb=128, n_tb=128, k_tb=16, m_w=32, n_w=64, m_t=8, n_t=8 at every checksum level;
// the "huge" tuple of Table 1 with k-steps of 16 instead of 8, a variant the
// table does not list.
#include "simt_ftgemm.cuh"

namespace ftg {
cudaError_t simt_launch_huge16(int level, const SimtMaps& maps, const SimtParams& p, int split,
                           cudaStream_t st) {
  using T = SimtTile<128, 128, 16, 32, 64, 8, 8>;
  return launch_simt_level<T>(level, maps, p, split, st);
}

// Load this tuple's kernels of every fp32 level into the current device's
// context (lazy module loading would otherwise load, and allocate, at the
// first launch of each).
cudaError_t simt_preload_huge16() {
  using T = SimtTile<128, 128, 16, 32, 64, 8, 8>;
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, simt_ftgemm_kernel<T, L_OFF, false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, simt_ftgemm_kernel<T, L_THREAD, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, simt_ftgemm_kernel<T, L_WARP, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, simt_ftgemm_kernel<T, L_BLOCK, true>);
  return e;
}
}  // namespace ftg
