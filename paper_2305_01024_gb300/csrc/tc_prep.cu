// tc_prep.cu -- encoding pass of the tensor-core path and the operand
// quantizer.
//
// Encoding (Eq. 1-2 of Wu, Zhai et al., ICS'23) for a TC_DM x TC_DN
// (120 x 248) data tile of C:
//   v_I[k] = sum_{i in I} A[i][k]   (e^T A per 120-row block of A)
//   w_J[k] = sum_{j in J} B[k][j]   (B e per 248-column block of B)
// accumulated in fp32 from the operand values as stored, then split into
// pieces representable in the operand type so the MMA can carry them:
//   bf16: x = hi + mid + lo, each piece a bf16 (24 significant bits in all);
//   e4m3: x = sum_c q_c / s_c with s_c = s_0 * 16^c, q_c = e4m3(residual * s_c)
//         and s_0 a power of two putting the block's largest |x| near 448.
// Norms of the rows of A and of the columns of B (through B^T) scale the
// detection threshold.  B is also transposed to the K-major layout the MMA
// reads.
//
// Quantizer: bf16 by round-to-nearest-even; e4m3 with a per-tensor scale
// amax / 448 and round-to-nearest-even with saturation (OCP FP8).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.cuh"

namespace ftg {

template <int DT>
__device__ __forceinline__ float ld_elem(const void* base, long long idx) {
  if constexpr (DT == 0) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[idx]);
  } else {
    __nv_fp8_e4m3 q;
    q.__x = reinterpret_cast<const __nv_fp8_storage_t*>(base)[idx];
    return float(q);
  }
}

// Every encode kernel runs over a batch of problems (TcBatch): a problem's
// blocks of launch `kind` start at blk_start[kind], found by binary search.
#define TC_BLOCK_OF(KIND)                                  \
  const int pi = tc_find_block(b, KIND, blockIdx.x);       \
  const TcProblem& P = tc_problem(b, pi);                  \
  const int lb = (int)blockIdx.x - P.blk_start[KIND]

// B (K x N, ldb elements) -> Bt (N x ldk): 32 x 32 tiles through shared memory
template <typename E>
__global__ void tc_transpose_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(P_TRANSPOSE);
  __shared__ E tile[32][33];
  const E* B = reinterpret_cast<const E*>(P.B);
  E* Bt = reinterpret_cast<E*>(P.Bt);
  const int nbx = (P.N + 31) / 32;
  const int n0 = (lb % nbx) * 32, k0 = (lb / nbx) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, n = n0 + tx;
    tile[r][tx] = (k < P.K && n < P.N) ? B[(long long)k * P.ldb + n] : E(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, k = k0 + tx;
    if (n < P.N && k < P.K) Bt[(long long)n * P.ldk + k] = tile[tx][r];
  }
}

// S[blk][k] = sum over the rows r of block blk (bs rows) of X[r][k]; X is
// R x K, K contiguous.  side 0: A, 120-row blocks -> Vf; side 1: B^T,
// 248-row blocks -> Wf.
template <int DT, int SIDE>
__global__ void tc_blocksum_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(SIDE == 0 ? P_SUM_A : P_SUM_B);
  const void* X = SIDE == 0 ? P.A : P.Bt;
  const long long ldx = SIDE == 0 ? P.lda : P.ldk;
  const int R = SIDE == 0 ? P.M : P.N, bs = SIDE == 0 ? TC_DM : TC_DN;
  float* S = SIDE == 0 ? P.Vf : P.Wf;
  const int nkx = (P.K + 255) / 256;
  const int k = (lb % nkx) * 256 + threadIdx.x, blk = lb / nkx;
  if (k >= P.K) return;
  const int r1 = min(R, (blk + 1) * bs);
  float s = 0.f;
  for (int r = blk * bs; r < r1; ++r) s += ld_elem<DT>(X, (long long)r * ldx + k);
  S[(long long)blk * P.K + k] = s;
}

// n[r] = ||X[r][:]||_2, one warp per row (side 0: rows of A; 1: rows of B^T)
template <int DT, int SIDE>
__global__ void tc_rownorm_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(SIDE == 0 ? P_NORM_A : P_NORM_B);
  const void* X = SIDE == 0 ? P.A : P.Bt;
  const long long ldx = SIDE == 0 ? P.lda : P.ldk;
  const int R = SIDE == 0 ? P.M : P.N;
  float* nrm = SIDE == 0 ? P.nA : P.nB;
  const int r = lb * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= R) return;
  float s = 0.f;
  for (int k = lane; k < P.K; k += 32) {
    const float v = ld_elem<DT>(X, (long long)r * ldx + k);
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) nrm[r] = sqrtf(s);
}

// fro[blk] = sqrt(sum_{r in blk} n[r]^2) for the row blocks of A (first
// tiles_m indices) and the column blocks of B (next tiles_n)
__global__ void tc_blockfro_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(P_FRO);
  const int i = lb * blockDim.x + threadIdx.x;
  if (i >= P.tiles_m + P.tiles_n) return;
  const bool side_a = i < P.tiles_m;
  const int blk = side_a ? i : i - P.tiles_m;
  const int R = side_a ? P.M : P.N, bs = side_a ? TC_DM : TC_DN;
  const float* nrm = side_a ? P.nA : P.nB;
  float s = 0.f;
  for (int r = blk * bs; r < min(R, (blk + 1) * bs); ++r) s = fmaf(nrm[r], nrm[r], s);
  (side_a ? P.froA : P.froB)[blk] = sqrtf(s);
}

// s0[blk]: power of two with max_k |S[blk][k]| * s0 in (224, 448]  (fp8 only)
__global__ void tc_blockscale_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(P_SCALE);
  __shared__ float red[32];
  const bool side_a = lb < P.tiles_m;
  const int blk = side_a ? lb : lb - P.tiles_m;
  const float* S = (side_a ? P.Vf : P.Wf) + (long long)blk * P.K;
  float m = 0.f;
  for (int k = threadIdx.x; k < P.K; k += blockDim.x) m = fmaxf(m, fabsf(S[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    float sc = 1.f;
    if (t > 0.f) {
      int e;
      frexpf(448.f / t, &e);  // 448/t in [2^(e-1), 2^e)
      sc = ldexpf(1.f, e - 1);
    }
    (side_a ? P.s0v : P.s0w)[blk] = sc;
  }
}

// Pieces of S[blk][k] into Pc[(blk*TC_CS_SLOTS + c)][k] (unused slots zero)
// and their multipliers scale[blk*TC_CS_SLOTS + c]; row blocks of A first,
// then column blocks of B.
template <int DT>
__global__ void tc_pieces_kernel(const __grid_constant__ TcBatch b) {
  TC_BLOCK_OF(P_PIECES);
  constexpr int NS = TC_CS_SLOTS;
  const int nkx = (P.K + 255) / 256;
  const int k = (lb % nkx) * 256 + threadIdx.x, bi = lb / nkx;
  const bool side_a = bi < P.tiles_m;
  const int blk = side_a ? bi : bi - P.tiles_m;
  const float* S = side_a ? P.Vf : P.Wf;
  void* Pc = side_a ? P.Vt : P.Wt;
  float* scale = side_a ? P.vscale : P.wscale;
  const float* s0 = side_a ? P.s0v : P.s0w;
  if (lb % nkx == 0 && threadIdx.x < NS) {
    const int c = threadIdx.x;
    float m = 0.f;
    if (DT == 0) {
      m = c < 3 ? 1.f : 0.f;
    } else if (c < 5) {
      m = s0[blk];
      for (int q = 0; q < c; ++q) m *= 16.f;
      m = 1.f / m;
    }
    scale[blk * NS + c] = m;
  }
  if (k >= P.K) return;
  float x = S[(long long)blk * P.K + k];
  if constexpr (DT == 0) {
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(Pc);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
    for (int c = 0; c < NS; ++c) {
      const __nv_bfloat16 v = c == 0 ? hi : c == 1 ? mid : c == 2 ? lo : __float2bfloat16_rn(0.f);
      out[(long long)(blk * NS + c) * P.ldk + k] = v;
    }
  } else {
    __nv_fp8_storage_t* out = reinterpret_cast<__nv_fp8_storage_t*>(Pc);
    float sc = s0[blk];
    for (int c = 0; c < NS; ++c) {
      __nv_fp8_storage_t q = 0;
      if (c < 5) {
        q = __nv_cvt_float_to_fp8(x * sc, __NV_SATFINITE, __NV_E4M3);
        __nv_fp8_e4m3 qq;
        qq.__x = q;
        x -= float(qq) / sc;
        sc *= 16.f;
      }
      out[(long long)(blk * NS + c) * P.ldk + k] = q;
    }
  }
}

// ---- quantizer ------------------------------------------------------------

__global__ void amax_kernel(const float* __restrict__ x, long long n, unsigned int* __restrict__ amax_bits) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));  // |x| >= 0: bits order as values
}

__global__ void cast_bf16_kernel(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void cast_e4m3_kernel(const float* __restrict__ x, long long n, const unsigned int* __restrict__ amax_bits,
                                 __nv_fp8_storage_t* __restrict__ y, float* __restrict__ scale_out) {
  const float amax = __uint_as_float(*amax_bits);
  const float scale = amax > 0.f ? amax / 448.f : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = scale;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __nv_cvt_float_to_fp8(x[i] / scale, __NV_SATFINITE, __NV_E4M3);
}

// ---------------------------------------------------------------------------

// Blocks each batched encode launch gives one problem.
void tc_prep_blocks(const TcProblem& P, int out[P_KINDS]) {
  const int nkx = (P.K + 255) / 256;
  out[P_TRANSPOSE] = ((P.N + 31) / 32) * ((P.K + 31) / 32);
  out[P_SUM_A] = nkx * P.tiles_m;
  out[P_SUM_B] = nkx * P.tiles_n;
  out[P_NORM_A] = (P.M + 7) / 8;
  out[P_NORM_B] = (P.N + 7) / 8;
  out[P_FRO] = (P.tiles_m + P.tiles_n + 127) / 128;
  out[P_SCALE] = P.tiles_m + P.tiles_n;
  out[P_PIECES] = nkx * (P.tiles_m + P.tiles_n);
}

// The encode pass of a batch: B^T for every problem; with checksums also
// the block sums, norms, Frobenius norms and pieces.  total[kind] = blocks
// of each launch over the batch.
cudaError_t launch_tc_prep(int dt, bool abft, const TcBatch& b, const int total[P_KINDS], int* launches,
                           cudaStream_t st) {
  auto go = [&](int kind) { return total[kind] > 0; };
  if (go(P_TRANSPOSE)) {
    if (dt == 0) tc_transpose_kernel<uint16_t><<<total[P_TRANSPOSE], dim3(32, 8), 0, st>>>(b);
    else tc_transpose_kernel<uint8_t><<<total[P_TRANSPOSE], dim3(32, 8), 0, st>>>(b);
    ++*launches;
  }
  if (!abft) return cudaGetLastError();
  if (dt == 0) {
    tc_blocksum_kernel<0, 0><<<total[P_SUM_A], 256, 0, st>>>(b);
    tc_blocksum_kernel<0, 1><<<total[P_SUM_B], 256, 0, st>>>(b);
    tc_rownorm_kernel<0, 0><<<total[P_NORM_A], 256, 0, st>>>(b);
    tc_rownorm_kernel<0, 1><<<total[P_NORM_B], 256, 0, st>>>(b);
  } else {
    tc_blocksum_kernel<1, 0><<<total[P_SUM_A], 256, 0, st>>>(b);
    tc_blocksum_kernel<1, 1><<<total[P_SUM_B], 256, 0, st>>>(b);
    tc_rownorm_kernel<1, 0><<<total[P_NORM_A], 256, 0, st>>>(b);
    tc_rownorm_kernel<1, 1><<<total[P_NORM_B], 256, 0, st>>>(b);
  }
  tc_blockfro_kernel<<<total[P_FRO], 128, 0, st>>>(b);
  *launches += 5;
  if (dt == 1) {
    tc_blockscale_kernel<<<total[P_SCALE], 256, 0, st>>>(b);
    ++*launches;
  }
  if (dt == 0) tc_pieces_kernel<0><<<total[P_PIECES], 256, 0, st>>>(b);
  else tc_pieces_kernel<1><<<total[P_PIECES], 256, 0, st>>>(b);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_quantize(int dt, const float* x, long long n, void* y, unsigned int* amax_bits, float* scale,
                            int* launches, cudaStream_t st) {
  const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  if (dt == 0) {
    cast_bf16_kernel<<<grid, 256, 0, st>>>(x, n, (__nv_bfloat16*)y);
    ++*launches;
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  amax_kernel<<<grid, 256, 0, st>>>(x, n, amax_bits);
  cast_e4m3_kernel<<<grid, 256, 0, st>>>(x, n, amax_bits, (__nv_fp8_storage_t*)y, scale);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace ftg
