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

// B (K x N, ldb elements) -> Bt (N x ldk): 32 x 32 tiles through shared memory
template <typename E>
__global__ void tc_transpose_kernel(const E* __restrict__ B, long long ldb, int K, int N, E* __restrict__ Bt,
                                    long long ldk) {
  __shared__ E tile[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, n = n0 + tx;
    tile[r][tx] = (k < K && n < N) ? B[(long long)k * ldb + n] : E(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, k = k0 + tx;
    if (n < N && k < K) Bt[(long long)n * ldk + k] = tile[tx][r];
  }
}

// S[b][k] = sum over rows r in block b (bs rows) of X[r][k]; X is R x K (K-major)
template <int DT>
__global__ void tc_blocksum_kernel(const void* __restrict__ X, long long ldx, int R, int K, int bs,
                                   float* __restrict__ S) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= K) return;
  const int r1 = min(R, (b + 1) * bs);
  float s = 0.f;
  for (int r = b * bs; r < r1; ++r) s += ld_elem<DT>(X, (long long)r * ldx + k);
  S[(long long)b * K + k] = s;
}

// n[r] = ||X[r][:]||_2, one warp per row
template <int DT>
__global__ void tc_rownorm_kernel(const void* __restrict__ X, long long ldx, int R, int K,
                                  float* __restrict__ nrm) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= R) return;
  float s = 0.f;
  for (int k = lane; k < K; k += 32) {
    const float v = ld_elem<DT>(X, (long long)r * ldx + k);
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) nrm[r] = sqrtf(s);
}

// fro[b] = sqrt(sum_{r in block b} n[r]^2)
__global__ void tc_blockfro_kernel(const float* __restrict__ nrm, int R, int bs, int nb,
                                   float* __restrict__ fro) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  float s = 0.f;
  for (int r = b * bs; r < min(R, (b + 1) * bs); ++r) s = fmaf(nrm[r], nrm[r], s);
  fro[b] = sqrtf(s);
}

// s0[b]: power of two with max_k |S[b][k]| * s0 in (224, 448]  (fp8 only)
__global__ void tc_blockscale_kernel(const float* __restrict__ S, int K, float* __restrict__ s0) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  float m = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, fabsf(S[(long long)b * K + k]));
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
    s0[b] = sc;
  }
}

// Pieces of S[b][k] into P[(b*TC_CS_SLOTS + c)][k] (unused slots zero) and
// their multipliers scale[b*TC_CS_SLOTS + c].
template <int DT>
__global__ void tc_pieces_kernel(const float* __restrict__ S, int nb, int K, long long ldp,
                                 void* __restrict__ P, float* __restrict__ scale, const float* __restrict__ s0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  constexpr int NS = TC_CS_SLOTS;
  if (blockIdx.x == 0 && threadIdx.x < NS) {
    const int c = threadIdx.x;
    float m = 0.f;
    if (DT == 0) {
      m = c < 3 ? 1.f : 0.f;
    } else if (c < 5) {
      m = s0[b];
      for (int q = 0; q < c; ++q) m *= 16.f;
      m = 1.f / m;
    }
    scale[b * NS + c] = m;
  }
  if (k >= K) return;
  float x = S[(long long)b * K + k];
  if constexpr (DT == 0) {
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(P);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
    for (int c = 0; c < NS; ++c) {
      const __nv_bfloat16 v = c == 0 ? hi : c == 1 ? mid : c == 2 ? lo : __float2bfloat16_rn(0.f);
      out[(long long)(b * NS + c) * ldp + k] = v;
    }
  } else {
    __nv_fp8_storage_t* out = reinterpret_cast<__nv_fp8_storage_t*>(P);
    float sc = s0[b];
    for (int c = 0; c < NS; ++c) {
      __nv_fp8_storage_t q = 0;
      if (c < 5) {
        q = __nv_cvt_float_to_fp8(x * sc, __NV_SATFINITE, __NV_E4M3);
        __nv_fp8_e4m3 qq;
        qq.__x = q;
        x -= float(qq) / sc;
        sc *= 16.f;
      }
      out[(long long)(b * NS + c) * ldp + k] = q;
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

// Everything the tensor-core kernel needs besides A and B, written into the
// caller's buffers (see TcPrepBuffers).
cudaError_t launch_tc_prep(int dt, const void* A, long long lda, const void* B, long long ldb, int M, int N,
                           int K, bool abft, const TcPrepBuffers& w, int* launches, cudaStream_t st) {
  {
    dim3 g((N + 31) / 32, (K + 31) / 32);
    if (dt == 0)
      tc_transpose_kernel<uint16_t><<<g, dim3(32, 8), 0, st>>>((const uint16_t*)B, ldb, K, N, (uint16_t*)w.Bt, w.ldk);
    else
      tc_transpose_kernel<uint8_t><<<g, dim3(32, 8), 0, st>>>((const uint8_t*)B, ldb, K, N, (uint8_t*)w.Bt, w.ldk);
    ++*launches;
  }
  if (!abft) return cudaGetLastError();
  const int tiles_m = (M + TC_DM - 1) / TC_DM, tiles_n = (N + TC_DN - 1) / TC_DN;
  auto blocksum = [&](const void* X, long long ldx, int R, int bs, float* S) {
    dim3 g((K + 255) / 256, (R + bs - 1) / bs);
    if (dt == 0) tc_blocksum_kernel<0><<<g, 256, 0, st>>>(X, ldx, R, K, bs, S);
    else tc_blocksum_kernel<1><<<g, 256, 0, st>>>(X, ldx, R, K, bs, S);
    ++*launches;
  };
  auto rownorm = [&](const void* X, long long ldx, int R, float* n) {
    if (dt == 0) tc_rownorm_kernel<0><<<(R + 7) / 8, 256, 0, st>>>(X, ldx, R, K, n);
    else tc_rownorm_kernel<1><<<(R + 7) / 8, 256, 0, st>>>(X, ldx, R, K, n);
    ++*launches;
  };
  auto pieces = [&](const float* S, int nb, void* P, float* scale, float* s0) {
    if (dt == 1) {
      tc_blockscale_kernel<<<nb, 256, 0, st>>>(S, K, s0);
      ++*launches;
    }
    dim3 g((K + 255) / 256, nb);
    if (dt == 0) tc_pieces_kernel<0><<<g, 256, 0, st>>>(S, nb, K, w.ldk, P, scale, s0);
    else tc_pieces_kernel<1><<<g, 256, 0, st>>>(S, nb, K, w.ldk, P, scale, s0);
    ++*launches;
  };
  blocksum(A, lda, M, TC_DM, w.Vf);
  blocksum(w.Bt, w.ldk, N, TC_DN, w.Wf);
  rownorm(A, lda, M, w.nA);
  rownorm(w.Bt, w.ldk, N, w.nB);
  tc_blockfro_kernel<<<(tiles_m + 127) / 128, 128, 0, st>>>(w.nA, M, TC_DM, tiles_m, w.froA);
  tc_blockfro_kernel<<<(tiles_n + 127) / 128, 128, 0, st>>>(w.nB, N, TC_DN, tiles_n, w.froB);
  *launches += 2;
  pieces(w.Vf, tiles_m, w.Vt, w.vscale, w.s0v);
  pieces(w.Wf, tiles_n, w.Wt, w.wscale, w.s0w);
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
