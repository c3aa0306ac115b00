// encode.cu -- checksum encoding (Eq. 1-2 of Wu, Zhai et al., ICS'23), the
// norms that scale the detection threshold, the k-major operand layout the
// SIMT kernel streams with TMA, and the split-K reduction.
//
// Both GEMM operands are consumed k-major: B (K x N) as given, A as its
// transpose A^T (K x M).  On a k-major matrix X (K x L) one pass gives
//   S[b][k] = sum_{l in block b of n_u columns} X[k][l]   (block checksums)
//   n[l]    = ||X(:, l)||_2                               (column norms)
// so with X = A^T it yields e^T A per row block of A and ||A(i,:)||, and
// with X = B it yields B e per column block and ||B(:,j)||.
#include <algorithm>

#include "internal.cuh"

namespace ftg {

// A (M x K, lda) -> At (K x ldt): 32 x 32 tiles through shared memory, both
// the read and the write coalesced.
__global__ void transpose_kernel(const float* __restrict__ A, long long lda, int M, int K,
                                 float* __restrict__ At, long long ldt) {
  __shared__ float tile[32][33];
  const int m0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int m = m0 + r, k = k0 + tx;
    tile[r][tx] = (m < M && k < K) ? __ldg(A + (long long)m * lda + k) : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, m = m0 + tx;
    if (k < K && m < M) At[(long long)k * ldt + m] = tile[tx][r];
  }
}

// Row-padded copy X (R x C, ldx) -> Y (R x ldy), for operands whose stride
// or base address does not meet the 16-byte rule of TMA.
__global__ void copy_pad_kernel(const float* __restrict__ X, long long ldx, int R, int Cn,
                                float* __restrict__ Y, long long ldy) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)R * Cn) return;
  const int r = (int)(idx / Cn), c = (int)(idx % Cn);
  Y[(long long)r * ldy + c] = __ldg(X + (long long)r * ldx + c);
}

constexpr int kEncRows = 64;     // most k-rows per CTA
constexpr int kEncCols = 1024;   // columns per CTA (256 threads x 4)

// k-rows per CTA: enough CTAs to fill the GPU (about 4 per SM on 152 SMs)
// on small problems, at most kEncRows on large ones; a multiple of 8.
static int enc_rows(int K, int L) {
  const int colblocks = (L + kEncCols - 1) / kEncCols;
  const int want = std::max(1, 608 / colblocks);
  int rows = (K + want - 1) / want;
  rows = (rows + 7) / 8 * 8;
  return std::min(kEncRows, std::max(8, rows));
}

// One CTA: `rows` k-rows x kEncCols columns of a k-major X (float4 loads
// when `vec`: 16-byte aligned rows).  Block sums over groups of n_u columns
// (n_u a power of two, 2..1024) for every row, and partial column sums of
// squares over the CTA's rows.
__global__ void __launch_bounds__(256) encode_kmajor_kernel(const float* __restrict__ X, long long ldx,
                                                            int K, int L, int n_u, int rows, int vec,
                                                            float* __restrict__ S, long long lds,
                                                            float* __restrict__ part) {
  __shared__ float wpart[kEncRows][8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.x * kEncCols + tid * 4;
  const int k0 = blockIdx.y * rows;
  const int k1 = min(K, k0 + rows);
  const int g = n_u / 4;  // lanes per block when n_u <= 128
  float sq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {  // unrolled: several rows' loads in flight
    const float* row = X + (long long)k * ldx;
    float v[4];
    if (vec && c0 + 3 < L) {
      const float4 q4 = __ldg(reinterpret_cast<const float4*>(row + c0));
      v[0] = q4.x; v[1] = q4.y; v[2] = q4.z; v[3] = q4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = (c0 + q < L) ? __ldg(row + c0 + q) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sq[q] = fmaf(v[q], v[q], sq[q]);
    if (S) {
      float s = (v[0] + v[1]) + (v[2] + v[3]);
      if (n_u <= 128) {
        for (int o = 1; o < g; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (n_u >= 4) {
          if ((lane % g) == 0 && c0 < L) S[(long long)(c0 / n_u) * lds + k] = s;
        } else {
          // n_u == 2: each lane holds two blocks
          const float s0 = v[0] + v[1], s1 = v[2] + v[3];
          if (c0 < L) S[(long long)(c0 / 2) * lds + k] = s0;
          if (c0 + 2 < L) S[(long long)(c0 / 2 + 1) * lds + k] = s1;
        }
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) wpart[k - k0][warp] = s;
      }
    }
  }
  if (S && n_u > 128) {
    __syncthreads();
    // blocks of n_u columns = n_u/128 consecutive warps of this CTA
    const int wpb = n_u / 128;
    const int nblk = 8 / wpb;
    for (int t = tid; t < (k1 - k0) * nblk; t += 256) {
      const int kk = t / nblk, bl = t % nblk;
      const int cfirst = blockIdx.x * kEncCols + bl * n_u;
      if (cfirst >= L) continue;
      float s = 0.f;
      for (int w = 0; w < wpb; ++w) s += wpart[kk][bl * wpb + w];
      S[(long long)(cfirst / n_u) * lds + k0 + kk] = s;
    }
  }
  if (part) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c0 + q < L) part[(long long)blockIdx.y * L + c0 + q] = sq[q];
  }
}

__global__ void colnorm_finish_kernel(const float* __restrict__ part, int chunks, int L,
                                      float* __restrict__ nrm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(long long)c * L + j];
  nrm[j] = sqrtf(s);
}

// C = alpha * sum_s partial[s] + beta * C   (split-K; the sum is unprotected)
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M, int N,
                                     float alpha, float beta, float* C, long long ldc) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)M * N;
  if (idx >= total) return;
  const int r = (int)(idx / N), c = (int)(idx % N);
  float s = 0.f;
  for (int q = 0; q < splits; ++q) s += part[(long long)q * total + idx];
  float v = alpha * s;
  float* cp = C + (long long)r * ldc + c;
  *cp = beta != 0.f ? fmaf(beta, *cp, v) : v;
}

// ---------------------------------------------------------------------------

cudaError_t launch_transpose(const float* A, long long lda, int M, int K, float* At, long long ldt,
                             cudaStream_t st) {
  dim3 g((K + 31) / 32, (M + 31) / 32);
  transpose_kernel<<<g, dim3(32, 8), 0, st>>>(A, lda, M, K, At, ldt);
  return cudaGetLastError();
}

cudaError_t launch_copy_pad(const float* X, long long ldx, int R, int Cn, float* Y, long long ldy,
                            cudaStream_t st) {
  const long long total = (long long)R * Cn;
  copy_pad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, ldx, R, Cn, Y, ldy);
  return cudaGetLastError();
}

long long kmajor_scratch_floats(int K, int L) {
  const int rows = enc_rows(K, L);
  return (long long)((K + rows - 1) / rows) * L;
}

// S (may be null): [ceil(L/n_u)][lds] block sums; nrm (may be null): [L].
// scratch: kmajor_scratch_floats(K, L) floats when nrm is requested.
cudaError_t launch_encode_kmajor(const float* X, long long ldx, int K, int L, int n_u, float* S,
                                 long long lds, float* nrm, float* scratch, int* launches,
                                 cudaStream_t st) {
  if (n_u < 2 || n_u > kEncCols || (n_u & (n_u - 1))) return cudaErrorInvalidValue;
  const int vec = (ldx % 4 == 0) && (((uintptr_t)X & 15) == 0);
  const int rows = enc_rows(K, L);
  const int chunks = (K + rows - 1) / rows;
  dim3 g((L + kEncCols - 1) / kEncCols, chunks);
  encode_kmajor_kernel<<<g, 256, 0, st>>>(X, ldx, K, L, n_u, rows, vec, S, lds, nrm ? scratch : nullptr);
  *launches += 1;
  if (nrm) {
    colnorm_finish_kernel<<<(L + 255) / 256, 256, 0, st>>>(scratch, chunks, L, nrm);
    *launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(const float* part, int splits, int M, int N, float alpha,
                                 float beta, float* C, long long ldc, cudaStream_t st) {
  const long long total = (long long)M * N;
  splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, splits, M, N, alpha,
                                                                          beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace ftg
