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
// A (M x K, row-major) -> A^T (K x ldt), fused with the A side of the
// encoding (Eq. 1): V[b][k] = sum of the m_u rows of block b of column k
// (m_u a power of two, 2..128; 0 = no block sums) and the partial squared
// row norms of the 32 columns of this CTA's k-tile, part[k-tile][M].
// CTA tile: 128 rows x 32 columns through shared memory; A is read once.
__global__ void __launch_bounds__(256) transpose_encode_kernel(const float* __restrict__ A, long long lda, int M,
                                                               int K, float* __restrict__ At, long long ldt,
                                                               int m_u, float* __restrict__ V, long long ldv,
                                                               float* __restrict__ part) {
  __shared__ float tile[128][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 128;
  // load: warp w takes rows w, w + 8, ...; lane = column.  All 16 loads of
  // a thread are issued before any is used (bytes in flight hide latency).
  float vals[16];
  const int k = k0 + lane;
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int gi = m0 + warp + 8 * it;
    vals[it] = (gi < M && k < K) ? A[(long long)gi * lda + k] : 0.f;
  }
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int i = warp + 8 * it, gi = m0 + i;
    tile[i][lane] = vals[it];
    if (part) {
      float sq = vals[it] * vals[it];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0 && gi < M) part[(long long)blockIdx.x * M + gi] = sq;
    }
  }
  __syncthreads();
  // store: warp w writes A^T rows k0 + w, + 8, ...; lane covers rows
  // m = lane + 32 j of A (coalesced 128-byte segments)
  for (int kk = warp; kk < 32; kk += 8) {
    const int k = k0 + kk;
    if (k >= K) break;  // warp-uniform
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = tile[lane + 32 * j][kk];
      const int m = m0 + lane + 32 * j;
      if (m < M) At[(long long)k * ldt + m] = v[j];
    }
    if (V && m_u >= 2) {
      if (m_u <= 32) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float sv = v[j];
          for (int o = 1; o < m_u; o <<= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
          const int m = m0 + lane + 32 * j;
          if ((lane & (m_u - 1)) == 0 && m < M) V[(long long)(m / m_u) * ldv + k] = sv;
        }
      } else {
        // 64: j-pairs form a block; 128: all four
        const int per = m_u / 32;
        for (int jb = 0; jb < 4; jb += per) {
          float sv = 0.f;
          for (int j = jb; j < jb + per; ++j) sv += v[j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
          const int m = m0 + 32 * jb;
          if (lane == 0 && m < M) V[(long long)(m / m_u) * ldv + k] = sv;
        }
      }
    }
  }
}

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
  // rows are fetched four at a time, all four loads issued before use
  constexpr int AHEAD = 4;
  float4 buf[AHEAD];
  auto fetch = [&](int k) -> float4 {
    if (k >= k1) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float* row = X + (long long)k * ldx;
    if (vec && c0 + 3 < L) return __ldg(reinterpret_cast<const float4*>(row + c0));
    float t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = (c0 + q < L) ? __ldg(row + c0 + q) : 0.f;
    return make_float4(t[0], t[1], t[2], t[3]);
  };
  for (int kb = k0; kb < k1; kb += AHEAD) {
#pragma unroll
    for (int a = 0; a < AHEAD; ++a) buf[a] = fetch(kb + a);
#pragma unroll
  for (int a = 0; a < AHEAD; ++a) {
    const int k = kb + a;
    if (k >= k1) break;  // uniform over the CTA
    float v[4] = {buf[a].x, buf[a].y, buf[a].z, buf[a].w};
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

// nrm[j] = sqrt(sum over chunks of part[c][j]): a CTA finishes 32 columns,
// warp w summing chunks w, w + 8, ... (lane = column), then the 8 warps'
// sums in a fixed order.
__global__ void __launch_bounds__(256) colnorm_finish_kernel(const float* __restrict__ part, int chunks, int L,
                                                             float* __restrict__ nrm) {
  __shared__ float red[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < L) {
#pragma unroll 4
    for (int c = warp; c < chunks; c += 8) s += part[(long long)c * L + j];
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < L) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    nrm[j] = sqrtf(t);
  }
}

// Row-major A (M x K) read once: V[blk][k] = sum of A[i][k] over the m_u
// rows of block blk (e^T A per row block, Eq. 1) and squared row-norm
// partials per 256-column chunk (part[chunk][i], finished by
// colnorm_finish_kernel).  Block = (chunk, row block); warp w takes rows
// w, w+8, ..., four rows' loads issued before any is used; lane l the 8
// columns 8l..8l+7 of the chunk.  Column sums combine over the warps in
// warp order, so results are reproducible.
__global__ void __launch_bounds__(256) encode_rowmajor_kernel(const float* __restrict__ A, long long lda, int M,
                                                              int K, int m_u, int vec, float* __restrict__ V,
                                                              long long ldv, float* __restrict__ part) {
  __shared__ float colp[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * 256 + lane * 8, r0 = blockIdx.y * m_u, r1 = min(M, r0 + m_u);
  const bool fast = vec && k0 + 8 <= K;
  float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto row8 = [&](int r, float* v) {
    const float* p = A + (long long)r * lda + k0;
    if (fast) {
      const float4 u = __ldg(reinterpret_cast<const float4*>(p)), w = __ldg(reinterpret_cast<const float4*>(p) + 1);
      v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w; v[4] = w.x; v[5] = w.y; v[6] = w.z; v[7] = w.w;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = k0 + e < K ? p[e] : 0.f;
    }
  };
  auto take = [&](int r, const float* v) {
    float sq = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      cs[e] += v[e];
      sq = fmaf(v[e], v[e], sq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (part && lane == 0) part[(long long)blockIdx.x * M + r] = sq;
  };
  int r = r0 + warp;
  for (; r + 24 < r1; r += 32) {  // four rows of this warp, loads first
    float v[4][8];
#pragma unroll
    for (int g = 0; g < 4; ++g) row8(r + 8 * g, v[g]);
#pragma unroll
    for (int g = 0; g < 4; ++g) take(r + 8 * g, v[g]);
  }
  for (; r < r1; r += 8) {
    float v[8];
    row8(r, v);
    take(r, v);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) colp[warp][lane * 8 + e] = cs[e];
  __syncthreads();
  const int k = blockIdx.x * 256 + threadIdx.x;
  if (V && k < K) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += colp[w][threadIdx.x];
    V[(long long)blockIdx.y * ldv + k] = s;
  }
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

// A^T plus, when V / nrm are given, the A-side block sums and row norms;
// scratch: ceil(K/32) * M floats when nrm is requested.
cudaError_t launch_transpose_encode(const float* A, long long lda, int M, int K, float* At, long long ldt, int m_u,
                                    float* V, long long ldv, float* nrm, float* scratch, int* launches,
                                    cudaStream_t st) {
  if (V && (m_u < 2 || m_u > 128 || (m_u & (m_u - 1)))) return cudaErrorInvalidValue;
  dim3 g((K + 31) / 32, (M + 127) / 128);
  transpose_encode_kernel<<<g, 256, 0, st>>>(A, lda, M, K, At, ldt, V ? m_u : 0, V, ldv, nrm ? scratch : nullptr);
  ++*launches;
  if (nrm) {
    colnorm_finish_kernel<<<(M + 31) / 32, 256, 0, st>>>(scratch, (K + 31) / 32, M, nrm);
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_copy_pad(const float* X, long long ldx, int R, int Cn, float* Y, long long ldy,
                            cudaStream_t st) {
  const long long total = (long long)R * Cn;
  copy_pad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, ldx, R, Cn, Y, ldy);
  return cudaGetLastError();
}

// e^T A per m_u-row block (V, [ceil(M/m_u)][ldv]) and row norms of a
// row-major A (nA, [M]) reading A once; scratch: ceil(K/256) * M floats
// when nA is requested.
cudaError_t launch_encode_rowmajor(const float* A, long long lda, int M, int K, int m_u, float* V, long long ldv,
                                   float* nA, float* scratch, int* launches, cudaStream_t st) {
  const int vec = (lda % 4 == 0) && (((uintptr_t)A & 15) == 0);
  const int chunks = (K + 255) / 256;
  dim3 g(chunks, (M + m_u - 1) / m_u);
  encode_rowmajor_kernel<<<g, 256, 0, st>>>(A, lda, M, K, m_u, vec, V, ldv, nA ? scratch : nullptr);
  *launches += 1;
  if (nA) {
    colnorm_finish_kernel<<<(M + 31) / 32, 256, 0, st>>>(scratch, chunks, M, nA);
    *launches += 1;
  }
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
    colnorm_finish_kernel<<<(L + 31) / 32, 256, 0, st>>>(scratch, chunks, L, nrm);
    *launches += 1;
  }
  return cudaGetLastError();
}

// Coherence of every block, one CTA each: blocks 0..nb_a-1 of A (rows of
// m_u), then nb_b blocks of B (columns of n_u).  For block b of X with block
// sums S[b][0..K) and line norms nrm: ||S_b||_2 / (sqrt(count) *
// sqrt(sum of nrm^2 over the block)), in [0, 1]; 0 for an all-zero block.
// A feature of the learned threshold (1 when every line of the block is the
// same, about count^-1/2 for independent zero-mean lines).  Fixed-order
// reductions, so the value is reproducible.
__global__ void __launch_bounds__(256) block_coherence_kernel(const float* __restrict__ Sa, const float* __restrict__ Sb,
                                                              long long lds, int K, const float* __restrict__ nA,
                                                              const float* __restrict__ nB, int M, int N, int m_u,
                                                              int n_u, int nb_a, float* __restrict__ coA,
                                                              float* __restrict__ coB) {
  __shared__ float red[2][8];
  const bool side_a = (int)blockIdx.x < nb_a;
  const int b = side_a ? blockIdx.x : blockIdx.x - nb_a;
  const float* S = (side_a ? Sa : Sb) + (long long)b * lds;
  const float* nrm = side_a ? nA : nB;
  const int l0 = b * (side_a ? m_u : n_u), l1 = min(side_a ? M : N, l0 + (side_a ? m_u : n_u));
  float cs = 0.f, fr = 0.f;
  for (int k = threadIdx.x; k < K; k += 256) cs = fmaf(S[k], S[k], cs);
  for (int l = l0 + threadIdx.x; l < l1; l += 256) fr = fmaf(nrm[l], nrm[l], fr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cs += __shfl_xor_sync(0xffffffffu, cs, o);
    fr += __shfl_xor_sync(0xffffffffu, fr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = cs;
    red[1][threadIdx.x >> 5] = fr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float c = 0.f, f = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      c += red[0][w];
      f += red[1][w];
    }
    const float fro = sqrtf(f);
    (side_a ? coA : coB)[b] = fro > 0.f ? sqrtf(c) / (sqrtf((float)(l1 - l0)) * fro) : 0.f;
  }
}

cudaError_t launch_block_coherence(const float* V, const float* W, long long ldv, int K, const float* nA,
                                   const float* nB, int M, int N, int m_u, int n_u, float* coA, float* coB,
                                   cudaStream_t st) {
  const int nb_a = (M + m_u - 1) / m_u, nb_b = (N + n_u - 1) / n_u;
  block_coherence_kernel<<<nb_a + nb_b, 256, 0, st>>>(V, W, ldv, K, nA, nB, M, N, m_u, n_u, nb_a, coA, coB);
  return cudaGetLastError();
}

// Load the k-major layout and encoding kernels into the current device's
// context now (with lazy module loading a kernel is otherwise loaded, which
// allocates device memory, at its first launch).
cudaError_t preload_kmajor_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, transpose_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, copy_pad_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, encode_kmajor_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, colnorm_finish_kernel);
  return e;
}

cudaError_t launch_splitk_reduce(const float* part, int splits, int M, int N, float alpha,
                                 float beta, float* C, long long ldc, cudaStream_t st) {
  const long long total = (long long)M * N;
  splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, splits, M, N, alpha,
                                                                          beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace ftg
