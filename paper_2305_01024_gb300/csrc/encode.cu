// encode.cu -- checksum encoding (Eq. 1-2 of Wu, Zhai et al., ICS'23) and
// the norms that scale the detection threshold; split-K reduction.
//
//   V[b][k]  = sum_{i in rows b*m_u .. } A[i][k]     (e^T A per row block)
//   Wt[b][k] = sum_{j in cols b*n_u .. } B[k][j]     (B e per column block)
//   nA[i] = ||A(i,:)||_2,  nB[j] = ||B(:,j)||_2
//
// All four are HBM-bound passes over A or B; the GEMM kernels read the
// small vectors V/Wt with each k-slice.
#include "internal.cuh"

namespace ftg {

// V: one thread per (row block, k); consecutive threads take consecutive k,
// so every warp-wide load is one contiguous 128-byte row segment.
__global__ void encode_colsum_kernel(const float* __restrict__ A, long long lda, int M, int K,
                                     int m_u, float* __restrict__ V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= K) return;
  const int r1 = min(M, (b + 1) * m_u);
  float s = 0.f;
  for (int r = b * m_u; r < r1; ++r) s += __ldg(A + (long long)r * lda + k);
  V[(long long)b * K + k] = s;
}

// Wt: one warp per row k of B; each lane sums a run of columns of one block
// and the runs of a block are combined with shuffles (blocks are aligned to
// the warp's 32-column window when n_u is a power of two <= 32, else a lane
// accumulates across windows of the same block).
__global__ void encode_rowsum_kernel(const float* __restrict__ B, long long ldb, int K, int N,
                                     int n_u, float* __restrict__ Wt) {
  const int warps = blockDim.x >> 5;
  const int k = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const float* row = B + (long long)k * ldb;
  const int nb = (N + n_u - 1) / n_u;
  if (n_u <= 32 && (n_u & (n_u - 1)) == 0) {
    for (int c0 = 0; c0 < N; c0 += 32) {
      const int c = c0 + lane;
      float v = c < N ? __ldg(row + c) : 0.f;
      for (int o = 1; o < n_u; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int b = c / n_u;
      if ((lane % n_u) == 0 && b < nb) Wt[(long long)b * K + k] = v;
    }
  } else {
    for (int b = 0; b < nb; ++b) {
      const int c1 = min(N, (b + 1) * n_u);
      float v = 0.f;
      for (int c = b * n_u + lane; c < c1; c += 32) v += __ldg(row + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) Wt[(long long)b * K + k] = v;
    }
  }
}

// nA: one warp per row.
__global__ void encode_rownorm_kernel(const float* __restrict__ A, long long lda, int M, int K,
                                      float* __restrict__ nA) {
  const int warps = blockDim.x >> 5;
  const int r = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= M) return;
  const float* row = A + (long long)r * lda;
  float s = 0.f;
  for (int k = lane; k < K; k += 32) {
    const float v = __ldg(row + k);
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) nA[r] = sqrtf(s);
}

// nB in two deterministic passes: partial sums of squares over chunks of
// 256 rows (one thread per column and chunk), then a sum over the chunks.
constexpr int kColnormChunk = 256;
__global__ void encode_colnorm_partial_kernel(const float* __restrict__ B, long long ldb, int K,
                                              int N, float* __restrict__ part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= N) return;
  const int k1 = min(K, (c + 1) * kColnormChunk);
  float s = 0.f;
  for (int k = c * kColnormChunk; k < k1; ++k) {
    const float v = __ldg(B + (long long)k * ldb + j);
    s = fmaf(v, v, s);
  }
  part[(long long)c * N + j] = s;
}
__global__ void encode_colnorm_finish_kernel(const float* __restrict__ part, int chunks, int N,
                                             float* __restrict__ nB) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(long long)c * N + j];
  nB[j] = sqrtf(s);
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

cudaError_t launch_encode(const float* A, long long lda, const float* B, long long ldb, int M,
                          int N, int K, int m_u, int n_u, float* V, float* Wt, float* nA,
                          float* nB, float* scratch, cudaStream_t st) {
  if (V) {
    dim3 g((K + 255) / 256, (M + m_u - 1) / m_u);
    encode_colsum_kernel<<<g, 256, 0, st>>>(A, lda, M, K, m_u, V);
  }
  if (Wt) encode_rowsum_kernel<<<(K + 7) / 8, 256, 0, st>>>(B, ldb, K, N, n_u, Wt);
  if (nA) encode_rownorm_kernel<<<(M + 7) / 8, 256, 0, st>>>(A, lda, M, K, nA);
  if (nB) {
    // scratch holds colnorm_scratch_floats(K, N) floats
    const int chunks = (K + kColnormChunk - 1) / kColnormChunk;
    encode_colnorm_partial_kernel<<<dim3((N + 255) / 256, chunks), 256, 0, st>>>(B, ldb, K, N, scratch);
    encode_colnorm_finish_kernel<<<(N + 255) / 256, 256, 0, st>>>(scratch, chunks, N, nB);
  }
  return cudaGetLastError();
}

long long colnorm_scratch_floats(int K, int N) {
  return (long long)((K + kColnormChunk - 1) / kColnormChunk) * N;
}

cudaError_t launch_splitk_reduce(const float* part, int splits, int M, int N, float alpha,
                                 float beta, float* C, long long ldc, cudaStream_t st) {
  const long long total = (long long)M * N;
  splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, splits, M, N, alpha,
                                                                          beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace ftg
