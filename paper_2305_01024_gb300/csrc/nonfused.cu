// nonfused.cu -- kernels of the non-fused ABFT baseline: the GEMM runs as a
// sequence of rank-K_s updates C_acc += A(:, s) B(s, :) (plain GEMM
// launches), the checksums C^c = (e^T A) B and C^r = A (B e) are updated by
// separate GEMM launches (Eq. 4), and after every step a separate kernel
// verifies each 128 x 128 tile of the accumulator against them, locates and
// corrects (Section 4.2.1).  This is the scheme the paper compares its fused
// kernels with (Section 5.3); here it runs on the same GPU with the same
// checksum units, threshold and fault model as the fused kernel.
#include <algorithm>

#include "internal.cuh"

namespace ftg {

constexpr int NF_T = 128;  // tile of the verification units

// acc[r0 + row][c0 + col] += delta (or the tile's row / column checksum) for
// every fault scheduled at a k-step in [ks_lo, ks_hi).
__global__ void nonfused_inject_kernel(const Fault* __restrict__ f, int nf, int ks_lo, int ks_hi, int tiles_n,
                                       float* __restrict__ acc, long long ldacc, float* __restrict__ Cc,
                                       long long ldcc, float* __restrict__ CrT, long long ldcr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const Fault F = f[i];
  if (F.kstep < ks_lo || F.kstep >= ks_hi) return;
  const int tm = F.tile / tiles_n, tn = F.tile % tiles_n;
  const int gr = tm * NF_T + F.row, gc = tn * NF_T + F.col;
  if (F.target == T_ACC) atomicAdd(&acc[(long long)gr * ldacc + gc], F.delta);
  else if (F.target == T_ROWSUM) atomicAdd(&CrT[(long long)tn * ldcr + gr], F.delta);
  else atomicAdd(&Cc[(long long)tm * ldcc + gc], F.delta);
}

// One CTA per 128 x 128 tile: fp32 row and column sums of the accumulator
// against the tile's checksums (row sums vs CrT[tile_n][row], column sums
// vs Cc[tile_m][col]), thresholds lambda * u * norms plus the checksum-growth
// term grow * |checksum| (screened at half of them), fp64 confirmation of
// the flagged rows and columns, location, correction (or, for a checksum
// hit, the checksum's reset) and the report.
__global__ void __launch_bounds__(256) nonfused_verify_kernel(float* __restrict__ acc, long long ldacc, int M, int N,
                                                              float* __restrict__ Cc, long long ldcc,
                                                              float* __restrict__ CrT, long long ldcr,
                                                              const float* __restrict__ nA,
                                                              const float* __restrict__ nB, float lam_u, float grow,
                                                              int kstep,
                                                              DevReport* rep, ftgemm_fault_record* recs) {
  __shared__ float colpart[8][NF_T];
  __shared__ float rsum[NF_T], tr[NF_T], tcv[NF_T], red[8];
  __shared__ int flag_r[NF_T], flag_c[NF_T];
  __shared__ double dsum_r[NF_T], dsum_c[NF_T];
  __shared__ int nr, nc;
  __shared__ unsigned long long bestr, bestc;
  __shared__ float froA_s, froB_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = blockIdx.y, tn = blockIdx.x;
  const int r0 = tm * NF_T, c0 = tn * NF_T;
  const int rows = min(NF_T, M - r0), cols = min(NF_T, N - c0);

  // Frobenius norms of the tile's row block of A and column block of B
  {
    // threads 0..127: the tile's rows of A; 128..255: its columns of B
    float a = tid < rows ? nA[r0 + tid] * nA[r0 + tid] : 0.f;
    float b = (tid >= NF_T && tid - NF_T < cols) ? nB[c0 + tid - NF_T] * nB[c0 + tid - NF_T] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) red[warp] = warp < 4 ? a : b;
    __syncthreads();
    if (tid == 0) {
      froA_s = sqrtf((red[0] + red[1]) + (red[2] + red[3]));
      froB_s = sqrtf((red[4] + red[5]) + (red[6] + red[7]));
    }
  }
  // row sums (warp per row, lanes over 4 column groups) and column partials
  float cp[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = warp; i < NF_T; i += 8) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      v[q] = (i < rows && c < cols) ? acc[(long long)(r0 + i) * ldacc + c0 + c] : 0.f;
      cp[q] += v[q];
    }
    float s = (v[0] + v[1]) + (v[2] + v[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rsum[i] = s;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) colpart[warp][lane + 32 * q] = cp[q];
  __syncthreads();
  int flag = 0;
  if (tid < NF_T) {
    const int i = tid;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += colpart[w][i];
    const float crv = i < rows ? CrT[(long long)tn * ldcr + r0 + i] : 0.f;
    const float ccv = i < cols ? Cc[(long long)tm * ldcc + c0 + i] : 0.f;
    tr[i] = i < rows ? ft_tau(lam_u, nA[r0 + i], froB_s, grow, crv) : 0.f;
    tcv[i] = i < cols ? ft_tau(lam_u, froA_s, nB[c0 + i], grow, ccv) : 0.f;
    flag_r[i] = i < rows && fabsf(rsum[i] - crv) > kScreen * tr[i];
    flag_c[i] = i < cols && fabsf(s - ccv) > kScreen * tcv[i];
    flag = flag_r[i] | flag_c[i];
  }
  if (!__syncthreads_or(flag)) return;

  // fp64 confirmation of the flagged rows and columns
  if (tid == 0) { nr = 0; nc = 0; bestr = 0ull; bestc = 0ull; }
  if (tid < NF_T) { dsum_r[tid] = 0.0; dsum_c[tid] = 0.0; }
  __syncthreads();
  double cd[4] = {0.0, 0.0, 0.0, 0.0};  // this warp's rows of the flagged columns
  for (int i = warp; i < rows; i += 8) {
    const bool fr = flag_r[i] != 0;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < cols) {
        const double x = (double)acc[(long long)(r0 + i) * ldacc + c0 + c];
        if (fr) s += x;
        if (flag_c[c]) cd[q] += x;
      }
    }
    if (fr) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) dsum_r[i] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < cols && flag_c[c]) atomicAdd(&dsum_c[c], cd[q]);  // one add per warp
  }
  __syncthreads();
  if (tid < NF_T) {
    const int i = tid;
    if (flag_r[i]) {
      const double d = dsum_r[i] - (double)CrT[(long long)tn * ldcr + r0 + i];
      if (fabs(d) > (double)tr[i]) {
        atomicAdd(&nr, 1);
        atomicMax(&bestr, flag_key(flag_score((float)d, tr[i]), i));
      }
    }
    if (flag_c[i]) {
      const double d = dsum_c[i] - (double)Cc[(long long)tm * ldcc + c0 + i];
      if (fabs(d) > (double)tcv[i]) {
        atomicAdd(&nc, 1);
        atomicMax(&bestc, flag_key(flag_score((float)d, tcv[i]), i));
      }
    }
  }
  __syncthreads();
  if (tid == 0 && (nr | nc)) {
    const int ir = nr ? key_index(bestr) : -1, jc = nc ? key_index(bestc) : -1;
    const double dR = nr ? dsum_r[ir] - (double)CrT[(long long)tn * ldcr + r0 + ir] : 0.0;
    const double dC = nc ? dsum_c[jc] - (double)Cc[(long long)tm * ldcc + c0 + jc] : 0.0;
    const float tR = nr ? tr[ir] : 0.f, tC = nc ? tcv[jc] : 0.f;
    ftgemm_fault_record rec;
    rec.tile_m = tm; rec.tile_n = tn; rec.kstep = kstep;
    rec.problem = 0; rec.reserved = 0;
    rec.row = ir >= 0 ? r0 + ir : -1;
    rec.col = jc >= 0 ? c0 + jc : -1;
    rec.residual_r = dR; rec.residual_c = dC; rec.tau = (double)tR + (double)tC;
    rec.delta = 0.0;
    if (nr == 1 && nc == 1) {
      if (fabs(dR - dC) <= (double)tR + (double)tC) {
        rec.kind = K_CORRECTED; rec.delta = dR;
        float* x = &acc[(long long)(r0 + ir) * ldacc + c0 + jc];
        *x = (float)((double)*x - dR);
      } else {
        rec.kind = K_UNCORRECTABLE;
      }
    } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
      // the checksum itself was hit: reset it from the data, C untouched
      rec.kind = K_CHECKSUM; rec.delta = nr ? -dR : -dC;
      if (nr) CrT[(long long)tn * ldcr + r0 + ir] = (float)dsum_r[ir];
      else Cc[(long long)tm * ldcc + c0 + jc] = (float)dsum_c[jc];
    } else {
      rec.kind = K_UNCORRECTABLE;
    }
    report_event(rep, recs, rec);
  }
}

// C = alpha * acc + beta * C (beta == 0: C is not read)
__global__ void nonfused_epilogue_kernel(const float* __restrict__ acc, long long ldacc, int M, int N, float alpha,
                                         float beta, float* __restrict__ C, long long ldc) {
  const long long total = (long long)M * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / N, c = i % N;
    const float o = alpha * acc[r * ldacc + c];
    C[r * ldc + c] = beta != 0.f ? fmaf(beta, C[r * ldc + c], o) : o;
  }
}

cudaError_t launch_nonfused_inject(const Fault* f, int nf, int ks_lo, int ks_hi, int tiles_n, float* acc,
                                   long long ldacc, float* Cc, long long ldcc, float* CrT, long long ldcr,
                                   cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  nonfused_inject_kernel<<<(nf + 255) / 256, 256, 0, st>>>(f, nf, ks_lo, ks_hi, tiles_n, acc, ldacc, Cc, ldcc, CrT,
                                                           ldcr);
  return cudaGetLastError();
}

cudaError_t launch_nonfused_verify(float* acc, long long ldacc, int M, int N, float* Cc, long long ldcc,
                                   float* CrT, long long ldcr, const float* nA, const float* nB, float lam_u,
                                   float grow, int kstep, DevReport* rep, ftgemm_fault_record* recs, cudaStream_t st) {
  dim3 g((N + NF_T - 1) / NF_T, (M + NF_T - 1) / NF_T);
  nonfused_verify_kernel<<<g, 256, 0, st>>>(acc, ldacc, M, N, Cc, ldcc, CrT, ldcr, nA, nB, lam_u, grow, kstep, rep,
                                            recs);
  return cudaGetLastError();
}

cudaError_t launch_nonfused_epilogue(const float* acc, long long ldacc, int M, int N, float alpha, float beta,
                                     float* C, long long ldc, cudaStream_t st) {
  const long long total = (long long)M * N;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  nonfused_epilogue_kernel<<<blocks, 256, 0, st>>>(acc, ldacc, M, N, alpha, beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace ftg
