// fp64.cuh -- launch parameters of the double / double-complex ABFT GEMM
// (fp64.cu), shared with the host entry points: the DGEMM / ZGEMM
// extension Section 6 names.
#pragma once
#include "internal.cuh"

namespace ftg {

// Operands row-major in the operand type (double, or interleaved (re, im)
// pairs); leading dimensions in elements of that type.
struct F64Params {
  int M, N, K;
  const void* A; long long lda;
  const void* B; long long ldb;
  void* C; long long ldc;
  double alpha_re, alpha_im, beta_re, beta_im;
  int beta_zero;
  // checksums (ABFT): V[tile_m][K], W[tile_n][K] (operand type), norms
  const void* V;
  const void* W;
  const double* nA;
  const double* nB;
  double lam_u;  // lambda * u: the norm term of the threshold
  double mu_u;   // mu * u: the checksum-growth term, mu_u * sqrt(k) * |checksum|
  int cadence;  // k-steps per verification period (>= 1)
  const Fault* faults;
  int nfaults;
  DevReport* rep;
  ftgemm_fault_record* recs;
  double* imag;  // complex: Im of (delta, residual_r, residual_c) per record slot
};

int f64_tile(bool cplx);
cudaError_t launch_f64_encode(bool cplx, const void* A, long long lda, const void* B, long long ldb, int M, int N,
                              int K, void* V, void* W, double* nA, double* nB, int* launches, cudaStream_t st);
cudaError_t launch_f64_gemm(bool cplx, bool abft, const F64Params& p, cudaStream_t st);

}  // namespace ftg
