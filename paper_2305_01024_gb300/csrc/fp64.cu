// fp64.cu -- double (DGEMM) and double-complex (ZGEMM) GEMM with online
// block-level ABFT, the extension Section 6 of Wu, Zhai et al. (ICS'23)
// names as future work.
//
// The scheme is the paper's, unchanged in kind: e^T A per block of rows and
// B e per block of columns (Eq. 1-2) ride along the K loop as one extra row
// and one extra column of the output tile (Eq. 4), every `cadence` k-steps
// the tile's row and column sums are compared with them against
// lambda * u * norms (u = 2^-53), and a single corrupted element is located
// and corrected (Section 4.2.1).  Complex values use |d| for the comparison.
//
// This part of GB300 has a low FP64 rate and no fast FP64 tensor path, so
// the kernel is a CUDA-core (DFMA) kernel: 256 threads, register tiles of
// 8 x 8 doubles (128 x 128 output tile) or 4 x 4 complex values (64 x 64),
// k-steps of 8 staged through shared memory with a register prefetch.  The
// checksum row and column cost one multiply-add per thread per k (1/64 of
// the data work for doubles, 1/32 for complex).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>

#include "fp64.cuh"

namespace ftg {

constexpr int F64_BK = 8;  // k-step

template <bool CPLX> struct F64Cfg;
template <> struct F64Cfg<false> {
  using T = double;
  static constexpr int BM = 128, BN = 128, TM = 8, TN = 8;
};
template <> struct F64Cfg<true> {
  using T = double2;
  static constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
};

// ---- scalar helpers: double and (re, im) pairs ----------------------------

__device__ __forceinline__ double f64_zero(double) { return 0.0; }
__device__ __forceinline__ double2 f64_zero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double f64_mac(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ double2 f64_mac(double2 c, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double f64_add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 f64_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double f64_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 f64_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double f64_abs(double a) { return fabs(a); }
__device__ __forceinline__ double f64_abs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double f64_abs2(double a) { return a * a; }
__device__ __forceinline__ double f64_abs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double f64_re(double a) { return a; }
__device__ __forceinline__ double f64_re(double2 a) { return a.x; }
__device__ __forceinline__ double f64_im(double) { return 0.0; }
__device__ __forceinline__ double f64_im(double2 a) { return a.y; }
__device__ __forceinline__ double f64_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 f64_shfl(double2 v, int o) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double f64_axpy(double w, double x, double y) { return fma(w, x, y); }
__device__ __forceinline__ double2 f64_axpy(double w, double2 x, double2 y) {
  return make_double2(fma(w, x.x, y.x), fma(w, x.y, y.y));
}
// real offset, or imaginary when `imag` (complex only)
__device__ __forceinline__ double f64_offset(double, double d, bool) { return d; }
__device__ __forceinline__ double2 f64_offset(double2, double d, bool imag) {
  return imag ? make_double2(0.0, d) : make_double2(d, 0.0);
}

// ---- encoding: checksum vectors and norms ----------------------------------

// out[b * ldo + c] = sum over rows r of block b (rows b*blk .. b*blk+blk-1) of
// X[r][c] (NORM: sqrt of the sum of |X[r][c]|^2, a double).  Block: 32
// columns x 8 row groups, summed in row-group order.
template <typename T, bool NORM>
__global__ void __launch_bounds__(256) f64_reduce_cols_kernel(const T* __restrict__ X, long long ld, int rows,
                                                              int cols, int blk, void* out, long long ldo) {
  using Acc = typename std::conditional<NORM, double, T>::type;
  __shared__ Acc part[8][32];
  const int cg = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cg, b = blockIdx.y;
  const int r0 = b * blk, r1 = min(rows, r0 + blk);
  Acc s = f64_zero(Acc{});
  if (c < cols) {
    for (int r = r0 + rg; r < r1; r += 8) {
      const T x = X[(long long)r * ld + c];
      if constexpr (NORM) s += f64_abs2(x);
      else s = f64_add(s, x);
    }
  }
  part[rg][cg] = s;
  __syncthreads();
  if (rg == 0 && c < cols) {
    Acc t = part[0][cg];
#pragma unroll
    for (int g = 1; g < 8; ++g) t = f64_add(t, part[g][cg]);
    if constexpr (NORM) reinterpret_cast<double*>(out)[(long long)b * ldo + c] = sqrt(t);
    else reinterpret_cast<T*>(out)[(long long)b * ldo + c] = t;
  }
}

// out[b * ldo + r] = sum over columns c of block b of X[r][c] (NORM: sqrt of
// the sum of |X[r][c]|^2).  One warp per (row, block), lanes strided over
// the block's columns, then an xor-tree across the lanes.
template <typename T, bool NORM>
__global__ void __launch_bounds__(256) f64_reduce_rows_kernel(const T* __restrict__ X, long long ld, int rows,
                                                              int cols, int blk, int nblk, void* out,
                                                              long long ldo) {
  const int lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (wid >= (long long)rows * nblk) return;  // warp-uniform
  const int r = (int)(wid / nblk), b = (int)(wid % nblk);
  const int c0 = b * blk, c1 = min(cols, c0 + blk);
  using Acc = typename std::conditional<NORM, double, T>::type;
  Acc s = f64_zero(Acc{});
  for (int c = c0 + lane; c < c1; c += 32) {
    const T x = X[(long long)r * ld + c];
    if constexpr (NORM) s += f64_abs2(x);
    else s = f64_add(s, x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = f64_add(s, f64_shfl(s, o));
  if (lane == 0) {
    if constexpr (NORM) reinterpret_cast<double*>(out)[(long long)b * ldo + r] = sqrt(s);
    else reinterpret_cast<T*>(out)[(long long)b * ldo + r] = s;
  }
}

// ---- the GEMM --------------------------------------------------------------


// The report of one verification event; the record's `reserved` field
// carries its slot so that the host can pair it with the imaginary parts.
__device__ void f64_report(const F64Params& p, ftgemm_fault_record r, double di, double dri, double dci) {
  atomicAdd(&p.rep->detected, 1ull);
  if (r.kind == K_CORRECTED) atomicAdd(&p.rep->corrected, 1ull);
  else if (r.kind == K_UNCORRECTABLE) atomicAdd(&p.rep->uncorrectable, 1ull);
  else atomicAdd(&p.rep->checksum_only, 1ull);
  const int slot = atomicAdd(&p.rep->n_records, 1);
  if (slot < p.rep->capacity) {
    r.reserved = slot;
    p.recs[slot] = r;
    if (p.imag) {
      p.imag[3 * (long long)slot] = di;
      p.imag[3 * (long long)slot + 1] = dri;
      p.imag[3 * (long long)slot + 2] = dci;
    }
  }
}

template <bool CPLX, bool ABFT>
__global__ void __launch_bounds__(256, 1) f64_gemm_kernel(const F64Params p) {
  using Cfg = F64Cfg<CPLX>;
  using T = typename Cfg::T;
  constexpr int BM = Cfg::BM, BN = Cfg::BN, TM = Cfg::TM, TN = Cfg::TN, BK = F64_BK;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;  // elements each thread stages per k-step
  static_assert(BM == 16 * TM && BN == 16 * TN && BN + BM <= 256, "thread layout");
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];
  __shared__ T vs[2][BK], ws[2][BK];
  __shared__ T rowsum[BM], colpart[8][BN], dres_r[BM], dres_c[BN];
  __shared__ double tau_r[BM], tau_c[BN], red[16];
  __shared__ unsigned long long best_r, best_c;
  __shared__ int nr, nc, ib, jb;
  __shared__ int fix_kind, fix_i, fix_j;  // 0 none, 1 correct acc, 2 reset row checksum, 3 reset column checksum
  __shared__ T fix_v;

  const T* A = reinterpret_cast<const T*>(p.A);
  const T* B = reinterpret_cast<const T*>(p.B);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31, warp = tid >> 5;
  const int tn = blockIdx.x, tm = blockIdx.y, tiles_n = gridDim.x;
  const int m0 = tm * BM, n0 = tn * BN;
  const int rows = min(BM, p.M - m0), cols = min(BN, p.N - n0);
  const int nks = (p.K + BK - 1) / BK;
  // the checksum element this thread carries: column checksum of column
  // `tid` (tid < BN) or row checksum of row `tid - BN` (BN <= tid < BN + BM)
  const bool own_c = tid < BN, own_r = tid >= BN && tid < BN + BM;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = f64_zero(T{});
  T csum = f64_zero(T{});
  double tau_own = 0.0;

  if constexpr (ABFT) {
    // Frobenius norms of the tile's rows of A and columns of B, then the
    // thresholds lambda*u*||A(i,:)||*||B(:,J)||_F and lambda*u*||A(I,:)||_F*||B(:,j)||
    double a2 = 0.0, b2 = 0.0;
    if (tid < rows) a2 = p.nA[m0 + tid] * p.nA[m0 + tid];
    if (tid < cols) b2 = p.nB[n0 + tid] * p.nB[n0 + tid];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    if (lane == 0) {
      red[warp] = a2;
      red[8 + warp] = b2;
    }
    __syncthreads();
    double fa = 0.0, fb = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      fa += red[w];
      fb += red[8 + w];
    }
    fa = sqrt(fa);
    fb = sqrt(fb);
    if (own_c) tau_own = tid < cols ? p.lam_u * fa * p.nB[n0 + tid] : 0.0;
    if (own_r) tau_own = tid - BN < rows ? p.lam_u * p.nA[m0 + tid - BN] * fb : 0.0;
    if (own_c) tau_c[tid] = tau_own;
    if (own_r) tau_r[tid - BN] = tau_own;
  }

  // this tile's faults: [f_next, f_end) of the table sorted by (tile, k-step)
  int f_next = 0, f_end = 0, f_ks = INT_MAX;
  if (p.nfaults > 0) {
    const int tile = tm * tiles_n + tn;
    f_next = first_fault(p.faults, p.nfaults, tile);
    f_end = f_next;
    while (f_end < p.nfaults && p.faults[f_end].tile == tile) ++f_end;
    if (f_next < f_end) f_ks = p.faults[f_next].kstep;
  }

  // staging of one k-step into registers (zero outside the matrix)
  T ra[LA], rb[LB], rv = f64_zero(T{});
  auto load = [&](int s) {
    const int k0 = s * BK;
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q, r = e / BK, kk = e % BK;
      ra[q] = (m0 + r < p.M && k0 + kk < p.K) ? A[(long long)(m0 + r) * p.lda + k0 + kk] : f64_zero(T{});
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q, kk = e / BN, c = e % BN;
      rb[q] = (n0 + c < p.N && k0 + kk < p.K) ? B[(long long)(k0 + kk) * p.ldb + n0 + c] : f64_zero(T{});
    }
    if constexpr (ABFT) {
      if (tid < 2 * BK) {
        const int kk = tid % BK;
        const T* src = reinterpret_cast<const T*>(tid < BK ? p.V : p.W) + (long long)(tid < BK ? tm : tn) * p.K;
        rv = k0 + kk < p.K ? src[k0 + kk] : f64_zero(T{});
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[buf][e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[buf][e / BN][e % BN] = rb[q];
    }
    if constexpr (ABFT) {
      if (tid < BK) vs[buf][tid] = rv;
      else if (tid < 2 * BK) ws[buf][tid - BK] = rv;
    }
  };

  load(0);
  store(0);
  __syncthreads();
  for (int s = 0; s < nks; ++s) {
    const int buf = s & 1;
    if (s + 1 < nks) load(s + 1);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][(i >> 2) * 64 + ty * 4 + (i & 3)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][(j >> 2) * 64 + tx * 4 + (j & 3)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = f64_mac(acc[i][j], a[i], b[j]);
      if constexpr (ABFT) {
        // Eq. 4: c^c += (e^T A_I(:,k)) B_J(k,:),  c^r += A_I(:,k) (B_J(k,:) e)
        if (own_c) csum = f64_mac(csum, vs[buf][kk], Bs[buf][kk][tid]);
        else if (own_r) csum = f64_mac(csum, As[buf][kk][tid - BN], ws[buf][kk]);
      }
    }
    // faults scheduled after this k-step (Section 5.3): additive offsets
    while (f_ks == s) {
      const Fault F = p.faults[f_next];
      const bool imag = (F.target & 4) != 0;
      const int tg = F.target & 3;
      const T off = f64_offset(T{}, (double)F.delta, imag);
      if (tg == T_ACC) {
        if (ty == (F.row & 63) >> 2 && tx == (F.col & 63) >> 2) {
          // every element takes w * off with w = 1 only at the target: no
          // indexed access, so the accumulators stay in registers
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              const double w = ((i >> 2) * 64 + (i & 3) == (F.row & ~63) + (F.row & 3) &&
                                (j >> 2) * 64 + (j & 3) == (F.col & ~63) + (F.col & 3)) ? 1.0 : 0.0;
              acc[i][j] = f64_axpy(w, off, acc[i][j]);
            }
        }
      } else if (ABFT && tg == T_ROWSUM) {
        if (own_r && tid - BN == F.row) csum = f64_add(csum, off);
      } else if (ABFT && tg == T_COLSUM) {
        if (own_c && tid == F.col) csum = f64_add(csum, off);
      }
      ++f_next;
      f_ks = f_next < f_end ? p.faults[f_next].kstep : INT_MAX;
    }

    if constexpr (ABFT) {
      if ((s + 1) % p.cadence == 0 || s == nks - 1) {
        // row sums: across the 16 threads of a half-warp (tx), xor tree
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          T r = acc[i][0];
#pragma unroll
          for (int j = 1; j < TN; ++j) r = f64_add(r, acc[i][j]);
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) r = f64_add(r, f64_shfl(r, o));
          if (tx == 0) rowsum[(i >> 2) * 64 + ty * 4 + (i & 3)] = r;
        }
        // column sums: the two half-warps of a warp, then the 8 warps in order
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          T c = acc[0][j];
#pragma unroll
          for (int i = 1; i < TM; ++i) c = f64_add(c, acc[i][j]);
          c = f64_add(c, f64_shfl(c, 16));
          if (lane < 16) colpart[warp][(j >> 2) * 64 + tx * 4 + (j & 3)] = c;
        }
        if (tid == 0) {
          nr = 0;
          nc = 0;
          best_r = 0ull;
          best_c = 0ull;
          ib = INT_MAX;
          jb = INT_MAX;
          fix_kind = 0;
        }
        __syncthreads();
        T d = f64_zero(T{});
        bool flag = false;
        // this verification's threshold: the norm term plus the growth term
        // mu * u * sqrt(k) * |checksum| after k elements of K
        const double tau_now = tau_own + p.mu_u * sqrt((double)min((s + 1) * BK, p.K)) * f64_abs(csum);
        if (own_c) {
          T c = colpart[0][tid];
#pragma unroll
          for (int w = 1; w < 8; ++w) c = f64_add(c, colpart[w][tid]);
          colpart[0][tid] = c;  // the column sum, kept for a checksum reset
          d = f64_sub(c, csum);
          flag = tid < cols && f64_abs(d) > tau_now;
          dres_c[tid] = d;
          tau_c[tid] = tid < cols ? tau_now : 0.0;
        } else if (own_r) {
          d = f64_sub(rowsum[tid - BN], csum);
          flag = tid - BN < rows && f64_abs(d) > tau_now;
          dres_r[tid - BN] = d;
          tau_r[tid - BN] = tid - BN < rows ? tau_now : 0.0;
        }
        if (__syncthreads_or(flag)) {
          // rare path: count, then the largest |d|/tau (exact in double;
          // ties to the smaller index)
          double score = 0.0;
          if (flag) {
            const double a = f64_abs(d);
            score = tau_now > 0.0 ? a / tau_now : __longlong_as_double(0x7ff0000000000000ll);
            atomicAdd(own_c ? &nc : &nr, 1);
            atomicMax(own_c ? &best_c : &best_r, (unsigned long long)__double_as_longlong(score));
          }
          __syncthreads();
          if (flag && (unsigned long long)__double_as_longlong(score) == (own_c ? best_c : best_r))
            atomicMin(own_c ? &jb : &ib, own_c ? tid : tid - BN);
          __syncthreads();
          if (tid == 0) {
            const int ir = nr ? ib : -1, jc = nc ? jb : -1;
            const T dR = ir >= 0 ? dres_r[ir] : f64_zero(T{});
            const T dC = jc >= 0 ? dres_c[jc] : f64_zero(T{});
            const double tR = ir >= 0 ? tau_r[ir] : 0.0, tC = jc >= 0 ? tau_c[jc] : 0.0;
            ftgemm_fault_record rec;
            rec.tile_m = tm;
            rec.tile_n = tn;
            rec.kstep = s;
            rec.row = ir >= 0 ? m0 + ir : -1;
            rec.col = jc >= 0 ? n0 + jc : -1;
            rec.problem = 0;
            rec.reserved = 0;
            rec.residual_r = f64_re(dR);
            rec.residual_c = f64_re(dC);
            rec.tau = tR + tC;
            T delta = f64_zero(T{});
            if (nr == 1 && nc == 1) {
              if (f64_abs(f64_sub(dR, dC)) <= tR + tC) {
                rec.kind = K_CORRECTED;
                delta = dR;
                fix_kind = 1;
                fix_i = ir;
                fix_j = jc;
                fix_v = dR;
              } else {
                rec.kind = K_UNCORRECTABLE;
              }
            } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
              // the checksum itself was hit: reset it from the data, C untouched
              rec.kind = K_CHECKSUM;
              delta = f64_zero(T{});
              delta = f64_sub(delta, nr ? dR : dC);  // checksum - data sum
              fix_kind = nr ? 2 : 3;
              fix_i = ir;
              fix_j = jc;
            } else {
              rec.kind = K_UNCORRECTABLE;
            }
            rec.delta = f64_re(delta);
            f64_report(p, rec, f64_im(delta), f64_im(dR), f64_im(dC));
          }
          __syncthreads();
          if (fix_kind == 1) {
            const int fr = fix_i, fc = fix_j;
            if (ty == (fr & 63) >> 2 && tx == (fc & 63) >> 2) {
              const T fv = fix_v;
#pragma unroll
              for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                  const double w = ((i >> 2) * 64 + (i & 3) == (fr & ~63) + (fr & 3) &&
                                    (j >> 2) * 64 + (j & 3) == (fc & ~63) + (fc & 3)) ? -1.0 : 0.0;
                  acc[i][j] = f64_axpy(w, fv, acc[i][j]);
                }
            }
          } else if (fix_kind == 2) {
            if (own_r && tid - BN == fix_i) csum = rowsum[fix_i];
          } else if (fix_kind == 3) {
            if (own_c && tid == fix_j) csum = colpart[0][fix_j];
          }
        }
      }
    }
    if (s + 1 < nks) store(buf ^ 1);
    __syncthreads();
  }

  // epilogue: C = alpha * acc + beta * C
  T* Cp = reinterpret_cast<T*>(p.C);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + (i >> 2) * 64 + ty * 4 + (i & 3);
    if (r >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + (j >> 2) * 64 + tx * 4 + (j & 3);
      if (c >= p.N) continue;
      T* dst = Cp + (long long)r * p.ldc + c;
      if constexpr (CPLX) {
        const double2 v = acc[i][j];
        double2 o = make_double2(p.alpha_re * v.x - p.alpha_im * v.y, p.alpha_re * v.y + p.alpha_im * v.x);
        if (!p.beta_zero) {
          const double2 q = *dst;
          o.x += p.beta_re * q.x - p.beta_im * q.y;
          o.y += p.beta_re * q.y + p.beta_im * q.x;
        }
        *dst = o;
      } else {
        const double o = p.alpha_re * acc[i][j];
        *dst = p.beta_zero ? o : fma(p.beta_re, *dst, o);
      }
    }
  }
}

// ---- launchers ---------------------------------------------------------------

int f64_tile(bool cplx) { return cplx ? F64Cfg<true>::BM : F64Cfg<false>::BM; }

// V[tiles_m][K], W[tiles_n][K] (operand type) and nA[M], nB[N] (double).
cudaError_t launch_f64_encode(bool cplx, const void* A, long long lda, const void* B, long long ldb, int M, int N,
                              int K, void* V, void* W, double* nA, double* nB, int* launches, cudaStream_t st) {
  const int T = f64_tile(cplx), tiles_m = (M + T - 1) / T, tiles_n = (N + T - 1) / T;
  const dim3 gv((K + 31) / 32, tiles_m), gn((N + 31) / 32, 1);
  const long long wW = (long long)K * tiles_n, wA = (long long)M;
  const int bW = (int)((wW + 7) / 8), bA = (int)((wA + 7) / 8);
  if (cplx) {
    const double2* a = reinterpret_cast<const double2*>(A);
    const double2* b = reinterpret_cast<const double2*>(B);
    f64_reduce_cols_kernel<double2, false><<<gv, 256, 0, st>>>(a, lda, M, K, T, V, K);
    f64_reduce_rows_kernel<double2, false><<<bW, 256, 0, st>>>(b, ldb, K, N, T, tiles_n, W, K);
    f64_reduce_rows_kernel<double2, true><<<bA, 256, 0, st>>>(a, lda, M, K, K, 1, nA, M);
    f64_reduce_cols_kernel<double2, true><<<gn, 256, 0, st>>>(b, ldb, K, N, K, nB, N);
  } else {
    const double* a = reinterpret_cast<const double*>(A);
    const double* b = reinterpret_cast<const double*>(B);
    f64_reduce_cols_kernel<double, false><<<gv, 256, 0, st>>>(a, lda, M, K, T, V, K);
    f64_reduce_rows_kernel<double, false><<<bW, 256, 0, st>>>(b, ldb, K, N, T, tiles_n, W, K);
    f64_reduce_rows_kernel<double, true><<<bA, 256, 0, st>>>(a, lda, M, K, K, 1, nA, M);
    f64_reduce_cols_kernel<double, true><<<gn, 256, 0, st>>>(b, ldb, K, N, K, nB, N);
  }
  *launches += 4;
  return cudaGetLastError();
}

cudaError_t launch_f64_gemm(bool cplx, bool abft, const F64Params& p, cudaStream_t st) {
  const int T = f64_tile(cplx);
  const dim3 grid((p.N + T - 1) / T, (p.M + T - 1) / T);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  if (cplx) {
    if (abft) f64_gemm_kernel<true, true><<<grid, 256, 0, st>>>(p);
    else f64_gemm_kernel<true, false><<<grid, 256, 0, st>>>(p);
  } else {
    if (abft) f64_gemm_kernel<false, true><<<grid, 256, 0, st>>>(p);
    else f64_gemm_kernel<false, false><<<grid, 256, 0, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace ftg
