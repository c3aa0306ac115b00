// simt_ftgemm.cuh -- fp32 CUDA-core SGEMM with online ABFT fused into the
// K loop (Sections 3 and 4 of Wu, Zhai et al., ICS'23), for sm_103a.
//
// Structure (Section 3.1): a CTA computes an MT x NT tile of C; its KT-wide
// slices of A and B move global -> registers -> shared memory, double
// buffered so one __syncthreads per k-step suffices; a warp owns a WM x WN
// sub-tile arranged as 4 x 8 lanes, each lane an TM x TN fragment held in
// registers and built from float4 shared-memory reads (rows in chunks of 4,
// chunk stride 16, so a warp's reads are conflict-free broadcasts).
//
// ABFT (Section 4.2), template parameter LEVEL:
//   THREAD: each thread keeps the row checksums C_t e and column checksums
//           e^T C_t of its own fragment, updated with every rank-1 step from
//           the fragment sums e^T a and b e (Section 4.2.1).
//   WARP:   checksums of the warp tile; e^T A_w and B_w e come from the
//           encoding pass and are staged with each k-slice; every lane owns
//           TM/8 row and TN/4 column checksum entries (Section 4.2.2).
//   BLOCK:  checksums of the CTA tile; each thread owns one of the
//           MT + NT entries, updated once per k-step from the staged slice
//           and the encoded vectors e^T A_tb, B_tb e (Section 4.2.3).
// Verification runs every `cadence` k-steps and after the last one: the
// fragment/warp/tile row and column sums are compared with the checksums,
// one flagged row and one flagged column locate the fault and the row
// residual is subtracted there (Section 4.2.1); other patterns are reported.
// Faults are additive offsets on accumulator registers (Section 5.3).
#pragma once
#include <climits>

#include "internal.cuh"

namespace ftg {

template <int MT_, int NT_, int KT_, int WM_, int WN_, int TM_, int TN_>
struct SimtTile {
  static constexpr int MT = MT_, NT = NT_, KT = KT_, WM = WM_, WN = WN_, TM = TM_, TN = TN_;
  static constexpr int NTHR = (MT / TM) * (NT / TN);
  static constexpr int NWARP = NTHR / 32;
  static constexpr int WGM = MT / WM, WGN = NT / WN;  // warp grid
  static constexpr int LM = WM / TM, LN = WN / TN;    // lane grid (4 x 8)
  static constexpr int VM = TM < 4 ? TM : 4, VN = TN < 4 ? TN : 4;
  static constexpr int CM = TM / VM, CN = TN / VN;    // float-vector chunks
  static constexpr int LDA = MT + 4;                  // padded, transposed A slice
  static constexpr int LDB = NT;
  static constexpr int MINB = 512 / NTHR;             // CTAs per SM to aim for
  static_assert(LM * LN == 32, "a warp is 32 lanes");
  static_assert(WGM * WGN == NWARP, "warp grid covers the tile");
  static_assert((MT * KT) % NTHR == 0 && (NT * KT) % NTHR == 0, "even slice split");
};

template <class T, int LEVEL>
struct SimtSmem {
  static constexpr int NV = LEVEL == L_WARP ? T::WGM : 1;
  static constexpr int NW = LEVEL == L_WARP ? T::WGN : 1;
  float As[2][T::KT][T::LDA];
  float Bs[2][T::KT][T::LDB];
  float vs[2][T::KT][NV];
  float ws[2][T::KT][NW];
  float nA[T::MT];
  float nB[T::NT];
  float froAw[T::WGM];
  float froBw[T::WGN];
  float rowpart[LEVEL == L_BLOCK ? T::WGN : 1][T::MT];
  float colpart[LEVEL == L_BLOCK ? T::WGM : 1][T::NT];
  float cval[LEVEL == L_BLOCK ? T::MT + T::NT : 1];
  float tres[LEVEL == L_BLOCK ? T::MT + T::NT : 1];
  double sum_r, sum_c, fix_delta;
  unsigned long long bestr, bestc;
  int nr, nc;
  int fix_row, fix_col, reset_entry;
  float reset_value;
  float red[32];
};

template <int N>
__device__ __forceinline__ void lds_vec(float* d, const float* s) {
  if constexpr (N == 4) {
    float4 v = *reinterpret_cast<const float4*>(s);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else if constexpr (N == 2) {
    float2 v = *reinterpret_cast<const float2*>(s);
    d[0] = v.x; d[1] = v.y;
  } else {
    d[0] = s[0];
  }
}

template <int N>
__device__ __forceinline__ void ldg_vec(float* d, const float* s) {
  if constexpr (N == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(s));
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else if constexpr (N == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(s));
    d[0] = v.x; d[1] = v.y;
  } else {
    d[0] = __ldg(s);
  }
}

template <int N>
__device__ __forceinline__ void sts_vec(float* d, const float* s) {
  if constexpr (N == 4) {
    *reinterpret_cast<float4*>(d) = make_float4(s[0], s[1], s[2], s[3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2*>(d) = make_float2(s[0], s[1]);
  } else {
    d[0] = s[0];
  }
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Sum over the CTA; every thread gets the total.  Uses S.red.
template <class T, class Sm>
__device__ __forceinline__ float cta_sum(Sm& S, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < T::NWARP; ++w) t += S.red[w];
  return t;
}

template <class T, int LEVEL, bool VEC>
__global__ void __launch_bounds__(T::NTHR, T::MINB) simt_ftgemm_kernel(const SimtParams p) {
  constexpr int MT = T::MT, NT = T::NT, KT = T::KT, TM = T::TM, TN = T::TN;
  constexpr int NTHR = T::NTHR, LM = T::LM, LN = T::LN, VM = T::VM, VN = T::VN;
  using Sm = SimtSmem<T, LEVEL>;
  constexpr int NV = Sm::NV, NW = Sm::NW;
  __shared__ __align__(16) Sm S;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / T::WGN, wn = warp % T::WGN;
  const int tm = lane / LN, tn = lane % LN;
  const int tile_m = blockIdx.y, tile_n = blockIdx.x;
  const int row0 = tile_m * MT, col0 = tile_n * NT;
  const int M = p.M, N = p.N, K = p.K;
  const int ks0 = blockIdx.z * p.ks_per_split;
  const int ks1 = min(ks0 + p.ks_per_split, p.ksteps);
  const int arow = wm * T::WM + tm * VM;
  const int bcol = wn * T::WN + tn * VN;
  // tile-local row/column of fragment element i / j
#define FROW(i) (arow + ((i) / VM) * (LM * VM) + ((i) % VM))
#define FCOL(j) (bcol + ((j) / VN) * (LN * VN) + ((j) % VN))

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  // ---- checksum state ---------------------------------------------------
  constexpr int RPL = (TM + LN - 1) / LN;   // WARP: row entries per lane
  constexpr int CPL = (TN + LM - 1) / LM;   // WARP: column entries per lane
  constexpr int ENT = (MT + NT + NTHR - 1) / NTHR;  // BLOCK: entries per thread
  float cr[LEVEL == L_THREAD ? TM : 1], cc[LEVEL == L_THREAD ? TN : 1];
  float wr[LEVEL == L_WARP ? RPL : 1], wc[LEVEL == L_WARP ? CPL : 1];
  float bc[LEVEL == L_BLOCK ? ENT : 1];
#pragma unroll
  for (int i = 0; i < (LEVEL == L_THREAD ? TM : 1); ++i) cr[i] = 0.f;
#pragma unroll
  for (int j = 0; j < (LEVEL == L_THREAD ? TN : 1); ++j) cc[j] = 0.f;
#pragma unroll
  for (int x = 0; x < (LEVEL == L_WARP ? RPL : 1); ++x) wr[x] = 0.f;
#pragma unroll
  for (int y = 0; y < (LEVEL == L_WARP ? CPL : 1); ++y) wc[y] = 0.f;
#pragma unroll
  for (int q = 0; q < (LEVEL == L_BLOCK ? ENT : 1); ++q) bc[q] = 0.f;

  float froAt = 0.f, froBt = 0.f;  // THREAD: Frobenius norms of the fragment's rows/cols
  if constexpr (LEVEL != L_OFF) {
    for (int r = tid; r < MT; r += NTHR) S.nA[r] = (row0 + r < M) ? p.nA[row0 + r] : 0.f;
    for (int c = tid; c < NT; c += NTHR) S.nB[c] = (col0 + c < N) ? p.nB[col0 + c] : 0.f;
    __syncthreads();
    if constexpr (LEVEL == L_THREAD) {
#pragma unroll
      for (int i = 0; i < TM; ++i) froAt += S.nA[FROW(i)] * S.nA[FROW(i)];
#pragma unroll
      for (int j = 0; j < TN; ++j) froBt += S.nB[FCOL(j)] * S.nB[FCOL(j)];
      froAt = sqrtf(froAt);
      froBt = sqrtf(froBt);
    } else if constexpr (LEVEL == L_WARP) {
      float a = 0.f, b = 0.f;
      for (int r = lane; r < T::WM; r += 32) a += S.nA[wm * T::WM + r] * S.nA[wm * T::WM + r];
      for (int c = lane; c < T::WN; c += 32) b += S.nB[wn * T::WN + c] * S.nB[wn * T::WN + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0 && wn == 0) S.froAw[wm] = sqrtf(a);
      if (lane == 0 && wm == 0) S.froBw[wn] = sqrtf(b);
      __syncthreads();
    } else {
      float a = 0.f, b = 0.f;
      for (int r = tid; r < MT; r += NTHR) a += S.nA[r] * S.nA[r];
      for (int c = tid; c < NT; c += NTHR) b += S.nB[c] * S.nB[c];
      a = cta_sum<T>(S, a);
      b = cta_sum<T>(S, b);
      if (tid == 0) { S.froAw[0] = sqrtf(a); S.froBw[0] = sqrtf(b); }
      __syncthreads();
    }
  }

  // ---- scheduled faults of this tile ------------------------------------
  const int my_tile = tile_m * p.tiles_n + tile_n;
  int fidx = 0, next_ks = INT_MAX;
  if (p.nfaults > 0) {
    fidx = first_fault(p.faults, p.nfaults, my_tile);
    while (fidx < p.nfaults && p.faults[fidx].tile == my_tile && p.faults[fidx].kstep < ks0) ++fidx;
    if (fidx < p.nfaults && p.faults[fidx].tile == my_tile) next_ks = p.faults[fidx].kstep;
  }

  // ---- global -> register staging -------------------------------------
  constexpr int A_PER = MT * KT / NTHR, B_PER = NT * KT / NTHR;
  constexpr int AV = VEC ? (A_PER >= 4 ? 4 : A_PER) : 1;
  constexpr int BV = VEC ? (B_PER >= 4 ? 4 : B_PER) : 1;
  constexpr int A_LD = A_PER / AV, B_LD = B_PER / BV;
  float ra[A_PER], rb[B_PER], rv = 0.f;
  const int nvb = (M + MT / NV - 1) / (MT / NV);
  const int nwb = (N + NT / NW - 1) / (NT / NW);

  auto gload = [&](int ks) {
    const int k0 = ks * KT;
#pragma unroll
    for (int l = 0; l < A_LD; ++l) {
      const int e = (tid + l * NTHR) * AV;
      const int r = e / KT, k = e % KT;
      const int gr = row0 + r, gk = k0 + k;
      if (gr < M && gk < K) {
        if constexpr (VEC) ldg_vec<AV>(&ra[l * AV], p.A + (long long)gr * p.lda + gk);
        else ra[l] = __ldg(p.A + (long long)gr * p.lda + gk);
      } else {
#pragma unroll
        for (int q = 0; q < AV; ++q) ra[l * AV + q] = 0.f;
      }
    }
#pragma unroll
    for (int l = 0; l < B_LD; ++l) {
      const int e = (tid + l * NTHR) * BV;
      const int k = e / NT, n = e % NT;
      const int gk = k0 + k, gn = col0 + n;
      if (gk < K && gn < N) {
        if constexpr (VEC) ldg_vec<BV>(&rb[l * BV], p.B + (long long)gk * p.ldb + gn);
        else rb[l] = __ldg(p.B + (long long)gk * p.ldb + gn);
      } else {
#pragma unroll
        for (int q = 0; q < BV; ++q) rb[l * BV + q] = 0.f;
      }
    }
    if constexpr (LEVEL == L_WARP || LEVEL == L_BLOCK) {
      if (tid < KT * NV) {
        const int k = tid / NV, u = tid % NV, vb = tile_m * NV + u;
        rv = (k0 + k < K && vb < nvb) ? __ldg(p.V + (long long)vb * K + k0 + k) : 0.f;
      } else if (tid < KT * (NV + NW)) {
        const int t = tid - KT * NV, k = t / NW, u = t % NW, wb = tile_n * NW + u;
        rv = (k0 + k < K && wb < nwb) ? __ldg(p.Wt + (long long)wb * K + k0 + k) : 0.f;
      }
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int l = 0; l < A_LD; ++l) {
      const int e = (tid + l * NTHR) * AV;
      const int r = e / KT, k = e % KT;
#pragma unroll
      for (int q = 0; q < AV; ++q) S.As[buf][k + q][r] = ra[l * AV + q];
    }
#pragma unroll
    for (int l = 0; l < B_LD; ++l) {
      const int e = (tid + l * NTHR) * BV;
      const int k = e / NT, n = e % NT;
      sts_vec<BV>(&S.Bs[buf][k][n], &rb[l * BV]);
    }
    if constexpr (LEVEL == L_WARP || LEVEL == L_BLOCK) {
      if (tid < KT * NV) S.vs[buf][tid / NV][tid % NV] = rv;
      else if (tid < KT * (NV + NW)) {
        const int t = tid - KT * NV;
        S.ws[buf][t / NW][t % NW] = rv;
      }
    }
  };

  if (ks0 < ks1) {
    gload(ks0);
    sstore(0);
  }
  __syncthreads();

  int cur = 0;
  for (int ks = ks0; ks < ks1; ++ks) {
    const bool more = ks + 1 < ks1;
    if (more) gload(ks + 1);

    // ---- rank-KT update of the fragment (and thread-level checksums) ----
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      float a[TM], b[TN];
#pragma unroll
      for (int c = 0; c < T::CM; ++c) lds_vec<VM>(&a[c * VM], &S.As[cur][k][arow + c * LM * VM]);
#pragma unroll
      for (int c = 0; c < T::CN; ++c) lds_vec<VN>(&b[c * VN], &S.Bs[cur][k][bcol + c * LN * VN]);
      if constexpr (LEVEL == L_THREAD) {
        float as = 0.f, bs = 0.f;
#pragma unroll
        for (int i = 0; i < TM; ++i) as += a[i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bs += b[j];
#pragma unroll
        for (int i = 0; i < TM; ++i) cr[i] = fmaf(a[i], bs, cr[i]);
#pragma unroll
        for (int j = 0; j < TN; ++j) cc[j] = fmaf(as, b[j], cc[j]);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }

    // ---- warp / block checksum update from the staged slice (Eq. 4) -----
    if constexpr (LEVEL == L_WARP) {
#pragma unroll
      for (int x = 0; x < RPL; ++x) {
        const int i = tn + x * LN;
        if (i < TM) {
          const int r = FROW(i);
          float s = wr[x];
#pragma unroll
          for (int k = 0; k < KT; ++k) s = fmaf(S.As[cur][k][r], S.ws[cur][k][wn], s);
          wr[x] = s;
        }
      }
#pragma unroll
      for (int y = 0; y < CPL; ++y) {
        const int j = tm + y * LM;
        if (j < TN) {
          const int c = FCOL(j);
          float s = wc[y];
#pragma unroll
          for (int k = 0; k < KT; ++k) s = fmaf(S.vs[cur][k][wm], S.Bs[cur][k][c], s);
          wc[y] = s;
        }
      }
    } else if constexpr (LEVEL == L_BLOCK) {
#pragma unroll
      for (int q = 0; q < ENT; ++q) {
        const int e = tid + q * NTHR;
        if (e < NT) {
          float s = bc[q];
#pragma unroll
          for (int k = 0; k < KT; ++k) s = fmaf(S.vs[cur][k][0], S.Bs[cur][k][e], s);
          bc[q] = s;
        } else if (e < NT + MT) {
          float s = bc[q];
#pragma unroll
          for (int k = 0; k < KT; ++k) s = fmaf(S.As[cur][k][e - NT], S.ws[cur][k][0], s);
          bc[q] = s;
        }
      }
    }

    if (more) sstore(cur ^ 1);
    __syncthreads();

    // ---- fault injection after this k-step (Section 5.3) ----------------
    if (ks == next_ks) {
      while (fidx < p.nfaults && p.faults[fidx].tile == my_tile && p.faults[fidx].kstep == ks) {
        const Fault f = p.faults[fidx++];
        if (f.target == T_ACC) {
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
              if (FROW(i) == f.row && FCOL(j) == f.col) acc[i][j] += f.delta;
        } else if constexpr (LEVEL == L_THREAD) {
          bool mine_r = false, mine_c = false;
#pragma unroll
          for (int i = 0; i < TM; ++i) mine_r |= FROW(i) == f.row;
#pragma unroll
          for (int j = 0; j < TN; ++j) mine_c |= FCOL(j) == f.col;
          if (mine_r && mine_c) {
            if (f.target == T_ROWSUM) {
#pragma unroll
              for (int i = 0; i < TM; ++i) if (FROW(i) == f.row) cr[i] += f.delta;
            } else {
#pragma unroll
              for (int j = 0; j < TN; ++j) if (FCOL(j) == f.col) cc[j] += f.delta;
            }
          }
        } else if constexpr (LEVEL == L_WARP) {
          const bool my_warp = f.row / T::WM == wm && f.col / T::WN == wn;
          if (my_warp && f.target == T_ROWSUM) {
#pragma unroll
            for (int x = 0; x < RPL; ++x)
              if (tn + x * LN < TM && FROW(tn + x * LN) == f.row) wr[x] += f.delta;
          } else if (my_warp) {
#pragma unroll
            for (int y = 0; y < CPL; ++y)
              if (tm + y * LM < TN && FCOL(tm + y * LM) == f.col) wc[y] += f.delta;
          }
        } else if constexpr (LEVEL == L_BLOCK) {
          const int e = f.target == T_ROWSUM ? NT + f.row : f.col;
#pragma unroll
          for (int q = 0; q < ENT; ++q)
            if (tid + q * NTHR == e) bc[q] += f.delta;
        }
      }
      next_ks = (fidx < p.nfaults && p.faults[fidx].tile == my_tile) ? p.faults[fidx].kstep : INT_MAX;
    }

    // ---- verification at the end of a period ----------------------------
    // Fast path: fp32 sums of the unit's rows and columns against the
    // checksums; a residual above tau flags its row / column.  Rare path
    // (something flagged): the flagged row and column sums are recomputed
    // exactly in fp64 from the accumulators, so a large fault's rounding in
    // the fp32 sums cannot spoil the located value or the consistency test.
    if constexpr (LEVEL != L_OFF) {
      if (((ks - ks0 + 1) % p.cadence) == 0 || ks == ks1 - 1) {
        if constexpr (LEVEL == L_THREAD) {
          int nr = 0, nc = 0, ir = -1, jc = -1;
          float br = -1.f, bcs = -1.f, tR = 0.f, tC = 0.f;
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < TN; ++j) s += acc[i][j];
            const float d = s - cr[i];
            const float tau = p.lam_u * S.nA[FROW(i)] * froBt;
            if (fabsf(d) > tau) {
              ++nr;
              const float sc = flag_score(d, tau);
              if (sc > br) { br = sc; ir = i; tR = tau; }
            }
          }
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < TM; ++i) s += acc[i][j];
            const float d = s - cc[j];
            const float tau = p.lam_u * froAt * S.nB[FCOL(j)];
            if (fabsf(d) > tau) {
              ++nc;
              const float sc = flag_score(d, tau);
              if (sc > bcs) { bcs = sc; jc = j; tC = tau; }
            }
          }
          if (nr | nc) {
            double SR = 0.0, SC = 0.0, dR = 0.0, dC = 0.0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
              if (i == ir) {
#pragma unroll
                for (int j = 0; j < TN; ++j) SR += (double)acc[i][j];
                dR = SR - (double)cr[i];
              }
#pragma unroll
            for (int j = 0; j < TN; ++j)
              if (j == jc) {
#pragma unroll
                for (int i = 0; i < TM; ++i) SC += (double)acc[i][j];
                dC = SC - (double)cc[j];
              }
            ftgemm_fault_record rec;
            rec.tile_m = tile_m; rec.tile_n = tile_n; rec.kstep = ks;
            rec.row = ir >= 0 ? row0 + FROW(ir) : -1;
            rec.col = jc >= 0 ? col0 + FCOL(jc) : -1;
            rec.residual_r = dR; rec.residual_c = dC; rec.tau = (double)tR + (double)tC;
            rec.delta = 0.0;
            if (nr == 1 && nc == 1) {
              if (fabs(dR - dC) <= (double)tR + (double)tC) {
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                  for (int j = 0; j < TN; ++j)
                    if (i == ir && j == jc) acc[i][j] = (float)((double)acc[i][j] - dR);
                rec.kind = K_CORRECTED; rec.delta = dR;
              } else {
                rec.kind = K_UNCORRECTABLE;
              }
            } else if (nr == 1 && nc == 0) {
#pragma unroll
              for (int i = 0; i < TM; ++i) if (i == ir) cr[i] = (float)SR;
              rec.kind = K_CHECKSUM; rec.delta = -dR;
            } else if (nr == 0 && nc == 1) {
#pragma unroll
              for (int j = 0; j < TN; ++j) if (j == jc) cc[j] = (float)SC;
              rec.kind = K_CHECKSUM; rec.delta = -dC;
            } else {
              rec.kind = K_UNCORRECTABLE;
            }
            report_event(p.rep, p.recs, rec);
          }
        } else {
          // fragment partial sums, then all-reduce inside the warp
          float pr[TM], pc[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < TN; ++j) s += acc[i][j];
            pr[i] = s;
          }
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < TM; ++i) s += acc[i][j];
            pc[j] = s;
          }
#pragma unroll
          for (int o = 1; o < LN; o <<= 1)
#pragma unroll
            for (int i = 0; i < TM; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], o);
#pragma unroll
          for (int o = LN; o < 32; o <<= 1)
#pragma unroll
            for (int j = 0; j < TN; ++j) pc[j] += __shfl_xor_sync(0xffffffffu, pc[j], o);

          if constexpr (LEVEL == L_WARP) {
            // lane (tm, tn) owns row values i = tn + x*LN and column values j = tm + y*LM
            int fr = 0, fc = 0;
            unsigned long long kr = 0ull, kc = 0ull;
#pragma unroll
            for (int x = 0; x < RPL; ++x) {
              const int i = tn + x * LN;
              float s = 0.f;
#pragma unroll
              for (int ii = 0; ii < TM; ++ii) if (ii == i) s = pr[ii];
              const float d = s - wr[x];
              const float tau = (i < TM) ? p.lam_u * S.nA[FROW(i)] * S.froBw[wn] : 0.f;
              if (i < TM && fabsf(d) > tau) {
                ++fr;
                const unsigned long long key = flag_key(flag_score(d, tau), FROW(i));
                kr = key > kr ? key : kr;
              }
            }
#pragma unroll
            for (int y = 0; y < CPL; ++y) {
              const int j = tm + y * LM;
              float s = 0.f;
#pragma unroll
              for (int jj = 0; jj < TN; ++jj) if (jj == j) s = pc[jj];
              const float d = s - wc[y];
              const float tau = (j < TN) ? p.lam_u * S.froAw[wm] * S.nB[FCOL(j)] : 0.f;
              if (j < TN && fabsf(d) > tau) {
                ++fc;
                const unsigned long long key = flag_key(flag_score(d, tau), FCOL(j));
                kc = key > kc ? key : kc;
              }
            }
            const int nr = __reduce_add_sync(0xffffffffu, fr);
            const int nc = __reduce_add_sync(0xffffffffu, fc);
            if (nr | nc) {
              kr = warp_max_u64(kr);
              kc = warp_max_u64(kc);
              const int ir = nr ? key_index(kr) : -1;  // tile-local row
              const int jc = nc ? key_index(kc) : -1;  // tile-local column
              // exact fp64 sums of the flagged row and column over the warp tile
              double SR = 0.0, SC = 0.0, cR = 0.0, cC = 0.0;
              float tR = 0.f, tC = 0.f;
#pragma unroll
              for (int i = 0; i < TM; ++i)
                if (FROW(i) == ir) {
#pragma unroll
                  for (int j = 0; j < TN; ++j) SR += (double)acc[i][j];
                }
#pragma unroll
              for (int j = 0; j < TN; ++j)
                if (FCOL(j) == jc) {
#pragma unroll
                  for (int i = 0; i < TM; ++i) SC += (double)acc[i][j];
                }
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                SR += __shfl_xor_sync(0xffffffffu, SR, o);
                SC += __shfl_xor_sync(0xffffffffu, SC, o);
              }
              bool own_r = false, own_c = false;
#pragma unroll
              for (int x = 0; x < RPL; ++x)
                if (tn + x * LN < TM && FROW(tn + x * LN) == ir) {
                  own_r = true; cR = wr[x]; tR = p.lam_u * S.nA[ir] * S.froBw[wn];
                }
#pragma unroll
              for (int y = 0; y < CPL; ++y)
                if (tm + y * LM < TN && FCOL(tm + y * LM) == jc) {
                  own_c = true; cC = wc[y]; tC = p.lam_u * S.froAw[wm] * S.nB[jc];
                }
              const unsigned mr = __ballot_sync(0xffffffffu, own_r);
              const unsigned mc = __ballot_sync(0xffffffffu, own_c);
              const int lr = mr ? __ffs(mr) - 1 : 0, lc = mc ? __ffs(mc) - 1 : 0;
              cR = __shfl_sync(0xffffffffu, cR, lr);
              tR = __shfl_sync(0xffffffffu, tR, lr);
              cC = __shfl_sync(0xffffffffu, cC, lc);
              tC = __shfl_sync(0xffffffffu, tC, lc);
              const double dR = nr ? SR - cR : 0.0, dC = nc ? SC - cC : 0.0;
              int kind;
              double delta = 0.0;
              if (nr == 1 && nc == 1) {
                if (fabs(dR - dC) <= (double)tR + (double)tC) {
                  kind = K_CORRECTED; delta = dR;
#pragma unroll
                  for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j)
                      if (FROW(i) == ir && FCOL(j) == jc) acc[i][j] = (float)((double)acc[i][j] - dR);
                } else {
                  kind = K_UNCORRECTABLE;
                }
              } else if (nr == 1 && nc == 0) {
                kind = K_CHECKSUM;
                delta = -dR;  // the checksum's offset
#pragma unroll
                for (int x = 0; x < RPL; ++x)
                  if (tn + x * LN < TM && FROW(tn + x * LN) == ir) wr[x] = (float)SR;
              } else if (nr == 0 && nc == 1) {
                kind = K_CHECKSUM;
                delta = -dC;
#pragma unroll
                for (int y = 0; y < CPL; ++y)
                  if (tm + y * LM < TN && FCOL(tm + y * LM) == jc) wc[y] = (float)SC;
              } else {
                kind = K_UNCORRECTABLE;
              }
              if (lane == 0) {
                ftgemm_fault_record rec;
                rec.tile_m = tile_m; rec.tile_n = tile_n; rec.kstep = ks;
                rec.row = ir >= 0 ? row0 + ir : -1;
                rec.col = jc >= 0 ? col0 + jc : -1;
                rec.kind = kind; rec.delta = delta;
                rec.residual_r = dR; rec.residual_c = dC;
                rec.tau = (nr ? (double)tR : 0.0) + (nc ? (double)tC : 0.0);
                report_event(p.rep, p.recs, rec);
              }
            }
          } else {  // L_BLOCK
#pragma unroll
            for (int i = 0; i < TM; ++i)
              if ((i % LN) == tn) S.rowpart[wn][FROW(i)] = pr[i];
#pragma unroll
            for (int j = 0; j < TN; ++j)
              if ((j % LM) == tm) S.colpart[wm][FCOL(j)] = pc[j];
            __syncthreads();
            int myflag = 0;
            float dq[ENT], tq[ENT];
#pragma unroll
            for (int q = 0; q < ENT; ++q) {
              const int e = tid + q * NTHR;
              double s = 0.0;
              float tau = 0.f;
              if (e < NT) {
#pragma unroll
                for (int w = 0; w < T::WGM; ++w) s += (double)S.colpart[w][e];
                tau = p.lam_u * S.froAw[0] * S.nB[e];
              } else if (e < NT + MT) {
#pragma unroll
                for (int w = 0; w < T::WGN; ++w) s += (double)S.rowpart[w][e - NT];
                tau = p.lam_u * S.nA[e - NT] * S.froBw[0];
              }
              dq[q] = (float)(s - (double)bc[q]);
              tq[q] = tau;
              if (e < NT + MT && fabsf(dq[q]) > tau) myflag = 1;
            }
            if (__syncthreads_or(myflag)) {
              if (tid == 0) {
                S.nr = 0; S.nc = 0; S.bestr = 0ull; S.bestc = 0ull;
                S.fix_row = -1; S.reset_entry = -1; S.sum_r = 0.0; S.sum_c = 0.0;
              }
              __syncthreads();
#pragma unroll
              for (int q = 0; q < ENT; ++q) {
                const int e = tid + q * NTHR;
                if (e < NT + MT && fabsf(dq[q]) > tq[q]) {
                  const float sc = flag_score(dq[q], tq[q]);
                  S.cval[e] = bc[q];
                  S.tres[e] = tq[q];
                  if (e < NT) { atomicAdd(&S.nc, 1); atomicMax(&S.bestc, flag_key(sc, e)); }
                  else { atomicAdd(&S.nr, 1); atomicMax(&S.bestr, flag_key(sc, e - NT)); }
                }
              }
              __syncthreads();
              const int nr = S.nr, nc = S.nc;
              const int ir = nr ? key_index(S.bestr) : -1;
              const int jc = nc ? key_index(S.bestc) : -1;
              {  // exact fp64 sums of the flagged row and column over the tile
                double sr = 0.0, sc = 0.0;
                bool hr = false, hc = false;
#pragma unroll
                for (int i = 0; i < TM; ++i)
                  if (FROW(i) == ir) {
                    hr = true;
#pragma unroll
                    for (int j = 0; j < TN; ++j) sr += (double)acc[i][j];
                  }
#pragma unroll
                for (int j = 0; j < TN; ++j)
                  if (FCOL(j) == jc) {
                    hc = true;
#pragma unroll
                    for (int i = 0; i < TM; ++i) sc += (double)acc[i][j];
                  }
                if (hr) atomicAdd(&S.sum_r, sr);
                if (hc) atomicAdd(&S.sum_c, sc);
              }
              __syncthreads();
              if (tid == 0) {
                const double dR = nr ? S.sum_r - (double)S.cval[NT + ir] : 0.0;
                const double dC = nc ? S.sum_c - (double)S.cval[jc] : 0.0;
                const float tR = nr ? S.tres[NT + ir] : 0.f, tC = nc ? S.tres[jc] : 0.f;
                ftgemm_fault_record rec;
                rec.tile_m = tile_m; rec.tile_n = tile_n; rec.kstep = ks;
                rec.row = ir >= 0 ? row0 + ir : -1;
                rec.col = jc >= 0 ? col0 + jc : -1;
                rec.residual_r = dR; rec.residual_c = dC;
                rec.tau = (double)tR + (double)tC;
                rec.delta = 0.0;
                if (nr == 1 && nc == 1) {
                  if (fabs(dR - dC) <= (double)tR + (double)tC) {
                    rec.kind = K_CORRECTED; rec.delta = dR;
                    S.fix_row = ir; S.fix_col = jc; S.fix_delta = dR;
                  } else {
                    rec.kind = K_UNCORRECTABLE;
                  }
                } else if (nr == 1 && nc == 0) {
                  rec.kind = K_CHECKSUM; rec.delta = -dR; S.reset_entry = NT + ir;
                  S.reset_value = (float)S.sum_r;
                } else if (nr == 0 && nc == 1) {
                  rec.kind = K_CHECKSUM; rec.delta = -dC; S.reset_entry = jc;
                  S.reset_value = (float)S.sum_c;
                } else {
                  rec.kind = K_UNCORRECTABLE;
                }
                report_event(p.rep, p.recs, rec);
              }
              __syncthreads();
              const int fr = S.fix_row, fcx = S.fix_col, re = S.reset_entry;
              if (fr >= 0) {
                const double fd = S.fix_delta;
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                  for (int j = 0; j < TN; ++j)
                    if (FROW(i) == fr && FCOL(j) == fcx) acc[i][j] = (float)((double)acc[i][j] - fd);
              }
              if (re >= 0) {
                const float rv2 = S.reset_value;
#pragma unroll
                for (int q = 0; q < ENT; ++q)
                  if (tid + q * NTHR == re) bc[q] = rv2;
              }
            }
          }
        }
      }
    }
    cur ^= 1;
  }

  // ---- epilogue: C = alpha * acc + beta * C (unprotected, Section 3.1) ----
  if (p.partial == nullptr) {
    const float alpha = p.alpha, beta = p.beta;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gr = row0 + FROW(i);
      if (gr >= M) continue;
      float* crow = p.C + (long long)gr * p.ldc;
#pragma unroll
      for (int c = 0; c < T::CN; ++c) {
        const int gc = col0 + FCOL(c * VN);
        if (VEC && VN == 4 && gc + 3 < N) {
          float4 o;
          float* op = reinterpret_cast<float*>(&o);
          if (beta != 0.f) {
            const float4 ci = *reinterpret_cast<const float4*>(crow + gc);
            const float* cp = reinterpret_cast<const float*>(&ci);
#pragma unroll
            for (int q = 0; q < 4; ++q) op[q] = fmaf(alpha, acc[i][c * VN + q], beta * cp[q]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) op[q] = alpha * acc[i][c * VN + q];
          }
          *reinterpret_cast<float4*>(crow + gc) = o;
        } else {
#pragma unroll
          for (int q = 0; q < VN; ++q) {
            if (gc + q < N) {
              const float v = alpha * acc[i][c * VN + q];
              crow[gc + q] = beta != 0.f ? fmaf(beta, crow[gc + q], v) : v;
            }
          }
        }
      }
    }
  } else {
    float* part = p.partial + (long long)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gr = row0 + FROW(i);
      if (gr >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gc = col0 + FCOL(j);
        if (gc < N) part[(long long)gr * N + gc] = acc[i][j];
      }
    }
  }
#undef FROW
#undef FCOL
}

template <class T, int LEVEL, bool VEC>
cudaError_t launch_simt(const SimtParams& p, int split, cudaStream_t st) {
  dim3 grid((p.N + T::NT - 1) / T::NT, (p.M + T::MT - 1) / T::MT, split);
  simt_ftgemm_kernel<T, LEVEL, VEC><<<grid, T::NTHR, 0, st>>>(p);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_simt_level(int level, bool vec, const SimtParams& p, int split, cudaStream_t st) {
  switch (level) {
    case L_OFF: return vec ? launch_simt<T, L_OFF, true>(p, split, st) : launch_simt<T, L_OFF, false>(p, split, st);
    case L_THREAD: return vec ? launch_simt<T, L_THREAD, true>(p, split, st) : launch_simt<T, L_THREAD, false>(p, split, st);
    case L_WARP: return vec ? launch_simt<T, L_WARP, true>(p, split, st) : launch_simt<T, L_WARP, false>(p, split, st);
    case L_BLOCK: return vec ? launch_simt<T, L_BLOCK, true>(p, split, st) : launch_simt<T, L_BLOCK, false>(p, split, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ftg
