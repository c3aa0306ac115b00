// tc_prep.cu -- encoding pass of the tensor-core path and the operand
// quantizer.
//
// Encoding (Eq. 1-2 of Wu, Zhai et al., ICS'23) for a DM x DN data tile of
// C (DM x DN = 125 x 252 for bf16, 123 x 248 for e4m3):
//   v_I[k] = sum_{i in I} A[i][k]   (e^T A per DM-row block of A)
//   w_J[k] = sum_{j in J} B[k][j]   (B e per DN-column block of B)
// accumulated in fp32 from the operand values as stored, then split into
// pieces representable in the operand type so the MMA can carry them:
//   bf16: x = hi + mid + lo, each piece a bf16 (24 significant bits in all);
//   e4m3: x = sum_c q_c / s_c with s_c = s_0 * 16^c, q_c = e4m3(residual * s_c)
//         and s_0 a power of two putting the block's largest |x| near 448.
// Norms of the rows of A and of the columns of B scale the detection
// threshold.  B is also transposed to the K-major layout the MMA reads,
// except a bf16 B without checksums, which the MMA reads in place.
// Each operand is read once: one kernel reads A for its block sums and row
// norms, one reads B for B^T, its block sums and column norms (partial
// norms per k-chunk, finished without atomics so results are reproducible).
//
// Quantizer: bf16 by round-to-nearest-even; e4m3 with a per-tensor scale
// amax / 448 and round-to-nearest-even with saturation (OCP FP8).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "ptx.cuh"

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
// blocks of launch `kind` start at blk_start[kind].  A group passes `bmap`,
// the problem of every block of the launch (built once, at group creation);
// otherwise the problem is found by binary search.
#define TC_BLOCK_OF(KIND)                                                  \
  const int pi = bmap ? bmap[blockIdx.x] : tc_find_block(b, KIND, blockIdx.x); \
  const TcProblem& P = tc_problem(b, pi);                                  \
  if (P.off) return; /* skipped by a device-array rebinding: not read */   \
  const int lb = (int)blockIdx.x - P.blk_start[KIND]

// Eight consecutive elements of row `row` (columns c0..c0+7, zero past
// `ncols`) as floats, and their raw codes; one vector load when aligned.
template <int DT>
__device__ __forceinline__ void ld8(const void* base, long long ld, long long row, int c0, int ncols, bool vec_ok,
                                    float* v, uint16_t* raw) {
  using E = typename std::conditional<DT == 0, uint16_t, uint8_t>::type;
  const E* p = reinterpret_cast<const E*>(base) + row * ld + c0;
  E e[8];
  if (vec_ok && c0 + 8 <= ncols) {
    if constexpr (DT == 0) {
      const uint4 q = *reinterpret_cast<const uint4*>(p);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) { e[2 * i] = (E)(w[i] & 0xFFFF); e[2 * i + 1] = (E)(w[i] >> 16); }
    } else {
      const uint2 q = *reinterpret_cast<const uint2*>(p);
      const uint32_t w[2] = {q.x, q.y};
#pragma unroll
      for (int i = 0; i < 8; ++i) e[i] = (E)((w[i >> 2] >> (8 * (i & 3))) & 0xFF);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) e[i] = c0 + i < ncols ? p[i] : E(0);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    raw[i] = e[i];
    if constexpr (DT == 0) {
      v[i] = __uint_as_float((uint32_t)e[i] << 16);  // bf16 -> fp32 is exact
    } else {
      __nv_fp8_e4m3 q;
      q.__x = (__nv_fp8_storage_t)e[i];
      v[i] = float(q);
    }
  }
}

// Raw codes of eight consecutive elements (one 16-byte load for bf16, one
// 8-byte load for e4m3, in .x/.y); the caller guarantees alignment and
// bounds.  Kept apart from the conversion so that a thread can issue several
// loads before it consumes any.
template <int DT>
__device__ __forceinline__ uint4 ldraw8(const void* base, long long ld, long long row, int c0) {
  if constexpr (DT == 0) {
    return __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const uint16_t*>(base) + row * ld + c0));
  } else {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint8_t*>(base) + row * ld + c0));
    return make_uint4(q.x, q.y, 0u, 0u);
  }
}

// Raw codes of eight consecutive elements at an 8-byte aligned address (two
// 8-byte loads for bf16, one for e4m3, in .x/.y(/.z/.w)), with the columns
// at or past `ncols` read as zero codes, by predicated loads (no branch, so
// a thread's loads stay in flight together); for bf16 each 8-byte half is
// loaded if it lies inside, so the caller guarantees that ncols - c0 is
// >= 8, <= 0 or (bf16) 4.
template <int DT>
__device__ __forceinline__ uint4 ldraw8_a8_upto(const void* base, long long ld, long long row, int c0, int ncols) {
  const uint2 z = make_uint2(0u, 0u);
  if constexpr (DT == 0) {
    const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(base) + row * ld + c0);
    const uint2 a = c0 + 4 <= ncols ? __ldg(p) : z;
    const uint2 c = c0 + 8 <= ncols ? __ldg(p + 1) : z;
    return make_uint4(a.x, a.y, c.x, c.y);
  } else {
    const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const uint8_t*>(base) + row * ld + c0);
    const uint2 q = c0 + 8 <= ncols ? __ldg(p) : z;
    return make_uint4(q.x, q.y, 0u, 0u);
  }
}

template <int DT>
__device__ __forceinline__ void cvt8(const uint4 q, float* v) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if constexpr (DT == 0) {
      v[i] = __uint_as_float(i & 1 ? w[i >> 1] & 0xFFFF0000u : w[i >> 1] << 16);  // exact
    } else {
      __nv_fp8_e4m3 e;
      e.__x = (__nv_fp8_storage_t)((w[i >> 2] >> (8 * (i & 3))) & 0xFF);
      v[i] = float(e);
    }
  }
}

// A: block sums over DM-row blocks (-> Vf), squared row-norm partials over
// 256-wide k-chunks (-> nA_part), and the copy of each block's rows
// TC_AROWS .. DM - 1 into the first rows of its tail in Vt (the MMA reads a
// tile's first TC_AROWS rows from A and the rest from the tail), one pass.
// Block = (row block, chunk); warp w takes rows w, w+8, ..., lane l the 8
// columns 8l..8l+7 of the chunk.
template <int DT>
__global__ void __launch_bounds__(256) tc_encode_a_kernel(const __grid_constant__ TcBatch b, const int* __restrict__ bmap) {
  TC_BLOCK_OF(P_ENC_A);
  constexpr int DM = tc_dm(DT, true);
  __shared__ float part[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkx = (P.K + 255) / 256;
  const int kx = lb % nkx, blk = lb / nkx;
  const int k0 = kx * 256, r0 = blk * DM;
  const int elem = DT == 0 ? 2 : 1;
  const bool vec_ok = ((uintptr_t)P.A % (8 * elem) == 0) && ((P.lda * elem) % (8 * elem) == 0);
  using E = typename std::conditional<DT == 0, uint16_t, uint8_t>::type;
  E* const tail = reinterpret_cast<E*>(P.Vt) + (long long)blk * TC_TAIL * P.ldk;
  float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto take = [&](const float* v, int r) {
    float sq = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      cs[e] += v[e];
      sq = fmaf(v[e], v[e], sq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) P.nA_part[(long long)kx * P.M + r] = sq;
  };
  const int kl = k0 + lane * 8;
  if (vec_ok && !__any_sync(0xffffffffu, kl < P.K && kl + 8 > P.K)) {
    // aligned A, and no lane's 8 columns straddle K (K a multiple of 8):
    // the warp's 15 or 16 rows in two groups of 8, eight raw loads in flight
    // (a row past the block or past M reads the block's last row, then is
    // skipped; a lane past K loads nothing and reads zeros, so the last
    // chunk of a K that is not a multiple of 256 takes this path too); the
    // kernel is bound by these rounds of load latency
    constexpr int RPW = (DM + 7) / 8, GRP = 8;
    static_assert(RPW % GRP == 0, "row groups");
    const bool in_k = kl < P.K;
    for (int g0 = 0; g0 < RPW; g0 += GRP) {
      uint4 q[GRP];
#pragma unroll
      for (int gi = 0; gi < GRP; ++gi)
        q[gi] = in_k ? ldraw8<DT>(P.A, P.lda, min(r0 + min(warp + 8 * (g0 + gi), DM - 1), P.M - 1), kl)
                     : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int gi = 0; gi < GRP; ++gi) {
        const int lr = warp + 8 * (g0 + gi), r = r0 + lr;
        if (lr < DM && r < P.M) {
          float v[8];
          cvt8<DT>(q[gi], v);
          take(v, r);
          // one 16-byte (bf16) / 8-byte (e4m3) store of the codes
          if (lr >= TC_AROWS && in_k) {
            E* dst = tail + (long long)(lr - TC_AROWS) * P.ldk + kl;
            if constexpr (DT == 0) *reinterpret_cast<uint4*>(dst) = q[gi];
            else *reinterpret_cast<uint2*>(dst) = make_uint2(q[gi].x, q[gi].y);
          }
        }
      }
    }
  } else {
    for (int lr = warp; lr < DM; lr += 8) {
      const int r = r0 + lr;
      if (r >= P.M) break;  // warp-uniform
      float v[8];
      uint16_t raw[8];
      ld8<DT>(P.A, P.lda, r, k0 + lane * 8, P.K, vec_ok, v, raw);
      take(v, r);
      if (lr >= TC_AROWS) {
        E* dst = tail + (long long)(lr - TC_AROWS) * P.ldk;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = k0 + lane * 8 + e;
          if (k < P.K) dst[k] = (E)raw[e];
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) part[warp][lane * 8 + e] = cs[e];
  __syncthreads();
  const int t = threadIdx.x;
  if (k0 + t < P.K) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += part[w][t];
    P.Vf[(long long)blk * P.ldk + k0 + t] = s;
  }
}

// B (K x N, N contiguous): B^T (N x ldk, K contiguous) in KC x NBW tiles
// through shared memory, TC_ENC_B_SUB consecutive tiles along K per block;
// KC is one 128-byte k-block of the operand type.  With checksums a block
// covers one DN-column data block of B (NBW = DN) and also writes its block
// sums (-> Wf), the squared column-norm partials (-> nB_part, one per
// TC_ENC_B_SUB * KC rows of K) and the copy of B^T's rows TC_BROWS .. DN - 1
// of the block into the first rows of its tail in Wt.  DN being a multiple
// of 4, every block starts on an 8-byte boundary of B's rows: lane l reads
// columns 8l .. 8l + 7 of a k-row as two 8-byte loads (bf16) or one (e4m3).
constexpr int TC_ENC_B_SUB = 4;

template <int DT, bool ABFT>
__global__ void __launch_bounds__(256) tc_encode_b_kernel(const __grid_constant__ TcBatch b, const int* __restrict__ bmap) {
  TC_BLOCK_OF(P_ENC_B);
  using E = typename std::conditional<DT == 0, uint16_t, uint8_t>::type;
  constexpr int KC = 128 / (int)sizeof(E);
  constexpr int NBW = ABFT ? tc_dn(DT, true) : TC_BN;
  static_assert(NBW % 4 == 0 && NBW > 31 * 8 - 8 && NBW <= 256, "block columns: 8-byte aligned, 31 or 32 lanes");
  constexpr int PITCH = 256 + (DT == 0 ? 10 : 20);  // elements; staggers the banks (a lane may store 8 past NBW)
  __shared__ __align__(16) E tile[KC][PITCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (P.K + KC - 1) / KC, nkg = (nkc + TC_ENC_B_SUB - 1) / TC_ENC_B_SUB;
  const int kg = lb % nkg, nb = lb / nkg;
  const int n0 = nb * NBW;
  const int lim = min(8, NBW - lane * 8);  // this lane's columns inside the block (8, 4 or <= 0)
  const bool in_cols = lim > 0;
  const bool vec_ok = ((uintptr_t)P.B % 8 == 0) && ((P.ldb * (long long)sizeof(E)) % 8 == 0);
  // vector loads, with a lane's columns past N read as zeros, unless some
  // lane's 8 columns straddle N otherwise than at an 8-byte half
  const int c0 = n0 + lane * 8;
  const bool fast = vec_ok && !__any_sync(0xffffffffu, in_cols && c0 < P.N && c0 + 8 > P.N &&
                                                            (DT != 0 || c0 + 4 != P.N));
  float sq[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto take = [&](const float* v, int k) {
    if constexpr (ABFT) {
      float rs = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float x = e < lim ? v[e] : 0.f;  // columns of the next block do not count
        rs += x;
        sq[e] = fmaf(x, x, sq[e]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
      if (lane == 0 && k < P.K) P.Wf[(long long)nb * P.ldk + k] = rs;
    }
  };
  E* Bt = reinterpret_cast<E*>(P.Bt);
  constexpr int EPV = 16 / (int)sizeof(E);  // elements per 16-byte vector
  for (int sub = 0; sub < TC_ENC_B_SUB; ++sub) {
    const int kc = kg * TC_ENC_B_SUB + sub;
    if (kc >= nkc) break;  // block-uniform
    const int k0 = kc * KC;
    if (fast) {
      // columns aligned: the warp's KC/8 k-rows in groups of 8, eight raw
      // loads in flight (rows past K read row K - 1, then count as zeros;
      // columns past N read as zeros, so the last, ragged block of a
      // problem takes this path too)
      constexpr int RPW = KC / 8, GRP = 8;
      static_assert(RPW % GRP == 0, "row groups");
      for (int g0 = 0; g0 < RPW; g0 += GRP) {
        uint4 q[GRP];
#pragma unroll
        for (int gi = 0; gi < GRP; ++gi)
          q[gi] = in_cols ? ldraw8_a8_upto<DT>(P.B, P.ldb, min(k0 + warp + 8 * (g0 + gi), P.K - 1), c0, P.N)
                          : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int gi = 0; gi < GRP; ++gi) {
          const int kk = warp + 8 * (g0 + gi), k = k0 + kk;
          const uint4 w = k < P.K ? q[gi] : make_uint4(0u, 0u, 0u, 0u);
          if (in_cols) {
            // row pitch and column offset are multiples of 4 bytes; a lane
            // past the block's last column writes inside the padded row
            uint32_t* t = reinterpret_cast<uint32_t*>(&tile[kk][lane * 8]);
            t[0] = w.x;
            t[1] = w.y;
            if constexpr (DT == 0) {
              t[2] = w.z;
              t[3] = w.w;
            }
          }
          float v[8];
          cvt8<DT>(w, v);
          take(v, k);
        }
      }
    } else {
      // B's base or row pitch not 8-byte aligned: element loads; columns
      // past the block or past N read as zeros
      const int ncols = min(P.N, n0 + NBW);
      for (int kk = warp; kk < KC; kk += 8) {
        const int k = k0 + kk;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint16_t raw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (k < P.K && in_cols) ld8<DT>(P.B, P.ldb, k, n0 + lane * 8, ncols, false, v, raw);
        if (in_cols) {
#pragma unroll
          for (int e = 0; e < 8; ++e) tile[kk][lane * 8 + e] = (E)raw[e];
        }
        take(v, k);
      }
    }
    __syncthreads();
    // B^T rows n0..n0+NBW-1, k0..k0+KC-1: 8 threads write one 128-byte row
    // segment (the k-range past K is zero, inside the padded row); with
    // checksums the block's rows TC_BROWS.. also go to its tail
    for (int i = threadIdx.x; i < NBW * 8; i += 256) {
      const int nn = i >> 3, vq = i & 7;
      const int n = n0 + nn;
      if (n >= P.N) continue;
      E o[EPV];
#pragma unroll
      for (int e = 0; e < EPV; ++e) o[e] = tile[vq * EPV + e][nn];
      uint4 w;
      if constexpr (DT == 0) {
        w.x = (uint32_t)o[0] | ((uint32_t)o[1] << 16); w.y = (uint32_t)o[2] | ((uint32_t)o[3] << 16);
        w.z = (uint32_t)o[4] | ((uint32_t)o[5] << 16); w.w = (uint32_t)o[6] | ((uint32_t)o[7] << 16);
      } else {
        uint32_t q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          q[j] = (uint32_t)o[4 * j] | ((uint32_t)o[4 * j + 1] << 8) | ((uint32_t)o[4 * j + 2] << 16) |
                 ((uint32_t)o[4 * j + 3] << 24);
        w = make_uint4(q[0], q[1], q[2], q[3]);
      }
      *reinterpret_cast<uint4*>(Bt + (long long)n * P.ldk + k0 + vq * EPV) = w;
      if (ABFT && nn >= TC_BROWS)
        *reinterpret_cast<uint4*>(reinterpret_cast<E*>(P.Wt) + ((long long)nb * TC_TAIL + nn - TC_BROWS) * P.ldk + k0 +
                                  vq * EPV) = w;
    }
    __syncthreads();  // the tile is refilled by the next chunk
  }
  if constexpr (ABFT) {
    // each warp saw 1/8 of the block's k rows: sum the warps' column partials
    __shared__ float sqw[8][256];
#pragma unroll
    for (int e = 0; e < 8; ++e) sqw[warp][lane * 8 + e] = sq[e];
    __syncthreads();
    for (int c = threadIdx.x; c < NBW; c += blockDim.x) {
      const int n = n0 + c;
      if (n < P.N) {
        float q = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) q += sqw[w][c];
        P.nB_part[(long long)kg * P.N + n] = q;
      }
    }
  }
}

// Norms from the partials: nA / nB and the Frobenius norm of each row block
// of A (first tiles_m blocks) and column block of B (next tiles_n); also the
// coherence ||v_I||_2 / (sqrt(|I|) ||A_I||_F) of each block (the same for
// w_J and B_J), a feature of the learned threshold.
template <int DT>
__global__ void __launch_bounds__(256) tc_norms_kernel(const __grid_constant__ TcBatch b, const int* __restrict__ bmap) {
  TC_BLOCK_OF(P_FIN);
  __shared__ float red[8], red2[8];
  __shared__ float sred[8][256];
  constexpr int KC = DT == 0 ? 64 : 128;
  constexpr int DM = tc_dm(DT, true), DN = tc_dn(DT, true);
  static_assert(DM <= 256 && DN <= 256, "one thread per row of a block");
  const bool side_a = lb < P.tiles_m;
  const int blk = side_a ? lb : lb - P.tiles_m;
  const int R = side_a ? P.M : P.N, bs = side_a ? DM : DN;
  const int nparts = side_a ? (P.K + 255) / 256 : (P.K + KC * TC_ENC_B_SUB - 1) / (KC * TC_ENC_B_SUB);
  const float* part = side_a ? P.nA_part : P.nB_part;
  float* nrm = side_a ? P.nA : P.nB;
  const int t = threadIdx.x, r = blk * bs + t, warp = t >> 5, lane = t & 31;
  // warp w sums partials w, w + 8, ... of rows blk*bs + lane + 32 j, all
  // j at once (8 independent loads per partial); then thread t adds the
  // 8 warps' sums of row t in warp order
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
  for (int c = warp; c < nparts; c += 8) {
    const float* pc = part + (long long)c * R;
#pragma unroll
    for (int j = 0; j < 8; ++j)  // rows outside the block read a valid row; their sums are never used
      acc[j] += pc[min(blk * bs + min(lane + 32 * j, bs - 1), R - 1)];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) sred[warp][lane + 32 * j] = acc[j];
  __syncthreads();
  float s = 0.f;
  if (t < bs && r < R) {
#pragma unroll
    for (int w = 0; w < 8; ++w) s += sred[w][t];
    nrm[r] = sqrtf(s);
  }
  // squared norm of the checksum vector of this block over K
  const float* S = (side_a ? P.Vf : P.Wf) + (long long)blk * P.ldk;
  float c = 0.f;
#pragma unroll 8
  for (int k = t; k < P.K; k += blockDim.x) c = fmaf(S[k], S[k], c);
  float f = s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((t & 31) == 0) {
    red[t >> 5] = f;
    red2[t >> 5] = c;
  }
  __syncthreads();
  if (t == 0) {
    float tot = 0.f, cs = 0.f;
    for (int w = 0; w < 8; ++w) {
      tot += red[w];
      cs += red2[w];
    }
    const float fro = sqrtf(tot);
    (side_a ? P.froA : P.froB)[blk] = fro;
    const int cnt = min(bs, R - blk * bs);
    (side_a ? P.coA : P.coB)[blk] = fro > 0.f ? sqrtf(cs) / (sqrtf((float)cnt) * fro) : 0.f;
  }
}

// s0[blk]: power of two with max_k |S[blk][k]| * s0 in (224, 448]  (fp8 only)
__global__ void tc_blockscale_kernel(const __grid_constant__ TcBatch b, const int* __restrict__ bmap) {
  TC_BLOCK_OF(P_SCALE);
  __shared__ float red[32];
  const bool side_a = lb < P.tiles_m;
  const int blk = side_a ? lb : lb - P.tiles_m;
  const float* S = (side_a ? P.Vf : P.Wf) + (long long)blk * P.ldk;
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

// Pieces of S[blk][k] into the block's tail rows in Pc (rows blk*TC_TAIL ..
// + 7) and their multipliers scale[blk*TC_TAIL + p] (piece p; 0 past the
// pieces in use); row blocks of A first, then column blocks of B.  A tail's
// rows 0 .. TC_TAIL - NP - 1 are rows TC_AROWS.. of the block of A (written
// by tc_encode_a), a B tail's rows 0 .. DN - TC_BROWS - 1 the same rows of
// B^T (tc_encode_b); those past M (N) are zeroed here; the NP pieces follow,
// then zeros.
template <int DT>
__global__ void tc_pieces_kernel(const __grid_constant__ TcBatch b, const int* __restrict__ bmap) {
  TC_BLOCK_OF(P_PIECES);
  constexpr int NS = TC_TAIL, KPT = 8;  // k per thread: one 16-byte (bf16) / 8-byte (fp8) store per slot
  constexpr int NP = tc_npiece(DT), DM = tc_dm(DT, true), DN = tc_dn(DT, true);
  const int nkx = (P.K + 256 * KPT - 1) / (256 * KPT);
  const int k0 = (lb % nkx) * 256 * KPT + threadIdx.x * KPT, bi = lb / nkx;
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
  if (k0 >= P.K) return;
  // slot of piece c, and whether slot c is left alone (a data row of A's
  // tail inside the matrix); rows are ldk long (a multiple of 128), so
  // k0 .. k0+7 stay inside the row; values past K are zero (the GEMM's TMA
  // never reads them)
  const int first = side_a ? DM - TC_AROWS : DN - TC_BROWS;  // slot of the first piece
  static_assert(DM - TC_AROWS + NP == NS && DN - TC_BROWS + NP <= NS, "pieces inside the tail");
  const int live_rows = side_a ? max(0, min(first, P.M - (blk * DM + TC_AROWS)))
                               : max(0, min(first, P.N - (blk * DN + TC_BROWS)));
  float x[KPT];
  {
    const float4* src = reinterpret_cast<const float4*>(S + (long long)blk * P.ldk + k0);
    const float4 u = src[0], v = src[1];
    const float t[KPT] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < KPT; ++j) x[j] = k0 + j < P.K ? t[j] : 0.f;
  }
  if constexpr (DT == 0) {
    uint16_t q[3][KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(x[j]);
      const float r1 = x[j] - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
      q[0][j] = __bfloat16_as_ushort(hi);
      q[1][j] = __bfloat16_as_ushort(mid);
      q[2][j] = __bfloat16_as_ushort(lo);
    }
    uint16_t* out = reinterpret_cast<uint16_t*>(Pc);
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      if (c < live_rows) continue;
      const int pc = c - first;  // piece in this slot
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int p = 0; p < NP; ++p)
        if (p == pc)
          w = make_uint4((uint32_t)q[p][0] | ((uint32_t)q[p][1] << 16), (uint32_t)q[p][2] | ((uint32_t)q[p][3] << 16),
                         (uint32_t)q[p][4] | ((uint32_t)q[p][5] << 16), (uint32_t)q[p][6] | ((uint32_t)q[p][7] << 16));
      *reinterpret_cast<uint4*>(out + (long long)(blk * NS + c) * P.ldk + k0) = w;
    }
  } else {
    __nv_fp8_storage_t* out = reinterpret_cast<__nv_fp8_storage_t*>(Pc);
    uint32_t lo4[NS], hi4[NS];
#pragma unroll
    for (int c = 0; c < NS; ++c) { lo4[c] = 0u; hi4[c] = 0u; }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      float sc = s0[blk], r = x[j];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const __nv_fp8_storage_t qv = __nv_cvt_float_to_fp8(r * sc, __NV_SATFINITE, __NV_E4M3);
        __nv_fp8_e4m3 qq;
        qq.__x = qv;
        r -= float(qq) / sc;
        sc *= 16.f;
        if (j < 4) lo4[c] |= (uint32_t)qv << (8 * j);
        else hi4[c] |= (uint32_t)qv << (8 * (j - 4));
      }
    }
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      if (c < live_rows) continue;
      const int pc = c - first;
      uint2 w = make_uint2(0u, 0u);
#pragma unroll
      for (int p = 0; p < NP; ++p)
        if (p == pc) w = make_uint2(lo4[p], hi4[p]);
      *reinterpret_cast<uint2*>(out + (long long)(blk * NS + c) * P.ldk + k0) = w;
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

// Column-norm partials of B per column: one per encode_b block along K.
int tc_nb_parts(int dt, long long K) {
  const long long kr = (dt == 0 ? 64 : 128) * TC_ENC_B_SUB;
  return (int)((K + kr - 1) / kr);
}

// Blocks each batched encode launch gives one problem.
// An MN-major B (checksums off) needs no encode blocks at all.
void tc_prep_blocks(const TcProblem& P, int dt, int out[P_KINDS]) {
  const int nkx = (P.K + 255) / 256, kc = dt == 0 ? 64 : 128;
  out[P_ENC_A] = nkx * P.tiles_m;
  out[P_ENC_B] = P.b_mn ? 0 : ((P.K + kc * TC_ENC_B_SUB - 1) / (kc * TC_ENC_B_SUB)) * P.tiles_n;
  out[P_FIN] = P.tiles_m + P.tiles_n;
  out[P_SCALE] = P.tiles_m + P.tiles_n;
  out[P_PIECES] = ((P.K + 2047) / 2048) * (P.tiles_m + P.tiles_n);  // 8 k per thread
}

// The encode pass of a batch: B^T for every problem that needs it; with checksums also
// the block sums, norms, Frobenius norms and pieces.  total[kind] = blocks
// of each launch over the batch.
// bmap: null, or per launch kind the problem of each of its blocks.
cudaError_t launch_tc_prep(int dt, bool abft, const TcBatch& b, const int total[P_KINDS],
                           const int* const* bmap, int* launches, cudaStream_t st) {
  auto mp = [&](int kind) -> const int* { return bmap ? bmap[kind] : nullptr; };
  if (!abft) {
    if (total[P_ENC_B] == 0) return cudaSuccess;  // every B is read in place
    if (dt == 0) tc_encode_b_kernel<0, false><<<total[P_ENC_B], 256, 0, st>>>(b, mp(P_ENC_B));
    else tc_encode_b_kernel<1, false><<<total[P_ENC_B], 256, 0, st>>>(b, mp(P_ENC_B));
    ++*launches;
    return cudaGetLastError();
  }
  if (dt == 0) {
    tc_encode_b_kernel<0, true><<<total[P_ENC_B], 256, 0, st>>>(b, mp(P_ENC_B));
    tc_encode_a_kernel<0><<<total[P_ENC_A], 256, 0, st>>>(b, mp(P_ENC_A));
    tc_norms_kernel<0><<<total[P_FIN], 256, 0, st>>>(b, mp(P_FIN));
  } else {
    tc_encode_b_kernel<1, true><<<total[P_ENC_B], 256, 0, st>>>(b, mp(P_ENC_B));
    tc_encode_a_kernel<1><<<total[P_ENC_A], 256, 0, st>>>(b, mp(P_ENC_A));
    tc_norms_kernel<1><<<total[P_FIN], 256, 0, st>>>(b, mp(P_FIN));
    tc_blockscale_kernel<<<total[P_SCALE], 256, 0, st>>>(b, mp(P_SCALE));
    ++*launches;
  }
  if (dt == 0) tc_pieces_kernel<0><<<total[P_PIECES], 256, 0, st>>>(b, mp(P_PIECES));
  else tc_pieces_kernel<1><<<total[P_PIECES], 256, 0, st>>>(b, mp(P_PIECES));
  *launches += 4;
  return cudaGetLastError();
}

// Rebinding of a group to a device array of problems (ftgemm_grouped_gemm_dev),
// one thread per problem of the caller's array; pos[q] is the schedule
// position of the caller's problem q.  An entry that meets tc_bind_rule
// replaces the operand pointers and epilogue scalars of its problem and the
// global address of the tensor maps that point at caller memory (A; B when
// the MMA reads it in place); the encode workspace and the other maps are
// the group's own.  An entry that breaks a rule marks its problem skipped
// (until a later rebinding meets the rules) and is counted in the report.
__global__ void tc_bind_kernel(TcProblem* __restrict__ probs, TcProbMaps* __restrict__ maps,
                               const int* __restrict__ pos, const ftgemm_problem* __restrict__ in, int count,
                               int dt, DevReport* rep) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const ftgemm_problem u = in[q];
  const int p = pos[q];
  TcProblem& P = probs[p];
  if (tc_bind_rule(P.M, P.N, P.K, P.lda, P.ldb, P.b_mn, dt, u) != TC_BIND_OK) {
    P.off = 1;
    atomicAdd(&rep->bind_errors, 1);
    return;
  }
  P.A = u.A;
  P.B = u.B;
  P.C = u.C;
  P.ldc = u.ldc;
  P.c_vec = (u.ldc % 4 == 0) && (((uintptr_t)u.C & 15) == 0);
  P.alpha = (float)u.alpha;
  P.beta = (float)u.beta;
  P.acc_scale = dt == 1 ? u.scale_a * u.scale_b : 1.f;
  P.off = 0;
  tensormap_replace_address(&maps[p].A, u.A);
  if (P.b_mn) tensormap_replace_address(&maps[p].B, u.B);
  tensormap_release();
}

cudaError_t launch_tc_bind(TcProblem* probs, TcProbMaps* maps, const int* pos, const ftgemm_problem* in, int count,
                           int dt, DevReport* rep, cudaStream_t st) {
  tc_bind_kernel<<<(count + 127) / 128, 128, 0, st>>>(probs, maps, pos, in, count, dt, rep);
  return cudaGetLastError();
}

// bits[t / 32] |= 1 << (t % 32) for the tile t of every fault (bits zeroed before)
__global__ void fault_bits_kernel(const Fault* __restrict__ f, int n, uint32_t* __restrict__ bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicOr(&bits[f[i].tile >> 5], 1u << (f[i].tile & 31));
}

cudaError_t launch_fault_bits(const Fault* f, int n, uint32_t* bits, size_t words, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, words * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  fault_bits_kernel<<<(n + 255) / 256, 256, 0, st>>>(f, n, bits);
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
