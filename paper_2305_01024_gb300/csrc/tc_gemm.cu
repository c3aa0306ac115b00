// tc_gemm.cu -- tensor-core (tcgen05 / TMEM) GEMM with the ABFT checksums
// carried through the MMA and verified from TMEM in the epilogue, for bf16
// and fp8 E4M3 operands with fp32 accumulation (sm_103a).
//
// The method is that of Wu, Zhai et al. (ICS'23): A encoded with column
// checksums e^T A (Eq. 1), B with row checksums B e (Eq. 2), their product
// carrying the checksums of C (Eq. 3), a flagged row and column locating a
// corrupted element whose residual is subtracted (Section 4.2.1).  On the
// tensor cores the checksums ride in extra MMAs of the same k-loop (Eq. 4):
//   row checksums     C_r (128 x 16) += A_tile (128 x k) * W (k x 16)
//   column checksums  C_c (256 x 16) += B_tile^T (256 x k) * V (k x 16)
// where the 16 columns of W hold the pieces of w = B_J e and those of V the
// pieces of v = e^T A_I, each piece representable in the operand type, so
// that sum_c scale_c * piece_c reproduces the fp32 checksum vector.  The
// column-checksum MMA swaps roles: the B tile already in shared memory is
// the A operand.  Verification happens once per tile, in the epilogue, from
// TMEM: fp32 sums screen every row and column, fp64 sums confirm.
//
// CTA: warp 0 issues TMA loads, warp 1 allocates TMEM and issues MMAs,
// warps 2..5 read TMEM (each warp the 32 lanes its index allows), verify,
// correct and store.  Tile 128 x 256, k-block = one 128-byte swizzle row
// (64 bf16 or 128 fp8), STAGES-deep ring.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <climits>

#include "internal.cuh"
#include "ptx.cuh"

namespace ftg {

template <int DT>
struct TcCfg {
  static constexpr int BM = 128, BN = 256;
  static constexpr int ELEM = DT == 0 ? 2 : 1;      // bytes per operand element
  static constexpr int BK = 128 / ELEM;             // one 128-byte row per k-block
  static constexpr int UK = 32 / ELEM;              // K per MMA instruction
  static constexpr int STAGES = 4;
  static constexpr int A_BYTES = BM * 128;          // 16 KB
  static constexpr int B_BYTES = BN * 128;          // 32 KB
  static constexpr int CS_BYTES = 16 * 128;         // 2 KB: 16 checksum pieces x k-block
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES + 2 * CS_BYTES;
  static constexpr int THREADS = 192;
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr uint32_t COL_ACC = 0, COL_CR = 256, COL_CC0 = 288, COL_CC1 = 320;
  static constexpr int NPIECE = DT == 0 ? 3 : 5;   // checksum pieces in use
};

// instruction descriptor: fp32 accumulator, K-major A and B, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int dt, int m, int n) {
  return (1u << 4)                                   // D format: f32
         | ((dt == 0 ? 1u : 0u) << 7)                // A format: bf16 (kind::f16) / e4m3
         | ((dt == 0 ? 1u : 0u) << 10)               // B format
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int DT>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (DT == 0) tc_mma_f16(d, a, b, idesc, acc);
  else tc_mma_f8(d, a, b, idesc, acc);
}

struct TcSmemTail {
  uint64_t full[4], empty[4], acc_full;
  uint32_t tmem_base;
  int abort;
  int nr, nc;
  unsigned long long bestr, bestc;
  int fix_row, fix_col, reset_side, reset_idx;
  double fix_delta, reset_value;
  float colpart[4][256];  // per epilogue warp partial column sums
  float crow[128];        // row checksums (reconstructed, fp32 screen)
  float ccol[256];        // column checksums
  float tr[128], tc[256]; // thresholds
  int flag_r[128], flag_c[256];
  double sum_r[128], sum_c[256];  // fp64 confirmation sums (flagged only)
};

template <int DT, bool ABFT>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmV,
                   const TcParams p) {
  using Cfg = TcCfg<DT>;
  constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, UK = Cfg::UK, S = Cfg::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~uintptr_t(1023));
  TcSmemTail& T = *reinterpret_cast<TcSmemTail*>(base + S * Cfg::STAGE_BYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile_m = blockIdx.y, tile_n = blockIdx.x;
  const int row0 = tile_m * BM, col0 = tile_n * BN;
  const int nkb = (p.K + BK - 1) / BK;
  auto sA = [&](int s) { return base + s * Cfg::STAGE_BYTES; };
  auto sB = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };
  auto sW = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES; };
  auto sV = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES + Cfg::CS_BYTES; };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], 1);
    }
    mbar_init(&T.acc_full, 1);
    T.abort = 0;
    T.fix_row = -1;
    T.fix_col = -1;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&T.tmem_base, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = T.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ---------------------------------------------------
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    const uint32_t bytes = Cfg::A_BYTES + Cfg::B_BYTES + (ABFT ? 2 * Cfg::CS_BYTES : 0);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait(&T.empty[s], (uint32_t)((kb / S) - 1) & 1u)) {
        atomicExch(&T.abort, 1);
        break;
      }
      mbar_arrive_expect_tx(&T.full[s], bytes);
      tma_load_2d(sA(s), &tmA, &T.full[s], kb * BK, row0);
      tma_load_2d(sB(s), &tmB, &T.full[s], kb * BK, col0);
      if constexpr (ABFT) {
        tma_load_2d(sW(s), &tmW, &T.full[s], kb * BK, tile_n * 16);
        tma_load_2d(sV(s), &tmV, &T.full[s], kb * BK, tile_m * 16);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer -----------------------------------------------------
    constexpr uint32_t id_main = tc_idesc(DT, BM, BN);
    constexpr uint32_t id_cs = tc_idesc(DT, 128, 16);
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(&T.full[s], (uint32_t)(kb / S) & 1u)) { ok = false; break; }
      tc_fence_after();
      const uint64_t da = smem_desc_sw128(sA(s)), db = smem_desc_sw128(sB(s));
      const uint64_t dw = smem_desc_sw128(sW(s)), dv = smem_desc_sw128(sV(s));
      const uint64_t db_hi = smem_desc_sw128(sB(s) + 128 * 128);  // B rows 128..255
#pragma unroll
      for (int kk = 0; kk < BK / UK; ++kk) {
        const uint32_t acc = (kb | kk) != 0;
        const uint64_t step = (uint64_t)(kk * 32) >> 4;  // 32 bytes per instruction
        tc_mma<DT>(tmem + Cfg::COL_ACC, da + step, db + step, id_main, acc);
        if constexpr (ABFT) {
          tc_mma<DT>(tmem + Cfg::COL_CR, da + step, dw + step, id_cs, acc);
          tc_mma<DT>(tmem + Cfg::COL_CC0, db + step, dv + step, id_cs, acc);
          tc_mma<DT>(tmem + Cfg::COL_CC1, db_hi + step, dv + step, id_cs, acc);
        }
      }
      tc_commit(&T.empty[s]);  // the stage is free once these MMAs completed
    }
    if (!ok) atomicExch(&T.abort, 1);
    tc_commit(&T.acc_full);
  } else if (warp >= 2) {
    // ---- epilogue -------------------------------------------------------
    const int lq = warp & 3;            // TMEM lane quarter this warp may access
    const int r = lq * 32 + lane;       // tile-local row == TMEM lane
    const int gr = row0 + r;
    const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
    bool done = mbar_wait(&T.acc_full, 0);
    if (!done) atomicExch(&T.abort, 1);
    tc_fence_after();
    const float alpha = p.alpha, beta = p.beta;
    const float acc_scale = p.acc_scale;  // fp8: product of the per-tensor scales
    // ----- scheduled faults of this tile (Section 5.3) -----
    // Verification runs once per tile after its last k-step; the accumulation
    // being additive, an offset is applied to the tensor-memory accumulator
    // here, where the k-step it was scheduled for only changes rounding.
    float cr_adj = 0.f, cc_adj0 = 0.f, cc_adj1 = 0.f;
    if (p.nfaults > 0) {
      const int my_tile = tile_m * p.tiles_n + tile_n;
      for (int f = first_fault(p.faults, p.nfaults, my_tile); f < p.nfaults && p.faults[f].tile == my_tile; ++f) {
        const Fault F = p.faults[f];
        if (F.target == T_ACC) {
          if ((F.row >> 5) == lq) {  // warp-uniform: this warp owns the lane
            const uint32_t a = tl + Cfg::COL_ACC + (uint32_t)(F.col & ~15);
            float v[16];
            tmem_ld16(a, v);
            tmem_wait_ld();
            if (lane == (F.row & 31)) {
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (q == (F.col & 15)) v[q] += F.delta;
            }
            tmem_st16(a, v);
            tmem_wait_st();
          }
        } else if (F.target == T_ROWSUM) {
          if (r == F.row) cr_adj += F.delta;
        } else {
          if (r == (F.col & 127)) {
            if (F.col < 128) cc_adj0 += F.delta;
            else cc_adj1 += F.delta;
          }
        }
      }
    }
    if constexpr (ABFT) {
      // ----- fp32 screen -----
      // row checksum of this row: sum_c piece_scale * C_r[r][c]
      float cs[16];
      tmem_ld16(tl + Cfg::COL_CR, cs);
      tmem_wait_ld();
      float crow = 0.f;
#pragma unroll
      for (int c = 0; c < Cfg::NPIECE; ++c) crow += cs[c] * p.wscale[(size_t)tile_n * 16 + c];
      crow += cr_adj;
      T.crow[r] = crow;
      // column checksums: lane quarter lq holds columns lq*32.. of each half
      tmem_ld16(tl + Cfg::COL_CC0, cs);
      tmem_wait_ld();
      float cc0 = 0.f;
#pragma unroll
      for (int c = 0; c < Cfg::NPIECE; ++c) cc0 += cs[c] * p.vscale[(size_t)tile_m * 16 + c];
      tmem_ld16(tl + Cfg::COL_CC1, cs);
      tmem_wait_ld();
      float cc1 = 0.f;
#pragma unroll
      for (int c = 0; c < Cfg::NPIECE; ++c) cc1 += cs[c] * p.vscale[(size_t)tile_m * 16 + c];
      T.ccol[r] = cc0 + cc_adj0;
      T.ccol[128 + r] = cc1 + cc_adj1;
      // row sums (two-term fp32 summation) and partial column sums
      float rs = 0.f, rc = 0.f;
      for (int ch = 0; ch < BN / 16; ++ch) {
        float v[16];
        tmem_ld16(tl + Cfg::COL_ACC + ch * 16, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float y = v[q] - rc;
          const float t = rs + y;
          rc = (t - rs) - y;
          rs = t;
        }
        // warp partial column sums of these 16 columns: a reduce-scatter
        // over the lanes leaves lanes 2q and 2q+1 with column idx(q)
        float w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = v[q];
#pragma unroll
        for (int lev = 16, half = 8; lev >= 2; lev >>= 1, half >>= 1) {
          const bool up = (lane & lev) != 0;
#pragma unroll
          for (int q = 0; q < half; ++q) {
            const float snd = up ? w[q] : w[q + half];
            const float kp = up ? w[q + half] : w[q];
            w[q] = kp + __shfl_xor_sync(0xffffffffu, snd, lev);
          }
        }
        w[0] += __shfl_xor_sync(0xffffffffu, w[0], 1);
        if ((lane & 1) == 0) {
          const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                          ((lane >> 1) & 1);
          T.colpart[lq][ch * 16 + idx] = w[0];
        }
      }
      // thresholds
      const float nAr = (gr < p.M) ? p.nA[gr] : 0.f;
      T.tr[r] = p.lam_u * nAr * p.froB[tile_n];
      for (int c = r; c < BN; c += 128) {
        const int gc = col0 + c;
        T.tc[c] = p.lam_u * p.froA[tile_m] * ((gc < p.N) ? p.nB[gc] : 0.f);
      }
      T.flag_r[r] = fabsf(rs - crow) > T.tr[r];
    }
    // epilogue-only named barrier among the 4 epilogue warps
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if constexpr (ABFT) {
      for (int c = r; c < BN; c += 128) {
        const float s = (T.colpart[0][c] + T.colpart[1][c]) + (T.colpart[2][c] + T.colpart[3][c]);
        T.flag_c[c] = fabsf(s - T.ccol[c]) > T.tc[c];
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      int any = 0;
      for (int c = lane; c < 128; c += 32) any |= T.flag_r[c];
      for (int c = lane; c < 256; c += 32) any |= T.flag_c[c];
      any = __any_sync(0xffffffffu, any);
      if (any) {
        // ----- fp64 confirmation of every screened row / column -----
        if (r == 0) { T.nr = 0; T.nc = 0; T.bestr = 0ull; T.bestc = 0ull; T.fix_row = -1; T.reset_side = -1; }
        for (int c = r; c < BN; c += 128) T.sum_c[c] = 0.0;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        double sr = 0.0;
        for (int ch = 0; ch < BN / 16; ++ch) {
          float v[16];
          tmem_ld16(tl + Cfg::COL_ACC + ch * 16, v);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            sr += (double)v[q];
            if (T.flag_c[ch * 16 + q]) atomicAdd(&T.sum_c[ch * 16 + q], (double)v[q]);
          }
        }
        T.sum_r[r] = sr;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (T.flag_r[r]) {
          const double d = sr - (double)T.crow[r];
          if (fabs(d) > (double)T.tr[r]) {
            atomicAdd(&T.nr, 1);
            atomicMax(&T.bestr, flag_key(flag_score((float)d, T.tr[r]), r));
          }
        }
        for (int c = r; c < BN; c += 128) {
          if (T.flag_c[c]) {
            const double d = T.sum_c[c] - (double)T.ccol[c];
            if (fabs(d) > (double)T.tc[c]) {
              atomicAdd(&T.nc, 1);
              atomicMax(&T.bestc, flag_key(flag_score((float)d, T.tc[c]), c));
            }
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (r == 0 && (T.nr | T.nc)) {
          const int nr = T.nr, nc = T.nc;
          const int ir = nr ? key_index(T.bestr) : -1, jc = nc ? key_index(T.bestc) : -1;
          const double dR = nr ? T.sum_r[ir] - (double)T.crow[ir] : 0.0;
          const double dC = nc ? T.sum_c[jc] - (double)T.ccol[jc] : 0.0;
          const float tR = nr ? T.tr[ir] : 0.f, tC = nc ? T.tc[jc] : 0.f;
          ftgemm_fault_record rec;
          rec.tile_m = tile_m; rec.tile_n = tile_n; rec.kstep = nkb - 1;
          rec.row = ir >= 0 ? row0 + ir : -1;
          rec.col = jc >= 0 ? col0 + jc : -1;
          rec.residual_r = dR; rec.residual_c = dC; rec.tau = (double)tR + (double)tC;
          rec.delta = 0.0;
          if (nr == 1 && nc == 1) {
            if (fabs(dR - dC) <= (double)tR + (double)tC) {
              rec.kind = K_CORRECTED; rec.delta = dR;
              T.fix_row = ir; T.fix_col = jc; T.fix_delta = dR;
            } else {
              rec.kind = K_UNCORRECTABLE;
            }
          } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
            rec.kind = K_CHECKSUM; rec.delta = nr ? -dR : -dC;
          } else {
            rec.kind = K_UNCORRECTABLE;
          }
          report_event(p.rep, p.recs, rec);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    }
    // ----- alpha * acc + beta * C, store -----
    const int fr = ABFT ? T.fix_row : -1;
    const int fc = ABFT ? T.fix_col : -1;
    const double fd = ABFT ? T.fix_delta : 0.0;
    // every lane reads tensor memory (the loads are warp-collective); only
    // rows inside the matrix store
    {
      const bool row_ok = gr < p.M;
      float* crow_ptr = p.C + (long long)(row_ok ? gr : 0) * p.ldc + col0;
      for (int ch = 0; ch < BN / 16; ++ch) {
        float v[16];
        tmem_ld16(tl + Cfg::COL_ACC + ch * 16, v);
        tmem_wait_ld();
        if (!row_ok) continue;
        if (ABFT && r == fr && fc >= ch * 16 && fc < ch * 16 + 16) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (ch * 16 + q == fc) v[q] = (float)((double)v[q] - fd);
        }
        const int c0 = col0 + ch * 16;
        if (p.c_vec && c0 + 15 < p.N) {
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            float4 o;
            if (beta != 0.f) {
              const float4 ci = *reinterpret_cast<const float4*>(crow_ptr + ch * 16 + q);
              o = make_float4(fmaf(beta, ci.x, alpha * acc_scale * v[q]),
                              fmaf(beta, ci.y, alpha * acc_scale * v[q + 1]),
                              fmaf(beta, ci.z, alpha * acc_scale * v[q + 2]),
                              fmaf(beta, ci.w, alpha * acc_scale * v[q + 3]));
            } else {
              o = make_float4(alpha * acc_scale * v[q], alpha * acc_scale * v[q + 1],
                              alpha * acc_scale * v[q + 2], alpha * acc_scale * v[q + 3]);
            }
            *reinterpret_cast<float4*>(crow_ptr + ch * 16 + q) = o;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (c0 + q < p.N) {
              const float o = alpha * acc_scale * v[q];
              crow_ptr[ch * 16 + q] = beta != 0.f ? fmaf(beta, crow_ptr[ch * 16 + q], o) : o;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && T.abort) atomicAdd(&p.rep->timeouts, 1);
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

template <int DT, bool ABFT>
cudaError_t launch_tc_impl(const TcMaps& maps, const TcParams& p, cudaStream_t st) {
  using Cfg = TcCfg<DT>;
  const size_t smem = 1024 + (size_t)Cfg::STAGES * Cfg::STAGE_BYTES + sizeof(TcSmemTail);
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<DT, ABFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.N + Cfg::BN - 1) / Cfg::BN, (p.M + Cfg::BM - 1) / Cfg::BM);
  tc_gemm_kernel<DT, ABFT><<<grid, Cfg::THREADS, smem, st>>>(maps.A, maps.B, maps.W, maps.V, p);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(int dt, bool abft, const TcMaps& maps, const TcParams& p, cudaStream_t st) {
  if (dt == 0) return abft ? launch_tc_impl<0, true>(maps, p, st) : launch_tc_impl<0, false>(maps, p, st);
  return abft ? launch_tc_impl<1, true>(maps, p, st) : launch_tc_impl<1, false>(maps, p, st);
}

size_t tc_smem_bytes(int dt) {
  return dt == 0 ? 1024 + (size_t)TcCfg<0>::STAGES * TcCfg<0>::STAGE_BYTES + sizeof(TcSmemTail)
                 : 1024 + (size_t)TcCfg<1>::STAGES * TcCfg<1>::STAGE_BYTES + sizeof(TcSmemTail);
}

}  // namespace ftg
