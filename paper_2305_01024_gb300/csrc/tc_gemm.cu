// tc_gemm.cu -- tensor-core (tcgen05 / TMEM) GEMM with the ABFT checksums
// carried through the MMA and verified from TMEM in the epilogue, for bf16
// and fp8 E4M3 operands with fp32 accumulation (sm_103a).
//
// The method is that of Wu, Zhai et al. (ICS'23): A encoded with column
// checksums e^T A (Eq. 1), B with row checksums B e (Eq. 2), their product
// carrying the checksums of C (Eq. 3), a flagged row and column locating a
// corrupted element whose residual is subtracted (Section 4.2.1).
//
// On the tensor cores the encoded operands of Eq. 1-3 are formed inside one
// MMA tile: with checksums on, the 128 x 256 MMA tile holds 128 - NP data
// rows of A plus NP rows carrying the pieces of v = e^T A_I, and DN data
// columns of B plus NP columns carrying the pieces of w = B_J e (NP = 3 for
// bf16, 5 for e4m3; DN = 256 - NP rounded down to a multiple of 4, so that
// C's rows take 16-byte stores: 252 and 248).  Each piece is representable
// in the operand type and sum_c scale_c * piece_c rebuilds the fp32 checksum
// vector.  The one MMA of each k-slice then accumulates C_IJ, its row
// checksums A_I w (TMEM columns DN ..) and its column checksums v B_J (TMEM
// lanes 128 - NP ..) -- Eq. 3, k-step by k-step as in Eq. 4 -- with no extra
// MMA instruction and no extra shared-memory operand traffic; the cost is
// the 1 - (125 * 252) / (128 * 256) = 3.9% (bf16; 6.9% for e4m3's 123 x
// 248) of the tile that carries checksums instead of data.  Each operand tile is
// loaded as a main box of 120 rows of A (248 of B^T) and an 8-row tail box
// that the encode pass fills with the tile's remaining data rows and its
// pieces, so every box starts on a 1024-byte swizzle group.  Verification
// runs once per tile, after its last k-step, from TMEM: fp32 sums screen
// every row and column, fp64 sums confirm the flagged ones.
//
// The kernel is persistent: one CTA per SM walks a static list of output
// tiles over a table of problems (one problem for ftgemm_gemm, many for the
// grouped call), tiles of one problem in a grouped raster.  Warp 0 issues
// TMA loads into a STAGES-deep ring, warp 1 allocates TMEM and issues MMAs
// into one of two 256-column accumulators, warps 2..5 read the other
// accumulator (each warp the 32 lanes its index allows), verify, correct and
// store -- so the epilogue of one tile overlaps the main loop of the next.
// k-block = one 128-byte swizzle row (64 bf16 or 128 fp8 elements).
//
// B operand.  Without checksums, for bf16 with a 16-byte aligned B, the MMA
// reads B where it lies, as an MN-major operand: four TMA boxes of 64
// columns x 64 k-rows per stage, each k-row a whole 128-byte line of B (the
// tiles are 256 columns wide), so no encode pass runs at all.  With
// checksums the data tile is 252 (e4m3: 248) columns wide, its boxes would
// start off the 128-byte lines of B, and the kernel reads B^T (written by
// the encode pass) K-major instead, as for e4m3 and unaligned B.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <climits>
#include <cstddef>

#include "internal.cuh"
#include "mlp.cuh"
#include "ptx.cuh"

namespace ftg {

// PAIR: a 2-CTA cluster computes a 256 x 256 MMA tile with one cta_group::2
// MMA (issued by the even CTA): each CTA holds 128 rows of A (its own data
// tile with checksums) and half of B's 256 columns, and its tensor
// memory holds its 128 rows of the accumulator, so the epilogue is the same
// as a single CTA's.  Per SM a k-block then moves 32 KB of operands into
// shared memory instead of 48 KB, and the ring holds 6 stages instead of 4.
constexpr int TC_PAIR_STAGES = 6, TC_MAX_STAGES = 6;

template <int DT, bool ABFT, bool PAIR = false>
struct TcCfg {
  static constexpr int BM = TC_BM, BN = TC_BN;        // MMA tile
  static constexpr int NPIECE = DT == 0 ? 3 : 5;      // checksum pieces in use
  static constexpr int DM = tc_dm(DT, ABFT), DN = tc_dn(DT, ABFT);  // data rows / columns of C per tile
  static constexpr int ELEM = DT == 0 ? 2 : 1;        // bytes per operand element
  static constexpr int BK = 128 / ELEM;               // one 128-byte row per k-block
  static constexpr int UK = 32 / ELEM;                // K per MMA instruction
  static constexpr int STAGES = PAIR ? TC_PAIR_STAGES : 4;
  static constexpr int A_BYTES = BM * 128;                   // 16 KB
  static constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * 128;  // 32 KB, or 16 KB a CTA of a pair
  static constexpr int MMA_M = PAIR ? 2 * BM : BM;            // rows of one MMA
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  // epilogue warps: with checksums two warpgroups (each tile's columns split
  // between them), without one; plus the TMA and MMA warps
  static constexpr int EW = ABFT ? 8 : 4;
  static constexpr int THREADS = 64 + 32 * EW;
  static constexpr int MN_BOX = 64 * 128;  // bytes of one 64-column x 64-row box of an MN-major B
  static constexpr uint32_t TMEM_COLS = 2 * BN;       // two fp32 accumulators
  static_assert(NPIECE == tc_npiece(DT) && NPIECE <= TC_MAX_PIECES, "column-checksum piece rows in shared memory");
  static_assert(!ABFT || (DM == TC_BM - NPIECE && DN + NPIECE <= TC_BN), "pieces inside the MMA tile");
  static_assert(DN % 4 == 0, "tile columns start 16-byte groups of C's rows (float4 stores)");
  // the tail boxes start on a 1024-byte (8-row) swizzle boundary
  static_assert((TC_AROWS * 128) % 1024 == 0 && (TC_BROWS * 128) % 1024 == 0, "tail boxes misaligned");
};

// instruction descriptor: fp32 accumulator, K-major A and B, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int dt, int m, int n) {
  return (1u << 4)                                   // D format: f32
         | ((dt == 0 ? 1u : 0u) << 7)                // A format: bf16 (kind::f16) / e4m3
         | ((dt == 0 ? 1u : 0u) << 10)               // B format
         | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

constexpr uint32_t TC_IDESC_B_MN = 1u << 16;  // instruction descriptor: B is MN-major

// Shared-memory descriptor of an MN-major operand stored as 128-byte swizzled
// boxes of 64 MN elements x 64 k-rows: within a box the 8-row groups along K
// are 1024 bytes apart (stride byte offset), and the 64-element groups along
// MN are whole boxes apart (leading byte offset).
__device__ __forceinline__ uint64_t smem_desc_mn_sw128(const void* tile, uint32_t box_bytes) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;             // start address
  d |= (uint64_t)((box_bytes >> 4) & 0x3FFF) << 16;  // leading byte offset: next 64 MN elements
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8 k-rows
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

template <int DT>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (DT == 0) tc_mma_f16(d, a, b, idesc, acc);
  else tc_mma_f8(d, a, b, idesc, acc);
}

struct TcSmemTail {
  uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem_base;
  int abort;
  int nr, nc;
  unsigned long long bestr, bestc;
  int fix_row[2], fix_col[2];      // per accumulator parity
  double fix_delta[2];
  unsigned int sink_max;           // residual sink: largest residual / (u * norms) of the tile
  alignas(16) float colpart[4][256];  // per TMEM lane quarter partial column sums (data rows); float4 stores
  float ccp[TC_MAX_PIECES][256];   // column-checksum pieces, TMEM lanes 128 - NP ..
  float crow[128];                 // row checksums
  float ccol[256];                 // column checksums
  // thresholds; before the threshold is formed, the same entry holds the
  // injected offset of that row's / column's checksum (read, then
  // overwritten, by the one thread that owns the row / column)
  float tr[128], tc[256];
  float rsp[2][128];               // fp32 row sums of each half of the columns
  uint8_t flag_r[128], flag_c[256];
  double sum_r[128], sum_c[256];   // fp64 confirmation sums
  double sum_rp[128];              // fp64 row sums of the second half of the columns
  // per epilogue warp: its 32 rows x 16 columns of one accumulator chunk,
  // 64-byte rows with the 16-byte column groups XOR-swizzled by (row / 2) % 4
  // (16-byte writes of 8 consecutive rows, and the read-back of 4 column
  // groups of 2 rows, hit distinct banks), read back row-segment-wise so
  // that C is written in 64-byte runs
  alignas(16) float stg[8][32][16];
};

static_assert(offsetof(TcSmemTail, colpart) % 16 == 0 && offsetof(TcSmemTail, stg) % 16 == 0,
              "vector stores into the epilogue's shared arrays");
static_assert(1024 + TcCfg<0, true>::STAGES * TcCfg<0, true>::STAGE_BYTES + sizeof(TcSmemTail) <= 227 * 1024 &&
                  1024 + TcCfg<0, true, true>::STAGES * TcCfg<0, true, true>::STAGE_BYTES + sizeof(TcSmemTail) <=
                      227 * 1024,
              "dynamic shared memory within the 227 KB a CTA may use");

// Named barrier 1 over the N epilogue threads (128 or 256).
template <int N>
__device__ __forceinline__ void epi_bar() {
  static_assert(N == 128 || N == 256, "epilogue thread count");
  if constexpr (N == 128) asm volatile("bar.sync 1, 128;" ::: "memory");
  else asm volatile("bar.sync 1, 256;" ::: "memory");
}

// The tiles one worker (a CTA, or a CTA pair) runs.  With a problem table:
// the worker's slice of the host-built tile list.  With one inline problem:
// every n-th entry (n workers) of a raster of TC_GROUP_M tile rows by all
// tile columns, column-major inside a group.  A pair's tile is two tile rows
// high: its tm counts pairs of tile rows, and CTA r of the pair takes tile
// row 2 tm + r.
struct TcTile {
  int pi, tm, tn, nkb;
};
template <bool PAIR>
__device__ __forceinline__ int tc_worker() {
  return PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
}
template <bool PAIR>
__device__ __forceinline__ int tc_my_count(const TcBatch& b) {
  const int w = tc_worker<PAIR>(), nw = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  if (b.table) return b.cta_start[w + 1] - b.cta_start[w];
  return w < b.total_tiles ? (b.total_tiles - 1 - w) / nw + 1 : 0;
}
template <bool PAIR>
__device__ __forceinline__ int tc_my_first(const TcBatch& b) {
  return b.table ? b.cta_start[tc_worker<PAIR>()] : 0;
}
template <bool PAIR>
__device__ __forceinline__ TcTile tc_my_tile(const TcBatch& b, int my0, int j) {
  TcTile x;
  if (b.table) {
    const int4 e = b.tile_list[my0 + j];
    x.pi = e.x; x.tm = e.y; x.tn = e.z; x.nkb = e.w;
    return x;
  }
  const TcProblem& P = b.one;
  const int nw = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int rows = PAIR ? (P.tiles_m + 1) / 2 : P.tiles_m, gm = PAIR ? TC_GROUP_M / 2 : TC_GROUP_M;
  const int id = tc_worker<PAIR>() + j * nw, per_group = gm * P.tiles_n;
  const int first_m = (id / per_group) * gm;
  const int gsize = min(rows - first_m, gm);
  x.pi = 0;
  x.tm = first_m + (id % per_group) % gsize;
  x.tn = (id % per_group) / gsize;
  x.nkb = P.nkb;
  return x;
}

template <int DT, bool ABFT, bool PAIR>
__global__ void __launch_bounds__(TcCfg<DT, ABFT, PAIR>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcBatch b, const __grid_constant__ TcMapsBatch mb, const TcRun run) {
  using Cfg = TcCfg<DT, ABFT, PAIR>;
  constexpr int BN = Cfg::BN, DM = Cfg::DM, DN = Cfg::DN, BK = Cfg::BK, UK = Cfg::UK;
  constexpr int S = Cfg::STAGES, CSR = TC_TAIL;
  static_assert(S <= TC_MAX_STAGES, "ring depth");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~uintptr_t(1023));
  TcSmemTail& T = *reinterpret_cast<TcSmemTail*>(base + S * Cfg::STAGE_BYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rank = PAIR ? (int)cluster_ctarank() : 0;  // CTA of the pair (0 issues the MMAs)
  const bool leader = rank == 0;
  auto sA = [&](int s) { return base + s * Cfg::STAGE_BYTES; };
  auto sB = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&T.acc_full[a], 1);
      mbar_init(&T.acc_empty[a], PAIR ? 2 * Cfg::EW : Cfg::EW);  // one arrival per epilogue warp (of both CTAs)
    }
    T.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc_pair(&T.tmem_base, Cfg::TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(&T.tmem_base, Cfg::TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  // the leader's barriers are initialised before the other CTA signals them
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = T.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: main boxes of A and B^T, then their tails ----------
    // A CTA of a pair loads its own 128 rows of A and its half of B (columns
    // 128 r .. 128 r + 127 of the MMA tile; the second half ends with the
    // tail of B^T), and completes the bytes on the leader's barrier, which
    // expects both CTAs' bytes.
    uint32_t it = 0;  // k-blocks issued, over all tiles of this CTA
    int last_pi = -1;
    bool dead = false;
    const int n_my = tc_my_count<PAIR>(b), my0 = tc_my_first<PAIR>(b);
    TcTile nx = n_my > 0 ? tc_my_tile<PAIR>(b, my0, 0) : TcTile{0, 0, 0, 0};
    for (int j = 0; j < n_my && !dead; ++j) {
      const TcTile x = nx;
      const TcProbMaps* mp = mb.table ? &mb.table[x.pi] : &mb.one;
      if (x.pi != last_pi) {
        if (mb.table) {
          tensormap_acquire(&mp->A);
          tensormap_acquire(&mp->B);
          if constexpr (PAIR) tensormap_acquire(&mp->B1);
          if constexpr (ABFT) {
            tensormap_acquire(&mp->W);
            tensormap_acquire(&mp->V);
          }
        }
        prefetch_tmap(&mp->A);
        prefetch_tmap(rank ? &mp->B1 : &mp->B);
        last_pi = x.pi;
      }
      const int tm = PAIR ? 2 * x.tm + rank : x.tm;  // this CTA's tile row
      const int row0 = tm * DM, col0 = x.tn * DN;
      const TcProblem& Px = tc_problem(b, x.pi);
      const bool mn = !ABFT && DT == 0 && Px.b_mn;
      const bool off = Px.off;  // skipped: the stages are released unloaded
      for (int kb = 0; kb < x.nkb; ++kb, ++it) {
        const int s = it % S;
        if (it >= S && !mbar_wait(&T.empty[s], ((it / S) & 1u) ^ 1u)) {
          dead = true;
          break;
        }
        if (off) {
          if (leader) mbar_arrive(&T.full[s]);
          if (kb == 0 && j + 1 < n_my) nx = tc_my_tile<PAIR>(b, my0, j + 1);
          continue;
        }
        if constexpr (PAIR) {
          const uint32_t cbar = mapa_rank(&T.full[s], 0);
          if (leader) mbar_arrive_expect_tx(&T.full[s], 2 * Cfg::STAGE_BYTES);
          tma_load_2d_pair(sA(s), &mp->A, cbar, kb * BK, row0);
          if (mn) {
#pragma unroll
            for (int g = 0; g < BN / 128; ++g)
              tma_load_2d_pair(sB(s) + g * Cfg::MN_BOX, &mp->B, cbar, col0 + 128 * rank + 64 * g, kb * BK);
          } else {
            tma_load_2d_pair(sB(s), rank ? &mp->B1 : &mp->B, cbar, kb * BK, col0 + 128 * rank);
          }
          if constexpr (ABFT) {
            tma_load_2d_pair(sA(s) + TC_AROWS * 128, &mp->V, cbar, kb * BK, tm * CSR);
            if (rank) tma_load_2d_pair(sB(s) + (TC_BROWS - 128) * 128, &mp->W, cbar, kb * BK, x.tn * CSR);
          }
        } else {
          // the same byte count either way: an MN-major B is 4 boxes of 8 KB
          mbar_arrive_expect_tx(&T.full[s], Cfg::STAGE_BYTES);
          tma_load_2d(sA(s), &mp->A, &T.full[s], kb * BK, row0);
          if (mn) {
#pragma unroll
            for (int g = 0; g < BN / 64; ++g)
              tma_load_2d(sB(s) + g * Cfg::MN_BOX, &mp->B, &T.full[s], col0 + 64 * g, kb * BK);
          } else {
            tma_load_2d(sB(s), &mp->B, &T.full[s], kb * BK, col0);
          }
          if constexpr (ABFT) {
            tma_load_2d(sA(s) + TC_AROWS * 128, &mp->V, &T.full[s], kb * BK, tm * CSR);
            tma_load_2d(sB(s) + TC_BROWS * 128, &mp->W, &T.full[s], kb * BK, x.tn * CSR);
          }
        }
        // look one tile ahead while this tile's loads are in flight
        if (kb == 0 && j + 1 < n_my) nx = tc_my_tile<PAIR>(b, my0, j + 1);
      }
    }
    if (dead) atomicExch(&T.abort, 1);
    // let the last loads land before the CTA may exit (bounded); in a pair
    // they complete on the leader's barriers, and the cluster barrier at
    // the end keeps both CTAs until the leader's MMAs have read them
    if (leader)
      for (uint32_t q = it > (uint32_t)S ? it - S : 0; q < it; ++q) mbar_wait(&T.full[q % S], (q / S) & 1u);
  } else if (warp == 1 && lane == 0 && leader) {
    // ---- MMA issuer: one 128 x 256 (a pair: 256 x 256) MMA per 32-byte k-slice
    constexpr uint32_t idesc = tc_idesc(DT, Cfg::MMA_M, BN);
    uint32_t it = 0;
    int lt = 0;  // tiles of this CTA so far
    bool dead = false;
    const int n_my = tc_my_count<PAIR>(b), my0 = tc_my_first<PAIR>(b);
    TcTile nx = n_my > 0 ? tc_my_tile<PAIR>(b, my0, 0) : TcTile{0, 0, 0, 0};
    for (; lt < n_my && !dead; ++lt) {
      const int nkb = nx.nkb;
      const bool mn = !ABFT && DT == 0 && tc_problem(b, nx.pi).b_mn;
      const uint32_t id_t = mn ? (idesc | TC_IDESC_B_MN) : idesc;
      const int ab = lt & 1;
      if (lt >= 2 && !mbar_wait(&T.acc_empty[ab], ((lt >> 1) - 1) & 1)) {
        dead = true;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(ab * BN);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % S;
        if (!mbar_wait(&T.full[s], (it / S) & 1u)) {
          dead = true;
          break;
        }
        tc_fence_after();
        const uint64_t da = smem_desc_sw128(sA(s));
        const uint64_t db = mn ? smem_desc_mn_sw128(sB(s), Cfg::MN_BOX) : smem_desc_sw128(sB(s));
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          // K-major: 32 bytes along the swizzled row per instruction;
          // MN-major: UK k-rows of 128 bytes
          const uint64_t step_a = (uint64_t)(kk * 32) >> 4;
          const uint64_t step_b = mn ? (uint64_t)(kk * UK * 128) >> 4 : step_a;
          if constexpr (PAIR) {
            if constexpr (DT == 0) tc_mma_f16_pair(d, da + step_a, db + step_b, id_t, (kb | kk) != 0);
            else tc_mma_f8_pair(d, da + step_a, db + step_b, id_t, (kb | kk) != 0);
          } else {
            tc_mma<DT>(d, da + step_a, db + step_b, id_t, (kb | kk) != 0);
          }
        }
        // the stage (in both CTAs of a pair) is free once these MMAs completed
        if constexpr (PAIR) tc_commit_pair(&T.empty[s], (uint16_t)3);
        else tc_commit(&T.empty[s]);
        if (kb == 0 && lt + 1 < n_my) nx = tc_my_tile<PAIR>(b, my0, lt + 1);
      }
      if constexpr (PAIR) tc_commit_pair(&T.acc_full[ab], (uint16_t)3);
      else tc_commit(&T.acc_full[ab]);
    }
    if (dead) atomicExch(&T.abort, 1);
    // let the last MMAs finish before TMEM may be released (bounded)
    if (lt > 0) mbar_wait(&T.acc_full[(lt - 1) & 1], ((lt - 1) >> 1) & 1);
  } else if (warp >= 2) {
    // ---- epilogue -------------------------------------------------------
    // With checksums two warpgroups share each tile: warp pairs with the
    // same TMEM lane quarter, one per half of the columns (eh).
    constexpr int EPI_T = 32 * Cfg::EW;      // epilogue threads
    constexpr int CH2 = BN / 32 / (Cfg::EW / 4);  // 32-column loads per warp and tile
    const int lq = warp & 3;            // TMEM lane quarter this warp may access
    const int ew = warp - 2;            // epilogue warp index
    const int eh = ew >> 2;             // half of the columns (0 without checksums)
    const int r = lq * 32 + lane;       // tile row == TMEM lane
    const int q = eh * 128 + r;         // this thread's index among the epilogue threads
    const bool data_row = r < DM;
    const int n_my = tc_my_count<PAIR>(b), my0 = tc_my_first<PAIR>(b);
    TcTile nx = n_my > 0 ? tc_my_tile<PAIR>(b, my0, 0) : TcTile{0, 0, 0, 0};
    bool dead = false;
    // hand an accumulator back to the MMA warp (the leader's, in a pair)
    auto acc_release = [&](int ab) {
      if constexpr (PAIR) mbar_arrive_cluster(mapa_rank(&T.acc_empty[ab], 0));
      else mbar_arrive(&T.acc_empty[ab]);
    };
    for (int lt = 0; lt < n_my; ++lt) {
      const TcTile x = nx;
      if (lt + 1 < n_my) nx = tc_my_tile<PAIR>(b, my0, lt + 1);  // consumed next tile
      const TcProblem& P = tc_problem(b, x.pi);
      const int ab = lt & 1;
      const int tm = PAIR ? 2 * x.tm + rank : x.tm;  // this CTA's tile row
      const int row0 = tm * DM, col0 = x.tn * DN, gr = row0 + r;
      const uint32_t tl = tmem + (uint32_t)(ab * BN) + ((uint32_t)(lq * 32) << 16);
      // a problem skipped by a rebinding, or the second tile row of a pair
      // past the problem's last one
      if (P.off || tm >= P.tiles_m) {
        // a problem skipped by a device-array rebinding: its accumulator
        // (from unloaded stages) is handed back without a store or a check
        if (!dead && !mbar_wait(&T.acc_full[ab], (lt >> 1) & 1)) {
          dead = true;
          atomicExch(&T.abort, 1);
        }
        tc_fence_after();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) acc_release(ab);
        continue;
      }
      // Everything this tile needs from global memory, and its threshold,
      // is fetched and computed before waiting for the accumulator, so the
      // load latency hides behind the tile's main loop.
      const int pM = P.M, pN = P.N;
      const float sc = P.alpha * P.acc_scale;  // fp8: product of the per-tensor scales
      const bool unit_sc = sc == 1.f;           // skip the scaling multiplies
      const float beta = P.beta;
      const int c_vec = P.c_vec;
      const long long ldc = P.ldc;
      float* const Cp = P.C;
      const int my_tile = P.tile_start + tm * P.tiles_n + x.tn;
      const bool has_fault =
          run.nfaults > 0 && ((run.fault_bits[my_tile >> 5] >> (my_tile & 31)) & 1u);
      float nA_r = 0.f, froA_t = 0.f, froB_t = 0.f, nB_c[2] = {0.f, 0.f};
      float wsc[Cfg::NPIECE], vsc[Cfg::NPIECE];
      float lam_u = P.lam_u;
      float grow = P.grow;  // the learned threshold replaces both analytic terms
      float feat[MLP_IN];
      if constexpr (ABFT) {
        nA_r = (data_row && gr < pM) ? P.nA[gr] : 0.f;
        froA_t = P.froA[tm];
        froB_t = P.froB[x.tn];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = q + EPI_T * h, gc = col0 + c;  // this thread's columns
          nB_c[h] = (c < DN && gc < pN) ? P.nB[gc] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < Cfg::NPIECE; ++q) {
          wsc[q] = P.wscale[(size_t)x.tn * CSR + q];
          vsc[q] = P.vscale[(size_t)tm * CSR + q];
        }
        // ----- threshold of this tile -----
        // analytic: lambda * u times the norms plus the growth term
        // mu * u * sqrt(K) times |checksum|; learned: lambda =
        // mlp_scale * 2^f(x) times the norms alone, with x the tile's
        // features (log2 K, block coherences, operand type, tile size),
        // evaluated on every epilogue warp; the analytic threshold is the
        // fallback for a non-finite or non-positive output
        const int rows = min(DM, pM - row0), cols = min(DN, pN - col0);
        feat[0] = log2f((float)P.K) * 0.0625f;
        feat[1] = P.coA ? P.coA[tm] : 0.f;
        feat[2] = P.coB ? P.coB[x.tn] : 0.f;
        feat[3] = DT == 0 ? 0.5f : 1.f;
        feat[4] = log2f((float)rows * (float)cols) * 0.0625f;
        if (P.mlp) {
          MlpAct act;
          mlp_forward_warp(P.mlp, feat, lane, act);
          const float lam = P.mlp_scale * exp2f(act.y);
          if (isfinite(lam) && lam > 0.f) {
            lam_u = lam * 5.9604644775390625e-8f;  // * 2^-24
            grow = 0.f;
          }
        }
      }
      // after one wait gave up the remaining tiles are walked without waits
      // (and without stores), so the barriers below still line up
      const bool ok = !dead && mbar_wait(&T.acc_full[ab], (lt >> 1) & 1);
      if (!ok && !dead) {
        dead = true;
        atomicExch(&T.abort, 1);
      }
      tc_fence_after();
      const bool row_ok = ok && data_row && gr < pM;
      float* crow_ptr = Cp + (long long)(row_ok ? gr : 0) * ldc + col0;
      // alpha * acc + beta * C of one 16-column chunk of the warp's 32 rows,
      // rows and columns inside the matrix only.  The chunk goes through the
      // warp's staging tile: lane l then writes 16 bytes of row 8s + l/4
      // (s = 0..3), so each store instruction covers 8 rows x 64 bytes
      // instead of 32 rows x 16 bytes.  All lanes call it.
      // With checksums it also leaves, in T.colpart[lq], the sums of the
      // chunk's 16 columns over the warp's data rows: each lane adds its 4
      // rows of 4 columns, then an xor tree over the 8 lanes of a column
      // group.
      auto store16w = [&](int ch, const float* v) {
        float(*S)[16] = T.stg[ew];
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<float4*>(&S[lane][4 * (g ^ ((lane >> 1) & 3))]) =
              make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
        __syncwarp();
        float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int sgrp = 0; sgrp < 4; ++sgrp) {
          const int rr = 8 * sgrp + (lane >> 2), cq = lane & 3;
          const int tr_ = lq * 32 + rr, gr_ = row0 + tr_;  // tile row, matrix row
          const float4 x = *reinterpret_cast<const float4*>(&S[rr][4 * (cq ^ ((rr >> 1) & 3))]);
          if constexpr (ABFT) {
            if (tr_ < DM) {
              cs.x += x.x; cs.y += x.y; cs.z += x.z; cs.w += x.w;
            }
          }
          const int c = ch * 16 + 4 * cq, gc = col0 + c;
          if (!ok || tr_ >= DM || gr_ >= pM || c >= DN) continue;
          float* dst = Cp + (long long)gr_ * ldc + gc;
          if (c_vec && c + 3 < DN && gc + 3 < pN) {
            float4 o = unit_sc ? x : make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
            if (beta != 0.f) {
              const float4 ci = *reinterpret_cast<const float4*>(dst);
              o.x = fmaf(beta, ci.x, o.x); o.y = fmaf(beta, ci.y, o.y);
              o.z = fmaf(beta, ci.z, o.z); o.w = fmaf(beta, ci.w, o.w);
            }
            *reinterpret_cast<float4*>(dst) = o;
          } else {
            const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (c + e < DN && gc + e < pN) {
                const float o = sc * xs[e];
                dst[e] = beta != 0.f ? fmaf(beta, dst[e], o) : o;
              }
            }
          }
        }
        if constexpr (ABFT) {
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) {
            cs.x += __shfl_xor_sync(0xffffffffu, cs.x, o);
            cs.y += __shfl_xor_sync(0xffffffffu, cs.y, o);
            cs.z += __shfl_xor_sync(0xffffffffu, cs.z, o);
            cs.w += __shfl_xor_sync(0xffffffffu, cs.w, o);
          }
          if (lane < 4) *reinterpret_cast<float4*>(&T.colpart[lq][ch * 16 + 4 * lane]) = cs;
        }
        __syncwarp();  // the tile is refilled by the next chunk
      };

      if constexpr (ABFT) {
        // the checksums' injected offsets start at zero (in tr / tc)
        if (eh == 0) T.tr[r] = 0.f;
        for (int c = q; c < BN; c += EPI_T) T.tc[c] = 0.f;
        if (q == 0) {
          T.fix_row[ab] = -1;
          T.fix_col[ab] = -1;
          T.fix_delta[ab] = 0.0;
          T.sink_max = 0u;
        }
        epi_bar<EPI_T>();
      }
      // ----- scheduled faults of this tile (Section 5.3) -----
      // Verification runs once per tile after its last k-step; the
      // accumulation being additive, an offset is applied to the
      // tensor-memory accumulator here, where the k-step it was scheduled
      // for only changes rounding.
      // one bit per tile keeps the table search off the path of fault-free tiles
      if (has_fault) {
        for (int f = first_fault(run.faults, run.nfaults, my_tile); f < run.nfaults && run.faults[f].tile == my_tile;
             ++f) {
          const Fault F = run.faults[f];
          if (F.target == T_ACC) {
            // warp-uniform: the warp that owns the lane and reads this column
            // later (so its own program order orders the write and the read)
            if ((F.row >> 5) == lq && (F.col * Cfg::EW / 4) / BN == eh) {
              const uint32_t a = tl + (uint32_t)(F.col & ~15);
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
          } else if constexpr (ABFT) {
            if (q == 0) {
              if (F.target == T_ROWSUM) T.tr[F.row] += F.delta;
              else T.tc[F.col] += F.delta;
            }
          }
        }
      }

      if constexpr (!ABFT) {
        // ----- alpha * acc + beta * C, store -----
        // every lane reads tensor memory (the loads are warp-collective);
        // only rows inside the matrix store
        // 32 columns per tensor-memory load: half the load-and-wait round trips
        for (int c2 = 0; c2 < BN / 32; ++c2) {
          float v2[32];
          tmem_ld32(tl + c2 * 32, v2);
          tmem_wait_ld();
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) store16w(2 * c2 + hh, v2 + 16 * hh);
        }
      } else {
        epi_bar<EPI_T>();
        // ----- one pass over the accumulator: fp32 screen sums and the store -----
        // C is written before verification; a confirmed fault is then
        // patched in place (a single element, below).  Each warp covers its
        // lane quarter's rows over its half of the columns.
        float rs = 0.f, rc = 0.f, crow = 0.f;
        // 32 columns per tensor-memory load, processed as two 16-column chunks
        for (int c2 = eh * CH2; c2 < (eh + 1) * CH2; ++c2) {
          float v2[32];
          tmem_ld32(tl + c2 * 32, v2);
          tmem_wait_ld();
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int ch = 2 * c2 + hh;
            const float* v = v2 + 16 * hh;
            // row sum over the data columns: a pairwise tree over the chunk,
            // then a compensated (two-term) add of the chunk's sum; the row
            // checksum pieces sit in columns DN..DN+NPIECE-1 of the last chunk
            constexpr int FULL = DN / 16, REM = DN % 16;
            static_assert(REM + Cfg::NPIECE <= 16, "pieces inside the last chunk");
            float part;
            if (ch < FULL) {
              float t[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) t[e] = v[e];
#pragma unroll
              for (int st = 8; st > 0; st >>= 1)
#pragma unroll
                for (int e = 0; e < st; ++e) t[e] += t[e + st];
              part = t[0];
            } else {
              float t[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) t[e] = e < REM ? v[e] : 0.f;
#pragma unroll
              for (int st = 8; st > 0; st >>= 1)
#pragma unroll
                for (int e = 0; e < st; ++e) t[e] += t[e + st];
              part = t[0];
#pragma unroll
              for (int pc = 0; pc < Cfg::NPIECE; ++pc) crow = fmaf(v[REM + pc], wsc[pc], crow);
            }
            {
              const float y = part - rc;
              const float tt = rs + y;
              rc = (tt - rs) - y;
              rs = tt;
            }
            // the column checksum pieces sit in lanes DM..DM+NPIECE-1
            if (r >= DM && r - DM < Cfg::NPIECE) {
#pragma unroll
              for (int e = 0; e < 16; ++e) T.ccp[r - DM][ch * 16 + e] = v[e];
            }
            store16w(ch, v);  // also the warp's column partial sums of the chunk
          }
        }
        T.rsp[eh][r] = rs;
        if (eh == Cfg::EW / 4 - 1) {  // the half holding the row-checksum pieces
          crow += T.tr[r];            // the injected offset of this row's checksum
          T.crow[r] = crow;
        }
        epi_bar<EPI_T>();
        constexpr float kU = 5.9604644775390625e-8f;  // 2^-24
        int flagged = 0;
        if (eh == 0) {
          // this row: both halves' sums against its checksum
          const float rsum = Cfg::EW == 8 ? T.rsp[0][r] + T.rsp[Cfg::EW / 4 - 1][r] : T.rsp[0][r];
          const float crw = T.crow[r];
          const float trv = (data_row && gr < pM) ? ft_tau(lam_u, nA_r, froB_t, grow, crw) : 0.f;
          T.tr[r] = trv;
          flagged = data_row && fabsf(rsum - crw) > kScreen * trv;
          T.flag_r[r] = (uint8_t)flagged;
          if (run.sink_lam && data_row && gr < pM) {
            const float den = kU * nA_r * froB_t;
            if (den > 0.f) atomicMax(&T.sink_max, __float_as_uint(fabsf(rsum - crw) / den));
          }
        }
        for (int c = q; c < BN; c += EPI_T) {
          const int hc = (c - q) / EPI_T;  // which of this thread's columns (0 or 1)
          int fl = 0;
          float cc = 0.f, tcv = 0.f;
          if (c < DN) {
#pragma unroll
            for (int e = 0; e < Cfg::NPIECE; ++e) cc = fmaf(T.ccp[e][c], vsc[e], cc);
            cc += T.tc[c];  // the injected offset of this column's checksum
            const int gc = col0 + c;
            const float nbc = hc == 0 ? nB_c[0] : nB_c[1];
            tcv = gc < pN ? ft_tau(lam_u, froA_t, nbc, grow, cc) : 0.f;
            const float sc2 = (T.colpart[0][c] + T.colpart[1][c]) + (T.colpart[2][c] + T.colpart[3][c]);
            fl = fabsf(sc2 - cc) > kScreen * tcv;
            if (run.sink_lam && gc < pN) {
              const float den = kU * froA_t * nbc;
              if (den > 0.f) atomicMax(&T.sink_max, __float_as_uint(fabsf(sc2 - cc) / den));
            }
          }
          T.ccol[c] = cc;
          T.tc[c] = tcv;
          T.flag_c[c] = (uint8_t)fl;
          flagged |= fl;
        }
        // barrier + OR over the epilogue warps: the same answer in all
        const int any_flag = bar_red_or(1, EPI_T, flagged);
        if (run.sink_lam && q == 0 && ok) {
          run.sink_lam[my_tile] = __uint_as_float(T.sink_max);
#pragma unroll
          for (int e = 0; e < MLP_IN; ++e) run.sink_x[(long long)my_tile * MLP_IN + e] = feat[e];
        }
        if (any_flag) {
          // ----- fp64 confirmation of every screened row / column -----
          if (q == 0) { T.nr = 0; T.nc = 0; T.bestr = 0ull; T.bestc = 0ull; }
          for (int c = q; c < BN; c += EPI_T) T.sum_c[c] = 0.0;
          epi_bar<EPI_T>();
          // fp64 sums only where the screen flagged, each half of the
          // columns apart: a flagged column (the same in all lanes) by a
          // warp shuffle reduction and one shared-memory add per warp; a
          // flagged row spread over 16 lanes (below).
          // The fp64 work stays inside the branches that need it: this
          // part's fp64 rate is 1/64 of fp32, and a warp instruction costs
          // the same whether one lane or all are active.
          for (int ch = eh * 2 * CH2; ch < (eh + 1) * 2 * CH2; ++ch) {
            float v[16];
            tmem_ld16(tl + ch * 16, v);
            tmem_wait_ld();
            // the flagged columns of this chunk, one at a time (warp-uniform)
            unsigned fcols = 0u;
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (ch * 16 + e < DN && T.flag_c[ch * 16 + e]) fcols |= 1u << e;
            while (fcols) {
              const int e = __ffs(fcols) - 1;
              fcols &= fcols - 1u;
              float ve = 0.f;
#pragma unroll
              for (int e2 = 0; e2 < 16; ++e2)
                if (e2 == e) ve = v[e2];
              double xs = data_row ? (double)ve : 0.0;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
              if (lane == 0) atomicAdd(&T.sum_c[ch * 16 + e], xs);
            }
          }
          // the flagged rows of this warp, one at a time (warp-uniform): the
          // row's lane passes each 16-column chunk through the warp's
          // staging row 0, lane e < 16 adds column e in fp64, and a shuffle
          // tree over the 16 lanes ends the sum (one lane summing alone
          // would issue 16 times the fp64 instructions)
          double sr = 0.0;
          for (unsigned frows = __ballot_sync(0xffffffffu, T.flag_r[r] != 0); frows; frows &= frows - 1u) {
            const int l0 = __ffs(frows) - 1;
            float* srow = T.stg[ew][0];
            double part = 0.0;
            for (int ch = eh * 2 * CH2; ch < (eh + 1) * 2 * CH2; ++ch) {
              float v[16];
              tmem_ld16(tl + ch * 16, v);
              tmem_wait_ld();
              if (lane == l0) {
#pragma unroll
                for (int g = 0; g < 4; ++g)
                  *reinterpret_cast<float4*>(&srow[4 * g]) =
                      make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
              }
              __syncwarp();
              if (lane < 16 && ch * 16 + lane < DN) part += (double)srow[lane];
              __syncwarp();  // the row is rewritten by the next chunk
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const double tot = __shfl_sync(0xffffffffu, part, 0);
            if (lane == l0) sr = tot;
          }
          if (eh == 0) T.sum_r[r] = sr;
          else T.sum_rp[r] = sr;
          epi_bar<EPI_T>();
          if (eh == 0) {
            const double srt = Cfg::EW == 8 ? T.sum_r[r] + T.sum_rp[r] : T.sum_r[r];
            T.sum_r[r] = srt;
            if (T.flag_r[r]) {
              const double dd = srt - (double)T.crow[r];
              if (fabs(dd) > (double)T.tr[r]) {
                atomicAdd(&T.nr, 1);
                atomicMax(&T.bestr, flag_key(flag_score((float)dd, T.tr[r]), r));
              }
            }
          }
          for (int c = q; c < DN; c += EPI_T) {
            if (T.flag_c[c]) {
              const double dd = T.sum_c[c] - (double)T.ccol[c];
              if (fabs(dd) > (double)T.tc[c]) {
                atomicAdd(&T.nc, 1);
                atomicMax(&T.bestc, flag_key(flag_score((float)dd, T.tc[c]), c));
              }
            }
          }
          epi_bar<EPI_T>();
          if (q == 0 && (T.nr | T.nc)) {
            const int nr = T.nr, nc = T.nc;
            const int ir = nr ? key_index(T.bestr) : -1, jc = nc ? key_index(T.bestc) : -1;
            const double dR = nr ? T.sum_r[ir] - (double)T.crow[ir] : 0.0;
            const double dC = nc ? T.sum_c[jc] - (double)T.ccol[jc] : 0.0;
            const float tR = nr ? T.tr[ir] : 0.f, tC = nc ? T.tc[jc] : 0.f;
            ftgemm_fault_record rec;
            rec.tile_m = tm; rec.tile_n = x.tn; rec.kstep = x.nkb - 1;
            rec.problem = P.id; rec.reserved = 0;
            rec.row = ir >= 0 ? row0 + ir : -1;
            rec.col = jc >= 0 ? col0 + jc : -1;
            rec.residual_r = dR; rec.residual_c = dC; rec.tau = (double)tR + (double)tC;
            rec.delta = 0.0;
            if (nr == 1 && nc == 1) {
              if (fabs(dR - dC) <= (double)tR + (double)tC) {
                rec.kind = K_CORRECTED; rec.delta = dR;
                T.fix_row[ab] = ir; T.fix_col[ab] = jc; T.fix_delta[ab] = dR;
              } else {
                rec.kind = K_UNCORRECTABLE;
              }
            } else if ((nr == 1 && nc == 0) || (nr == 0 && nc == 1)) {
              rec.kind = K_CHECKSUM; rec.delta = nr ? -dR : -dC;
            } else {
              rec.kind = K_UNCORRECTABLE;
            }
            report_event(run.rep, run.recs, rec);
          }
          epi_bar<EPI_T>();
          // ----- correct the located element of C (Section 4.2.1) -----
          // The warp owning its TMEM lane and its column (the one that
          // injected there, if anything did) rereads the accumulator: with
          // beta == 0 the value is recomputed from acc - delta; otherwise C
          // already holds alpha * acc + beta * C_in and alpha * delta is
          // taken off it.
          const int fr = T.fix_row[ab];
          if (fr >= 0 && (fr >> 5) == lq && (T.fix_col[ab] * Cfg::EW / 4) / BN == eh) {  // warp-uniform
            const int fc = T.fix_col[ab];
            const double fd = T.fix_delta[ab];
            float v[16];
            tmem_ld16(tl + (uint32_t)(fc & ~15), v);
            tmem_wait_ld();
            if (lane == (fr & 31) && row_ok) {
              float a = 0.f;
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (e == (fc & 15)) a = v[e];
              float* dst = crow_ptr + fc;
              if (beta == 0.f) *dst = sc * (float)((double)a - fd);
              else *dst = (float)((double)*dst - (double)sc * fd);
            }
          }
        }
      }
      // this warp is done with the accumulator: hand it back to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) acc_release(ab);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && T.abort) atomicAdd(&run.rep->timeouts, 1);
  // a pair stays together until both CTAs are done with each other's
  // barriers and tensor memory
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc_pair(tmem, Cfg::TMEM_COLS);
    else tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

template <int DT, bool ABFT, bool PAIR>
cudaError_t launch_tc_impl(const TcBatch& b, const TcMapsBatch& mb, const TcRun& run, int grid, cudaStream_t st) {
  using Cfg = TcCfg<DT, ABFT, PAIR>;
  const size_t smem = 1024 + (size_t)Cfg::STAGES * Cfg::STAGE_BYTES + sizeof(TcSmemTail);
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<DT, ABFT, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (!PAIR) {
    tc_gemm_kernel<DT, ABFT, false><<<grid, Cfg::THREADS, smem, st>>>(b, mb, run);
    return cudaGetLastError();
  } else {
    // clusters of two CTAs (an SM pair each)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(Cfg::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<DT, ABFT, true>, b, mb, run);
  }
}

// Persistent launch over b.total_tiles tiles with `grid` CTAs (<= one per SM;
// pair: an even number, two CTAs per tile of two tile rows).
cudaError_t launch_tc_gemm(int dt, bool abft, bool pair, const TcBatch& b, const TcMapsBatch& mb, const TcRun& run,
                           int grid, cudaStream_t st) {
  if (pair) {
    if (dt == 0)
      return abft ? launch_tc_impl<0, true, true>(b, mb, run, grid, st) : launch_tc_impl<0, false, true>(b, mb, run, grid, st);
    return abft ? launch_tc_impl<1, true, true>(b, mb, run, grid, st) : launch_tc_impl<1, false, true>(b, mb, run, grid, st);
  }
  if (dt == 0)
    return abft ? launch_tc_impl<0, true, false>(b, mb, run, grid, st) : launch_tc_impl<0, false, false>(b, mb, run, grid, st);
  return abft ? launch_tc_impl<1, true, false>(b, mb, run, grid, st) : launch_tc_impl<1, false, false>(b, mb, run, grid, st);
}

}  // namespace ftg
