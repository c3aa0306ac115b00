// internal.cuh -- device-side types shared by the libftgemm translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ftgemm.h"

namespace ftg {

// L_DETECT (internal, the offline scheme's detector): the tile's column
// checksums only, verified once per split, detection without correction.
enum Level { L_OFF = 0, L_THREAD = 1, L_WARP = 2, L_BLOCK = 3, L_TILE = 4, L_DETECT = 6 };
enum Kind { K_CORRECTED = 0, K_UNCORRECTABLE = 1, K_CHECKSUM = 2 };
enum Target { T_ACC = 0, T_ROWSUM = 1, T_COLSUM = 2 };

// One scheduled fault, sorted on the device table by (tile, kstep).
struct Fault {
  int32_t tile;   // tile_m * tiles_n + tile_n
  int32_t kstep;  // global k-step after which it is added
  int32_t row, col, target;
  float delta;
};

// Device report header; records live in a separate array of `capacity`.
struct DevReport {
  unsigned long long detected, corrected, uncorrectable, checksum_only;
  int n_records;
  int capacity;
  int timeouts;     // bounded device waits that gave up
  int bind_errors;  // device-array entries that broke a rebinding rule (problem skipped)
};

static_assert(sizeof(ftgemm_fault_record) == 64, "record layout");

__device__ __forceinline__ void report_event(DevReport* rep, ftgemm_fault_record* recs,
                                             const ftgemm_fault_record& r) {
  atomicAdd(&rep->detected, 1ull);
  if (r.kind == K_CORRECTED) atomicAdd(&rep->corrected, 1ull);
  else if (r.kind == K_UNCORRECTABLE) atomicAdd(&rep->uncorrectable, 1ull);
  else atomicAdd(&rep->checksum_only, 1ull);
  int slot = atomicAdd(&rep->n_records, 1);
  if (slot < rep->capacity) recs[slot] = r;
}

// Ordering key of a flagged residual: larger |d|/tau first, ties to the
// smaller index.  score >= 0, so its float bits order like the value.
__device__ __forceinline__ unsigned long long flag_key(float score, int idx) {
  return ((unsigned long long)__float_as_uint(score) << 32) |
         (unsigned long long)(0xFFFFFFFFu - (unsigned)idx);
}
__device__ __forceinline__ int key_index(unsigned long long key) {
  return (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
}
// Detection threshold of one row or column: lam_u * nx * ny (the norm term)
// plus grow * |c| (the checksum-growth term, grow = mu * u * sqrt(k)).
// Rounded step by step without contraction, so every place that forms it
// gets the same value.
__device__ __forceinline__ float ft_tau(float lam_u, float nx, float ny, float grow, float c) {
  return __fmaf_rn(grow, fabsf(c), __fmul_rn(__fmul_rn(lam_u, nx), ny));
}

// The fp32 screen flags a residual above half the threshold; the fp64
// confirmation then compares with the threshold itself.  The margin keeps
// the screen's own rounding from hiding a residual the fp64 sum would flag.
constexpr float kScreen = 0.5f;

__device__ __forceinline__ float flag_score(float d, float tau) {
  float a = fabsf(d);
  if (tau > 0.f) return a / tau;
  return a > 0.f ? __int_as_float(0x7f800000) : 0.f;
}

// Binary search of the first fault of `tile` in a table sorted by tile.
__device__ __forceinline__ int first_fault(const Fault* f, int n, int tile) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (f[mid].tile < tile) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Parameters of the SIMT fused-ABFT SGEMM (operands arrive through the TMA
// descriptors of SimtMaps: A^T and B k-major, e^T A and B e per k).
struct SimtParams {
  int M, N, K;
  float* C; long long ldc;
  int c_vec;        // C rows are 16-byte aligned (float4 epilogue)
  float alpha, beta;
  const float* nA;  // [M] row 2-norms of A
  const float* nB;  // [N] column 2-norms of B
  float lam_u;      // lambda * u: the norm term of the threshold
  float mu_u;       // mu * u: the checksum-growth term, mu_u * sqrt(k) * |checksum|
  int cadence;      // k-steps per period (>= 1)
  int ksteps;       // ceil(K / k_tb)
  int ks_per_split; // k-steps per split
  float* partial;   // [split][M][N] when split_k > 1, else nullptr
  const Fault* faults; int nfaults;
  DevReport* rep; ftgemm_fault_record* recs;
  int tiles_m, tiles_n;
  int group_m;      // tile rows per raster group
  // learned threshold (block level): lambda of a tile = mlp_scale * 2^f(x)
  // with f the network (device parameters, or null: analytic) and x the
  // tile's features, which need the coherences coA [tiles_m] / coB [tiles_n]
  const float* mlp; float mlp_scale;
  const float* coA; const float* coB;
  // residual sink (block level, optional): per tile the largest |residual|
  // / (u * norm product) over its rows, columns and periods (float bits,
  // combined with atomicMax; zeroed by the host), and its 5 features
  float* sink_lam; float* sink_x;
};

struct SimtMaps {
  CUtensorMap A;  // A^T: dims {M, K}, box {m_tb, k_tb}
  CUtensorMap B;  // B:   dims {N, K}, box {n_tb, k_tb}
  CUtensorMap V;  // e^T A per row block: dims {K, blocks}, box {k_tb, NV}
  CUtensorMap W;  // B e per column block: dims {K, blocks}, box {k_tb, NW}
};

// Tensor-core path geometry: the MMA tile is 128 x 256.  With checksums on,
// the last NP rows of A's tile carry the pieces of e^T A_I and NP columns of
// B's tile those of B_J e (NP = 3 for bf16, 5 for e4m3), leaving a data tile
// of C of 128 - NP rows and 256 - NP columns rounded down to a multiple of 4
// (every tile's first column then starts a 16-byte group of C's rows, which
// the epilogue stores as float4): 125 x 252 for bf16, 123 x 248 for e4m3.
// Each operand tile arrives as a main box (TC_AROWS rows of A, TC_BROWS rows
// of B^T) and an 8-row tail box, one 1024-byte swizzle group, so every box
// lands on a swizzle boundary: a tail holds the tile's remaining data rows of
// A (of B^T), copied there by the encode pass, then the NP pieces (zeros in
// the slots left over).
constexpr int TC_BM = 128, TC_BN = 256, TC_TAIL = 8;
constexpr int TC_MAX_PIECES = 5;  // checksum pieces in use: 3 (bf16) or 5 (e4m3)
constexpr int TC_AROWS = TC_BM - TC_TAIL, TC_BROWS = TC_BN - TC_TAIL;  // 120, 248: main boxes
__host__ __device__ constexpr int tc_npiece(int dt) { return dt == 0 ? 3 : 5; }
// data tile of C: rows, columns (checksums on: 125 x 252 bf16, 123 x 248 e4m3)
__host__ __device__ constexpr int tc_dm(int dt, bool abft) { return abft ? TC_BM - tc_npiece(dt) : TC_BM; }
__host__ __device__ constexpr int tc_dn(int dt, bool abft) { return abft ? (TC_BN - tc_npiece(dt)) & ~3 : TC_BN; }
constexpr int TC_GROUP_M = 16;  // tile rows per raster group

// Batched encode launches of the tensor-core path; a problem's first block
// in launch `kind` is TcProblem::blk_start[kind].
enum TcPrepKind { P_ENC_A = 0, P_ENC_B, P_FIN, P_SCALE, P_PIECES, P_KINDS };

// One GEMM of the tensor-core path: operands, encode buffers, epilogue.
// A table of these drives the encode launches and the persistent GEMM; a
// single GEMM passes one inline (kernel parameter space).
struct TcProblem {
  int M, N, K, id;                // id: index reported in fault records
  int tiles_m, tiles_n, tile_start, nkb;
  int blk_start[P_KINDS];
  const void* A; long long lda;   // M x K, operand type, K contiguous
  const void* B; long long ldb;   // K x N, operand type, N contiguous
  void* Bt; long long ldk;        // B^T (N x ldk); ldk also the row stride of Vt / Wt
  int b_mn;                       // checksums off, bf16, B 16-byte aligned: the MMA reads B
                                  // in place as an MN-major operand (no B^T, no encode pass)
  float* Vf; float* Wf;           // fp32 e^T A [tiles_m][ldk], B e [tiles_n][ldk] (first K used)
  void* Vt; void* Wt;             // tails [tiles * TC_TAIL][ldk], operand type: a tile's last
                                  // data rows of A (of B^T), then its pieces
  float* vscale; float* wscale;   // [tiles * TC_TAIL] multiplier of piece p at p
  float* s0v; float* s0w;         // [tiles] fp8 piece base scales
  float* nA; float* nB;           // [M] row 2-norms of A, [N] column 2-norms of B
  float* nA_part; float* nB_part; // squared-norm partials per k-chunk: [ceil(K/256)][M], [ceil(K/kc)][N]
  float* froA; float* froB;       // [tiles_m], [tiles_n] Frobenius norms of the blocks
  float* coA; float* coB;         // [tiles_m], [tiles_n] coherence of the blocks (threshold features)
  float* C; long long ldc;
  int c_vec;                      // C rows 16-byte aligned (float4 stores)
  float alpha, beta;
  float acc_scale;                // fp8: product of the per-tensor scales; bf16: 1
  float lam_u;                    // analytic threshold: factor lambda * u of the norm term
  float grow;                     // analytic threshold: mu * u * sqrt(K), factor of |checksum|
  const float* mlp;               // learned threshold: network parameters (device), or null
  float mlp_scale;                // lambda of a tile = mlp_scale * 2^network(features)
  int off;                        // 1: skipped (its last device-array rebinding broke a rule):
                                  // nothing of it is read or written
};

// Without checksums a bf16 B is read in place by the MMA (MN-major) when
// TMA can address it: 256-column tiles keep its boxes on 128-byte lines.
__host__ __device__ inline int tc_b_in_place(int dt, bool abft, const void* B, long long ldb) {
  return !abft && dt == 0 && ((uintptr_t)B & 15) == 0 && (ldb * 2) % 16 == 0;
}

// Rules a device-array entry `u` must meet to rebind a group's problem
// (ftgemm_grouped_gemm_dev).  The sizes and the leading dimensions of A and B
// are the ones the group was created with (M..ldb): they fix the tile
// schedule, the encode workspace and the tensor maps' strides.  A, B and C
// are non-null; A is 16-byte aligned (TMA); B is aligned to its element, and
// to 16 bytes when the MMA reads it in place (b_mn); C is 4-byte aligned
// with ldc >= N; e4m3 scales are positive and their product finite.
// Returns TC_BIND_OK or the first rule broken.
enum {
  TC_BIND_OK = 0, TC_BIND_SIZES = 1, TC_BIND_LD = 2, TC_BIND_NULL = 3, TC_BIND_ALIGN_A = 4,
  TC_BIND_ALIGN_B = 5, TC_BIND_C = 6, TC_BIND_SCALE = 7
};
__host__ __device__ inline int tc_bind_rule(long long M, long long N, long long K, long long lda, long long ldb,
                                            int b_mn, int dt, const ftgemm_problem& u) {
  if (u.m != M || u.n != N || u.k != K) return TC_BIND_SIZES;
  if (u.lda != lda || u.ldb != ldb) return TC_BIND_LD;
  if (!u.A || !u.B || !u.C) return TC_BIND_NULL;
  if ((uintptr_t)u.A & 15) return TC_BIND_ALIGN_A;
  if ((dt == 0 && ((uintptr_t)u.B & 1)) || (b_mn && ((uintptr_t)u.B & 15))) return TC_BIND_ALIGN_B;
  if (u.ldc < N || ((uintptr_t)u.C & 3)) return TC_BIND_C;
  if (dt == 1) {
    const float s = u.scale_a * u.scale_b;
    if (!(u.scale_a > 0.f && u.scale_b > 0.f && s > 0.f && s <= 3.4028234663852886e38f)) return TC_BIND_SCALE;
  }
  return TC_BIND_OK;
}

struct TcBatch {
  const TcProblem* table;  // device table of nprob problems, or null: use `one`
  // With a table: CTA c runs tile_list[cta_start[c] .. cta_start[c+1]), each
  // entry {problem, tile_m, tile_n, k-blocks} (a host-built schedule).
  // Without: CTA c runs raster tiles c, c + gridDim.x, ... of `one`.
  const int4* tile_list;
  const int* cta_start;
  int nprob;
  int total_tiles;
  TcProblem one;
};

struct alignas(128) TcProbMaps {
  CUtensorMap A;  // A:   dims {K, M}, box {k-block, 128, or TC_AROWS with checksums}, 128-byte swizzle
  CUtensorMap B;  // B^T: dims {K, N}, box {k-block, 256, or TC_BROWS}; b_mn: B, dims {N, K}, box {64, k-block}
  CUtensorMap W;  // tails of B^T:    dims {K, 8 * tiles_n}, box {k-block, 8}
  CUtensorMap V;  // tails of A:      dims {K, 8 * tiles_m}, box {k-block, 8}
  // CTA pairs (K-major B^T): B holds the first 128 columns of a pair's MMA
  // tile (box {k-block, 128}), B1 the second half's data columns (box
  // {k-block, TC_BROWS - 128} with checksums, whose tail follows from W; else 128)
  CUtensorMap B1;
};

struct TcMapsBatch {
  const TcProbMaps* table;  // device table (128-byte aligned), or null: use `one`
  TcProbMaps one;
};

struct TcRun {
  const Fault* faults; int nfaults;  // sorted by global tile (tile_start + local)
  const uint32_t* fault_bits;        // bit t set when global tile t has a fault (with faults only)
  DevReport* rep; ftgemm_fault_record* recs;
  // residual sink (optional): per global tile, the smallest lambda that
  // would have flagged nothing, and the tile's 5 threshold features
  float* sink_lam; float* sink_x;
};

__device__ __forceinline__ const TcProblem& tc_problem(const TcBatch& b, int pi) {
  return b.table ? b.table[pi] : b.one;
}

// Problem owning block `blk` of a batched launch of `kind`: the last problem
// whose first block is <= blk.
__device__ __forceinline__ int tc_find_block(const TcBatch& b, int kind, int blk) {
  if (!b.table) return 0;
  int lo = 0, hi = b.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.table[mid].blk_start[kind] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace ftg
