/*
 * ftgemm.h -- C ABI of libftgemm: GEMM with online algorithm-based fault
 * tolerance (ABFT) fused into the kernel, for NVIDIA GB300 (sm_103a).
 *
 * Method: Wu, Zhai et al., "Anatomy of High-Performance GEMM with Online Fault
 * Tolerance on GPUs" (ICS'23).  A is encoded with column checksums e^T A
 * (Eq. 1), B with row checksums B e (Eq. 2); their product carries the
 * checksums of C (Eq. 3).  In the outer-product form (Eq. 4) the checksums
 * are updated with every k-step, so each output tile can be verified during
 * the K loop: a residual above the threshold flags a row and a column, whose
 * crossing is the corrupted element, and the residual itself is the amount to
 * subtract (Section 4.2.1).  One fault per verification unit and period is
 * correctable (single-event upset, Section 4.1).
 *
 * Conventions used by every entry point
 *   - All matrices are row-major.  A is M x K (leading dimension lda >= K),
 *     B is K x N (ldb >= N), C is M x N (ldc >= N), in elements.
 *   - Sizes are at least 1 and at most INT32_MAX.  An empty product (M, N
 *     or K equal to 0) is rejected with FTGEMM_ERR_ARG before any work is
 *     enqueued, not run as a no-op; the handle stays usable.
 *   - Matrix pointers are DEVICE pointers owned by the caller.  Host pointers
 *     (schedules, injection arrays, reports) are read or written during the
 *     call only.
 *   - Work is enqueued on the handle's stream.  Only calls that return a
 *     report (or fetch one) synchronise that stream.
 *   - Return value: FTGEMM_OK (0) or a negative FTGEMM_ERR_* code; the text of
 *     the last error of the calling thread is given by ftgemm_last_error().
 *   - The handle owns its device workspaces (checksum vectors, norms, split-K
 *     partials, injection table, report ring); they grow on demand and are
 *     released by ftgemm_destroy().
 */
#ifndef FTGEMM_H
#define FTGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FTGEMM_OK 0
#define FTGEMM_ERR_ARG (-1)         /* null pointer, bad size or leading dim */
#define FTGEMM_ERR_UNSUPPORTED (-2) /* dtype / level / schedule combination  */
#define FTGEMM_ERR_ALIGN (-3)       /* pointer or stride alignment for TMA   */
#define FTGEMM_ERR_CUDA (-4)        /* a CUDA runtime call failed            */
#define FTGEMM_ERR_TIMEOUT (-5)     /* a bounded device wait gave up         */
#define FTGEMM_ERR_UNRECOVERED (-6) /* offline ABFT: every attempt was hit   */

typedef struct ftgemm_ctx* ftgemm_handle_t;

/* element type of A and B.  C is always fp32, accumulation is always fp32. */
typedef enum {
  FTGEMM_F32 = 0,  /* fp32 operands, CUDA-core (SIMT) kernels              */
  FTGEMM_BF16 = 1, /* bf16 operands, tcgen05 tensor-core kernel            */
  FTGEMM_E4M3 = 2  /* fp8 E4M3 operands with per-tensor scales, tcgen05    */
} ftgemm_dtype;

/* granularity of the checksum unit (Section 4.2) */
typedef enum {
  FTGEMM_FT_OFF = 0,    /* plain GEMM, no checksums                           */
  FTGEMM_FT_THREAD = 1, /* unit = one thread's m_t x n_t fragment (4.2.1)     */
  FTGEMM_FT_WARP = 2,   /* unit = one warp's m_w x n_w tile (4.2.2)           */
  FTGEMM_FT_BLOCK = 3,  /* unit = the threadblock's m_tb x n_tb tile (4.2.3)  */
  FTGEMM_FT_TILE = 4,   /* unit = the tensor-core CTA tile, verified in the
                           epilogue (bf16 / e4m3 only)                        */
  FTGEMM_FT_AUTO = 5    /* F32: the level ftgemm_autotune found fastest for
                           this shape (BLOCK when the shape is not tuned)     */
} ftgemm_ft_level;

/* Kernel schedule: the 7-parameter tile tuple of Table 1 plus the checksum
 * cadence and split-K.  m_tb x n_tb is the CTA tile, k_tb the k-step width,
 * m_w x n_w the warp tile, m_t x n_t the thread tile.  cadence is the number
 * of k-steps per verification period (0 = verify once, after the last
 * k-step).  split_k >= 1 splits the k-steps into that many independent
 * partial products; each verifies its own partial, their sum is unprotected. */
typedef struct {
  int32_t m_tb, n_tb, k_tb;
  int32_t m_w, n_w, m_t, n_t;
  int32_t cadence;
  int32_t split_k;
} ftgemm_schedule;

/* Seeded fault injection (Section 5.3: an additive offset on an accumulator
 * register emulates a bit flip in the computing units).  n entries, each a
 * position in the schedule's tiling: output tile (tile_m, tile_n), the k-step
 * after whose update the offset is added (in units of the kernel's k-step;
 * -1 = the last k-step), and the tile-local row/col.  target (may be NULL,
 * meaning 0 for all) selects what is hit: 0 the accumulator of (row, col),
 * 1 the row checksum of `row` in the unit that holds `col`, 2 the column
 * checksum of `col` in the unit that holds `row`.  All arrays are HOST
 * memory; they are copied during the call.  A position outside the matrix
 * or outside the k range is rejected with FTGEMM_ERR_ARG. */
typedef struct {
  int32_t n;
  const int32_t* tile_m;
  const int32_t* tile_n;
  const int32_t* kstep;
  const int32_t* row;
  const int32_t* col;
  const int32_t* target;
  const float* delta;
} ftgemm_inject_spec;

/* One verification event with a flagged residual.  row/col are GLOBAL
 * indices of the located element (-1 when none was flagged on that side).
 * kind: 0 corrected (one row and one column flagged, residuals consistent),
 *       1 uncorrectable (more than one row or column flagged, or the two
 *         residuals disagree: the single-event-upset model was violated),
 *       2 checksum hit (one row xor one column flagged: the checksum itself
 *         was corrupted; it is reset from the data and C is left alone).
 * delta: the amount subtracted (kind 0) or the checksum's offset (kind 2).
 * residual_r / residual_c: the residuals of the flagged row / column.
 * tau: the sum of the thresholds of the flagged row and column.
 * problem: index of the problem in a grouped call (0 otherwise).           */
typedef struct {
  int32_t tile_m, tile_n, kstep, row, col, kind;
  int32_t problem, reserved;
  double delta, residual_r, residual_c, tau;
} ftgemm_fault_record;

/* Caller-owned report.  records points to `capacity` caller-owned slots.
 * On return n_records is the number of events (may exceed capacity, then
 * overflow = 1 and only the first `capacity` in sorted order are written).
 * Records are sorted by (problem, tile_m, tile_n, kstep, row, col, kind).   */
typedef struct {
  int64_t detected;      /* unit-periods with at least one flagged residual */
  int64_t corrected;     /* kind 0 */
  int64_t uncorrectable; /* kind 1 */
  int64_t checksum_only; /* kind 2 */
  int32_t capacity;
  int32_t n_records;
  int32_t overflow;
  int32_t reserved;
  ftgemm_fault_record* records;
} ftgemm_report;

/* ---- handle ------------------------------------------------------------- */

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Makes `device`
 * current on the calling thread.  (Runtime plumbing, no counterpart in the
 * paper.) */
int ftgemm_create(ftgemm_handle_t* handle, int device, void* cuda_stream);
/* Release the handle and its workspaces (synchronises its stream).
 * (Runtime plumbing, no counterpart in the paper.) */
int ftgemm_destroy(ftgemm_handle_t handle);
/* Change the stream later calls enqueue on.  (Runtime plumbing, no
 * counterpart in the paper.) */
int ftgemm_set_stream(ftgemm_handle_t handle, void* cuda_stream);

/* Fix the schedule of later fp32 calls (NULL = choose per shape, see
 * ftgemm_get_schedule).  FTGEMM_ERR_UNSUPPORTED if the tile tuple is not one
 * of the compiled kernels (Table 1's five tuples); cadence must be >= 0 and
 * split_k >= 1. */
int ftgemm_set_schedule(ftgemm_handle_t handle, const ftgemm_schedule* schedule);
/* The schedule ftgemm_gemm would use for this problem: a tile tuple of
 * Table 1 (the kernel parameters of Section 3.2.2), the verification
 * cadence (default K_s = 256 of Section 5.3) and split-K. */
int ftgemm_get_schedule(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k,
                        ftgemm_dtype dtype, ftgemm_ft_level ft_level,
                        ftgemm_schedule* out);

/* Detection threshold (Section 2.2 leaves its value open).
 * mode 0, analytic: at a verification after k elements of K,
 *     tau_row(i) = lambda * u * ||A(i,:)||_2 * ||B(:,J)||_F + mu * u * sqrt(k) * |c_row(i)|
 *     tau_col(j) = lambda * u * ||A(I,:)||_F * ||B(:,j)||_2 + mu * u * sqrt(k) * |c_col(j)|,
 *   J (I) the columns (rows) of the verification unit, c the row / column
 *   checksum as it stands, u = 2^-24 (2^-53 for ftgemm_dgemm / _zgemm),
 *   mu = 8.  The first term covers the rounding error of zero-mean data, the
 *   second the growth of the partial sums of same-sign data.  lambda (> 0)
 *   sets the fp32 and fp64 paths' value (default 32; <= 0 keeps it); the
 *   tensor-core path keeps lambda = 32.  Turns the learned threshold off.
 *   Every path screens residuals in fp32 against tau / 2 and confirms the
 *   screened ones in fp64 against tau.
 * mode 1, learned (no counterpart in the paper; the tensor-core path at
 *   level TILE and the fp32 path at level BLOCK): each tile uses
 *   lambda_t = lambda * 2^f(x_t) in the norm term, with no growth term,
 *   f the 5 -> 32 -> 32 -> 1 ReLU network whose FTGEMM_MLP_PARAMS parameters
 *   mlp_weights holds (host array, copied; layout W1[32][5], b1[32],
 *   W2[32][32], b2[32], W3[32], b3), x_t the tile's features: log2(K)/16,
 *   the coherence ||e^T A_I||_2 / (sqrt|I| ||A_I||_F) of its row block, the
 *   same ||B_J e||_2 / (sqrt|J| ||B_J||_F) of its column block, the operand
 *   type (0 fp32, 0.5 bf16, 1 e4m3) and log2(|I| |J|)/16.  f is evaluated
 *   once per tile inside the GEMM kernel; a non-finite or non-positive
 *   lambda_t falls back to the analytic threshold.  lambda (the calibration
 *   scale) must be > 0.  The fp32 levels THREAD and WARP keep the analytic
 *   threshold.  Synchronises the handle's stream.
 * Other modes: FTGEMM_ERR_UNSUPPORTED. */
#define FTGEMM_MLP_INPUTS 5
#define FTGEMM_MLP_PARAMS 1281
int ftgemm_set_threshold(ftgemm_handle_t handle, int mode, double lambda,
                         const float* mlp_weights, size_t n_weights);

/* Residual sink for training the learned threshold (no counterpart in the
 * paper): while set, every tensor-core call at level TILE and every fp32
 * call at level BLOCK writes, for each of its tiles t (t = tile_m * tiles_n
 * + tile_n; in a group, offset by the tiles of the problems scheduled before
 * it), lam_needed[t] = the largest |residual| / (u * norm product) over the
 * tile's rows, columns and (fp32) verification periods -- the smallest
 * lambda of the norm term alone that flags nothing there -- and its 5
 * features into features[5t .. 5t+4] (device arrays of `capacity` tiles,
 * owned by the caller).  lam_needed = NULL removes the sink.  A call with
 * more tiles than `capacity` fails with FTGEMM_ERR_ARG. */
int ftgemm_set_residual_sink(ftgemm_handle_t handle, float* lam_needed, float* features,
                             int64_t capacity);

/* The threshold network on the GPU (no counterpart in the paper).
 * X: n x 5 features, t: n targets, theta: FTGEMM_MLP_PARAMS parameters,
 * all device fp32.  ftgemm_mlp_forward writes the n outputs to y (device).
 * ftgemm_mlp_grad writes the gradient of the mean squared error
 * (1/n) sum (f(x_i) - t_i)^2 to grad (device) and, if loss is not NULL, the
 * loss to *loss (host; synchronises).  ftgemm_mlp_train runs `epochs`
 * passes of minibatch Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate
 * lr) over the samples in order, `batch` per step, updating theta in place;
 * losses (host, may be NULL) receives the mean minibatch loss of each epoch
 * (synchronises).  Gradients are reduced in a fixed order: runs repeat bit
 * for bit. */
int ftgemm_mlp_forward(ftgemm_handle_t handle, int64_t n, const float* X, const float* theta, float* y);
int ftgemm_mlp_grad(ftgemm_handle_t handle, int64_t n, const float* X, const float* t,
                    const float* theta, float* grad, float* loss);
int ftgemm_mlp_train(ftgemm_handle_t handle, int64_t n, const float* X, const float* t,
                     int32_t epochs, int32_t batch, float lr, float* theta, float* losses);

/* Per-tensor scales of E4M3 operands: the product is scale_a * scale_b *
 * (A_q B_q) with A_q, B_q the stored codes (see ftgemm_quantize).  (No
 * counterpart in the paper, whose kernels are fp32.) */
int ftgemm_set_fp8_scales(ftgemm_handle_t handle, float scale_a, float scale_b);

/* ---- compute ------------------------------------------------------------ */

/* Operand quantization for the tensor-core path (no counterpart in the
 * paper, whose kernels are fp32).  x: n fp32 values (device); y: n outputs of
 * `dtype` (device).  FTGEMM_BF16: round to nearest even.  FTGEMM_E4M3: the
 * per-tensor scale s = amax(|x|) / 448 is computed on the device and
 * y = sat(RNE(x / s)) (OCP FP8 E4M3, saturating to +-448); if scale_out is
 * not NULL the stream is synchronised and s is written there (1 for bf16). */
int ftgemm_quantize(ftgemm_handle_t handle, int64_t n, const float* x, void* y,
                    ftgemm_dtype dtype, float* scale_out);

/* C = alpha * A * B + beta * C with online ABFT at `ft_level`: the checksums
 * of Eq. 1-2 carried through the K loop in the outer-product form of Eq. 4,
 * verified at the unit of Section 4.2.1 / 4.2.2 / 4.2.3 (or the tensor-core
 * tile), errors located and corrected as in Section 4.2.1 under the fault
 * model of Section 4.1; `inject` follows Section 5.3.
 * A, B: device pointers of `dtype` elements; C: device fp32.  With beta == 0
 * C is not read.  inject: NULL for none.  report: NULL = do not wait (events
 * accumulate in the handle until ftgemm_report_fetch); non-NULL = the
 * handle's events are cleared first, the stream is synchronised at the end
 * and the events of this call are returned.
 * Supported: F32 with OFF/THREAD/WARP/BLOCK; BF16 and E4M3 with OFF/TILE.
 * Tensor-core path (BF16/E4M3): the MMA tile is 128 x 256; at level TILE
 * its last 3 (BF16) or 5 (E4M3) rows and its last 4 (BF16) or 8 (E4M3)
 * columns carry the checksums, so a CTA computes a 125 x 252 (BF16) or 123 x 248 (E4M3) tile
 * of C (128 x 256 at level OFF; ftgemm_tc_tile returns it) and inject tile
 * indices and in-tile offsets refer to that grid; the k-step is one
 * 128-byte k-block (64 bf16 or 128 e4m3 elements); A must have a 16-byte
 * aligned base and row stride (FTGEMM_ERR_ALIGN otherwise); the checksums
 * of the tile are verified once, after its last k-step, from tensor memory;
 * injected faults are applied to the tensor-memory accumulator at that
 * point (the accumulation being additive, the k-step of a fault changes
 * only rounding); E4M3 results are scaled by ftgemm_set_fp8_scales.  B may
 * have any alignment: at level OFF a BF16 B with a 16-byte aligned base and
 * row stride is read in place, otherwise the call first writes a transposed
 * copy into the handle's workspace. */
int ftgemm_gemm(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k,
                double alpha, const void* A, int64_t lda, const void* B,
                int64_t ldb, double beta, float* C, int64_t ldc,
                ftgemm_dtype dtype, ftgemm_ft_level ft_level,
                const ftgemm_inject_spec* inject, ftgemm_report* report);

/* ---- grouped GEMM (tensor-core path) ----------------------------------- */

/* One GEMM of a group: C = alpha * A * B + beta * C, all device pointers,
 * row-major; A is m x k and B is k x n of the group's dtype, C is fp32. */
typedef struct {
  int64_t m, n, k;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
  double alpha, beta;
  float scale_a, scale_b; /* E4M3: per-tensor scales of A and B (ignored for BF16) */
} ftgemm_problem;

typedef struct ftgemm_group* ftgemm_group_t;

/* Prepare a group of GEMMs for one persistent launch (no counterpart in the
 * paper, whose experiments run one GEMM at a time; the tile shapes and the
 * online ABFT per tile are those of ftgemm_gemm's tensor-core path).  The
 * problems (host array, copied) fix the operand pointers and shapes; the
 * group owns the device problem table, the TMA descriptors and the encode
 * workspace (allocated here, synchronously).  dtype: BF16 or E4M3; level:
 * OFF or TILE.  The threshold in force on the handle is captured here.
 * Problems are scheduled longest-K first; records report the caller's
 * problem index.  Errors: FTGEMM_ERR_ARG (sizes, NULL, leading dimensions),
 * FTGEMM_ERR_ALIGN (A not 16-byte aligned), FTGEMM_ERR_UNSUPPORTED,
 * FTGEMM_ERR_CUDA (allocation). */
int ftgemm_group_create(ftgemm_handle_t handle, int32_t count, const ftgemm_problem* problems,
                        ftgemm_dtype dtype, ftgemm_ft_level ft_level, ftgemm_group_t* out);

/* Data tile of C that one tensor-core CTA computes and verifies (the
 * verification unit of the tensor-core path, Section 4.2's threadblock level
 * on the MMA tile): *rows x *cols = 128 x 256 at level OFF; at level TILE
 * 125 x 252 for BF16 and 123 x 248 for E4M3, the rest of the 128 x 256 MMA
 * tile carrying the checksum pieces.  Fault tile indices and in-tile offsets
 * of ftgemm_gemm and the grouped calls refer to this grid.  Host only, no
 * handle.  Errors: FTGEMM_ERR_ARG (NULL), FTGEMM_ERR_UNSUPPORTED (dtype F32,
 * levels other than OFF and TILE). */
int ftgemm_tc_tile(ftgemm_dtype dtype, ftgemm_ft_level ft_level, int32_t* rows, int32_t* cols);

/* The static schedule ftgemm_group_create builds, computed on the host
 * alone: no handle, no device work (no counterpart in the paper).  m, n, k:
 * host arrays of `count` problem sizes; dtype and ft_level as for
 * ftgemm_group_create; ncta: the persistent CTAs (ftgemm_group_create uses
 * min(total tiles, SM count)).  Problems are taken longest-K first (stable),
 * each problem's tiles in the kernel's raster (groups of 16 tile rows,
 * column by column inside a group), and each tile goes to the CTA with the
 * least work so far, a tile costing max(k-blocks, 6)
 * (longest-processing-time greedy).  Output: *total_tiles; if `tiles` is not
 * NULL, 4 * total_tiles int32 {problem (the caller's index), tile_m, tile_n,
 * k-blocks} listed CTA by CTA, each CTA's tiles in the order it runs them;
 * if `cta_start` is not NULL, ncta + 1 offsets: CTA c runs entries
 * cta_start[c] .. cta_start[c+1] - 1.  Both NULL: a size query.  Errors:
 * FTGEMM_ERR_ARG (NULL, sizes, ncta < 1, more than INT32_MAX tiles),
 * FTGEMM_ERR_UNSUPPORTED (dtype, level). */
int ftgemm_group_plan(int32_t count, const int64_t* m, const int64_t* n, const int64_t* k,
                      ftgemm_dtype dtype, ftgemm_ft_level ft_level, int32_t ncta, int32_t* tiles,
                      int32_t* cta_start, int32_t* total_tiles);

/* Tile grid of each problem (caller arrays of `count`): tiles of C of the
 * size ftgemm_tc_tile gives for the group's dtype and level.  (No
 * counterpart in the paper.) */
int ftgemm_group_tiles(ftgemm_group_t group, int32_t* tiles_m, int32_t* tiles_n);

/* Faults applied by every later ftgemm_grouped_gemm of the group (the
 * injection of Section 5.3, per problem): problem[i] is the problem of
 * fault i, the other fields as in ftgemm_gemm's inject
 * (tile indices and in-tile offsets on that problem's grid).  NULL or n = 0
 * clears them.  Synchronises the handle's stream; not for use while a
 * stream capture is in progress. */
int ftgemm_group_set_faults(ftgemm_group_t group, const int32_t* problem, const ftgemm_inject_spec* inject);

/* Enqueue the group on the handle's stream: the batched encode pass (Eq. 1-2)
 * and one persistent tensor-core launch over every tile of every problem,
 * each tile verified as in ftgemm_gemm (no counterpart in the paper, which
 * runs one GEMM at a time).  No host
 * synchronisation and no allocation, so the call can be captured into a CUDA
 * graph and replayed; each replay recomputes every C.  Fault events
 * accumulate in the handle; read them with ftgemm_report_fetch. */
int ftgemm_grouped_gemm(ftgemm_handle_t handle, ftgemm_group_t group);

/* ftgemm_grouped_gemm with the operands taken from a DEVICE array:
 * `problems` is a device pointer to `count` ftgemm_problem (count = the
 * group's, the caller's order, 8-byte aligned), read on the handle's stream
 * when the call runs, so a captured graph replays with whatever the array
 * holds at replay time (no host synchronisation, no allocation; the call
 * enqueues a small rebinding kernel, then what ftgemm_grouped_gemm does).
 * Each entry's m, n, k, lda and ldb must be those the group was created
 * with (they fix its tile schedule, its workspace and its tensor maps); A,
 * B, C, ldc, alpha, beta and the e4m3 scales are taken from the entry.  The
 * other rules, checked on the device, are those of ftgemm_group_bind_rule.
 * An entry that breaks one is skipped: its problem is neither read nor
 * written by this call or by later calls of the group until a rebinding
 * meets the rules, and the next ftgemm_report_fetch returns FTGEMM_ERR_ARG
 * (after filling the report).  A binding persists: a later
 * ftgemm_grouped_gemm computes on the operands last bound.  (No
 * counterpart in the paper, which runs one GEMM at a time.)
 * Host-side errors: FTGEMM_ERR_ARG (NULL, count differs, array misaligned,
 * another handle's group), FTGEMM_ERR_CUDA. */
int ftgemm_grouped_gemm_dev(ftgemm_handle_t handle, ftgemm_group_t group, int32_t count,
                            const ftgemm_problem* problems);

/* The rule ftgemm_grouped_gemm_dev applies on the device to an entry
 * `bound` of a group whose problem was `created` (both host structs; no
 * device work), for a group of `dtype` and `level`.  Returns 0 when `bound`
 * may rebind the problem, else the first rule broken: 1 m, n or k differ;
 * 2 lda or ldb differ; 3 A, B or C NULL; 4 A not 16-byte aligned; 5 B not
 * aligned to its element (bf16), or not 16-byte aligned where the MMA reads
 * it in place (bf16 at level OFF when the created B was 16-byte aligned with
 * a 16-byte multiple row stride); 6 ldc < n or C not 4-byte aligned; 7 an
 * e4m3 scale not positive or their product not finite.  Negative: an
 * error code (NULL argument, FTGEMM_ERR_UNSUPPORTED dtype or level). */
int ftgemm_group_bind_rule(const ftgemm_problem* created, const ftgemm_problem* bound, ftgemm_dtype dtype,
                           ftgemm_ft_level level);

/* Release a group (synchronises the handle's stream first).  (No
 * counterpart in the paper.) */
int ftgemm_group_destroy(ftgemm_group_t group);

/* ftgemm_group_create with the schedule chosen by measurement: the group is
 * built on single CTAs and on CTA pairs, both run once untimed and then
 * timed in `reps` rounds of one call each, the order alternating between
 * rounds (every C is overwritten); the one with the better best time is
 * returned in *out (the other is released); *pair_out (may be NULL): 1
 * pairs, 0 single CTAs.
 * Synchronises the handle's stream.  Errors: FTGEMM_ERR_ARG (NULL, count,
 * reps < 1) and those of ftgemm_group_create / ftgemm_grouped_gemm. */
int ftgemm_group_autotune(ftgemm_handle_t handle, int32_t count, const ftgemm_problem* problems,
                          ftgemm_dtype dtype, ftgemm_ft_level ft_level, int32_t reps, ftgemm_group_t* out,
                          int32_t* pair_out);

/* Autotuner (F32 SIMT path).  The paper picks kernel parameters per shape
 * by a code-generation search (Section 3.2); here the compiled tile tuples,
 * split-K and the verification cadence are timed on the given operands and
 * the fastest kept: (1) every tuple with the paper's period K_s = 256 and no
 * split-K, plus the default schedule; (2) split-K 2, 4, ... for the two
 * fastest while every split keeps >= 8 k-steps; (3) for the fastest,
 * verification once per split instead of every K_s.  With ft_level =
 * FTGEMM_FT_AUTO the search also runs at BLOCK, WARP and THREAD and keeps the
 * fastest level.  Each candidate runs once untimed, then `reps` times
 * between CUDA events (alpha = 1, beta = 0: C is overwritten).  The result is
 * cached in the handle for (m, n, k, ft_level) and used by later ftgemm_gemm
 * and ftgemm_get_schedule calls with that shape and level unless a schedule
 * is forced with ftgemm_set_schedule.  out / level_out may be NULL. */
int ftgemm_autotune(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, const float* A,
                    int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc,
                    ftgemm_ft_level ft_level, int32_t reps, ftgemm_schedule* out,
                    ftgemm_ft_level* level_out);

/* Autotuner for the tensor-core path (the parameter selection of Section
 * 3.2, done by measurement): times ftgemm_gemm on the given operands (C is
 * overwritten; alpha 1, beta 0, no faults) on single CTAs and on CTA pairs,
 * once each untimed and then in `reps` rounds of one call each (the order
 * alternating between rounds, so that a drift of the clocks weighs on both
 * alike), and caches the one with the better best time for (m, n, k,
 * dtype, ft_level); later ftgemm_gemm calls with that shape use it while
 * ftgemm_set_tc_pair is at its default (-1).  dtype BF16 or E4M3 (set the
 * fp8 scales first), ft_level OFF or TILE.  *pair_out (may be NULL): 1 if
 * pairs were faster, else 0.  Synchronises the handle's stream.  Errors:
 * FTGEMM_ERR_ARG, FTGEMM_ERR_UNSUPPORTED, and those of ftgemm_gemm. */
int ftgemm_autotune_tc(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                       const void* B, int64_t ldb, float* C, int64_t ldc, ftgemm_dtype dtype,
                       ftgemm_ft_level ft_level, int32_t reps, int32_t* pair_out);

/* Self-test of the bounded device waits (no counterpart in the paper).
 * Every mbarrier wait of the GEMM kernels gives up after about 2^31 SM
 * cycles, counts the give-up in the handle's report and lets the kernel
 * return, so that a lost copy or MMA completion ends in FTGEMM_ERR_TIMEOUT
 * rather than a hung GPU.  This call launches one CTA that waits on a
 * barrier nothing arrives on, with a limit of `limit_cycles` (1 .. 2^34),
 * then fetches the report: it returns FTGEMM_ERR_TIMEOUT when the path
 * works, and the handle stays usable.  Synchronises the handle's stream. */
int ftgemm_selftest_wait(ftgemm_handle_t handle, int64_t limit_cycles);

/* Non-fused ABFT baseline (the comparison scheme of Section 5.3, after Ding
 * et al.), for measurement: F32 only.  C is accumulated as a sequence of
 * rank-K_s updates C_acc += A(:, s) B(s, :) (K_s = ks, a multiple of 16;
 * <= 0 gives 256), each a separate GEMM launch; the checksums (e^T A) B and
 * A (B e) of every 128 x 128 tile are updated by separate GEMM launches
 * (Eq. 4); after each step faults scheduled inside it are applied and a
 * separate kernel verifies every tile, locates, corrects and reports, with
 * the threshold of ftgemm_set_threshold mode 0.  Finally C = alpha * C_acc +
 * beta * C.  inject: tile_m / tile_n on the 128 x 128 grid, kstep in units
 * of 16 of K (the fault lands at the end of the step holding it), as for
 * ftgemm_gemm at BLOCK level with cadence K_s / 16.  Uses a second handle
 * workspace (allocated on first use).  Errors as ftgemm_gemm. */
int ftgemm_gemm_nonfused(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, double alpha,
                         const float* A, int64_t lda, const float* B, int64_t ldb, double beta,
                         float* C, int64_t ldc, int32_t ks, const ftgemm_inject_spec* inject,
                         ftgemm_report* report);

/* Offline ABFT (Section 5.5): detect-only verification with recompute.
 * F32.  Attempt r computes C = alpha * A * B + beta * C_in with a
 * detect-only kernel on the 128 x 128 x 32 tile (16 x 8 fragments): each
 * tile keeps only its column checksums e^T C (no row checksums, no
 * correction state), compared once, after the last k-step, against the
 * analytic threshold; a mismatch is reported as a detection (kind
 * uncorrectable, row -1, the most flagged column) and nothing is corrected.
 * injects[r] holds the faults of attempt r (NULL entry or injects NULL: no
 * faults; positions as for ftgemm_gemm on that tiling, k-steps of 32; a
 * row-checksum target is not seen); if anything is detected the attempt is
 * discarded and the next one starts from C_in.
 * *runs_out (may be NULL) receives the attempts made.  Returns
 * FTGEMM_ERR_UNRECOVERED when all max_runs attempts were hit (C then holds
 * the last attempt).  report (may be NULL): the events of all attempts.
 * The online scheme (ftgemm_gemm) corrects in place instead; the paper's
 * expected attempt count under a per-tile error rate gamma0 is
 * (1 - gamma) / (1 - 2 gamma), gamma = 1 - (1 - gamma0)^tiles. */
int ftgemm_gemm_offline(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, double alpha,
                        const float* A, int64_t lda, const float* B, int64_t ldb, double beta,
                        float* C, int64_t ldc, const ftgemm_inject_spec* const* injects,
                        int32_t max_runs, int32_t* runs_out, ftgemm_report* report);

/* ---- double and double complex (Section 6: DGEMM / ZGEMM extension) ---- */

#define FTGEMM_DGEMM_TILE 128 /* output tile (and checksum unit) of ftgemm_dgemm */
#define FTGEMM_ZGEMM_TILE 64  /* output tile (and checksum unit) of ftgemm_zgemm */
#define FTGEMM_F64_KSTEP 8    /* k-step of both: the unit of inject kstep and cadence */
#define FTGEMM_TARGET_IMAG 4  /* ftgemm_zgemm inject target flag: offset on the imaginary part */

/* C = alpha * A * B + beta * C in double precision on the CUDA cores, with
 * the online ABFT of the paper at block level: e^T A per 128-row block and
 * B e per 128-column block (Eq. 1-2) accumulate beside each 128 x 128
 * output tile during the K loop (Eq. 4); every `cadence` k-steps of 8
 * (cadence <= 0: once, after the last k-step) the tile's row and column
 * sums are compared with them against the analytic threshold of
 * ftgemm_set_threshold mode 0 with u = 2^-53 (lambda * u * ||A(i,:)|| *
 * ||B(:,J)||_F + mu * u * sqrt(k) * |checksum| and its column form; the
 * comparison is in double, no screen), and one corrupted element is located and
 * corrected or a corrupted checksum reset (Section 4.2.1); records as for
 * ftgemm_gemm.  Device pointers, row-major, leading dimensions in elements
 * (lda >= k, ldb >= n, ldc >= n); beta == 0: C is not read.  ft_level:
 * FTGEMM_FT_OFF or FTGEMM_FT_BLOCK (FTGEMM_FT_AUTO runs BLOCK); others give
 * FTGEMM_ERR_UNSUPPORTED.  inject: tile_m / tile_n on the 128 x 128 grid,
 * kstep in units of 8 of K, target 0 / 1 / 2 as for ftgemm_gemm; the offset
 * is delta.  report may be NULL.  Enqueued on the handle's stream;
 * synchronises only when report is given. */
int ftgemm_dgemm(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, ftgemm_ft_level ft_level, int32_t cadence,
                 const ftgemm_inject_spec* inject, ftgemm_report* report);

/* The same for double complex on 64 x 64 tiles (ZGEMM, the other extension
 * Section 6 names): matrices of interleaved
 * (re, im) doubles (C99 double complex layout), 16-byte aligned, leading
 * dimensions in complex elements; alpha and beta are HOST arrays {re, im}.
 * Norms are sqrt(sum |a|^2); a residual d is flagged when |d| exceeds its
 * threshold; the largest |d| / tau is located.  inject targets may carry
 * FTGEMM_TARGET_IMAG: the offset is then delta * i.  Records hold the real
 * parts of delta, residual_r and residual_c; when `imag` (HOST, 3 doubles
 * per record slot of the report, may be NULL) is given it receives their
 * imaginary parts in the same order as report->records. */
int ftgemm_zgemm(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k, const double* alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, const double* beta,
                 double* C, int64_t ldc, ftgemm_ft_level ft_level, int32_t cadence,
                 const ftgemm_inject_spec* inject, ftgemm_report* report, double* imag);

/* Synchronise the handle's stream, copy out the events accumulated since the
 * last fetch (or the last call that returned a report) and clear them: the
 * located and corrected errors of Section 4.2.1, one record each.  The
 * report is filled in any case; the return value is then FTGEMM_ERR_TIMEOUT
 * if a bounded device wait gave up, else FTGEMM_ERR_ARG if entries of a
 * device problem array were skipped (ftgemm_grouped_gemm_dev), else
 * FTGEMM_OK. */
int ftgemm_report_fetch(ftgemm_handle_t handle, ftgemm_report* report);

/* Checksum encoding on its own (Eq. 1-2), fp32:
 *   V[b*k + kk] = sum_{i in [b*m_u, (b+1)*m_u)} A[i][kk]   (ceil(m/m_u) x k)
 *   W[b*k + kk] = sum_{j in [b*n_u, (b+1)*n_u)} B[kk][j]   (ceil(n/n_u) x k)
 *   nA[i] = ||A(i,:)||_2 (m values), nB[j] = ||B(:,j)||_2 (n values).
 * All pointers are device pointers; any output may be NULL to skip it. */
int ftgemm_encode(ftgemm_handle_t handle, int64_t m, int64_t n, int64_t k,
                  const float* A, int64_t lda, const float* B, int64_t ldb,
                  int32_t m_u, int32_t n_u, float* V, float* W, float* nA,
                  float* nB);

/* ---- instrumentation ---------------------------------------------------- */

/* Counters of the handle.  launches: kernels enqueued by this handle (all
 * kinds).  With timing enabled, CUDA events recorded on the handle's stream
 * bracket every main GEMM kernel launch; kernel_ms is the sum of their
 * durations and timed_launches their number. */
typedef struct {
  int64_t launches;
  int64_t timed_launches;
  double kernel_ms;
} ftgemm_stats;

/* Tensor-core calls on CTA pairs (mode 1), on single CTAs (0), or chosen by
 * operand type (-1, the default: bf16 on pairs, e4m3 on single CTAs, the
 * faster of the two as measured), for later ftgemm_gemm calls and groups
 * created afterwards.  Other modes: FTGEMM_ERR_ARG.  A pair is a
 * cluster of two CTAs on two SMs that compute one 256 x 256 MMA tile with
 * cta_group::2 MMAs: each CTA holds its own 128 rows of A and half of B's
 * columns, and verifies its own tile of C exactly as a single CTA does
 * (same tile grid, same checksum layout, same records), so results are
 * identical either way; each SM then moves 32 KB of operands per k-block
 * instead of 48 KB.  (Kernel schedule, no counterpart in the paper.) */
int ftgemm_set_tc_pair(ftgemm_handle_t handle, int mode);

/* Enable (1) or disable (0) the events around the main GEMM kernel.
 * (Measurement plumbing, no counterpart in the paper.) */
int ftgemm_enable_timing(ftgemm_handle_t handle, int enable);
/* Synchronise the handle's stream and read the counters; reset != 0 zeroes
 * them afterwards.  (Measurement plumbing, no counterpart in the paper.) */
int ftgemm_get_stats(ftgemm_handle_t handle, ftgemm_stats* out, int reset);

/* ---- allocation-free entry point --------------------------------------- */
/* The paper has no counterpart of this entry point.
 *
 * Size of the fixed device array ftgemm_gemm_noalloc works in (16 MiB).  It
 * is compiled into the library, so every GPU that loads the library holds it
 * until the process exits. */
#define FTGEMM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* C = alpha * A * B + beta * C (fp32, the 128 x 128 x 16 tile, the checksum
 * levels of Section 4.2, verification every 256 of K, no split-K, no fault
 * injection) without allocating any device memory and without a handle (no
 * counterpart in the paper).  It is for callers that may not call
 * cudaMalloc when they need the GEMM: a framework whose memory pool owns the
 * device, code that must not cause the device-wide synchronisation that
 * cudaMalloc / cudaFree can, or recovery code after an out-of-memory error.
 * All temporaries (transposed A, encoded vectors, norms, event report) live
 * in the library's fixed array of FTGEMM_NOALLOC_SCRATCH_BYTES; a problem
 * that needs more is rejected with FTGEMM_ERR_ARG and a message naming the
 * bytes it would need (roughly 4*K*M bytes plus small vectors).
 * The array is shared by every call and keeps the last call's contents; each
 * call clears the report counters it relies on.  Calls that overlap on the
 * GPU (different streams, concurrent host threads) race on the array:
 * serialise them.  The first call on a device sets that device up while it
 * is current: it looks up the array's address and loads every kernel a call
 * can launch.  With lazy module loading (CUDA's default) that set-up can
 * itself allocate device memory, so the promise holds from the second call
 * on: make one call (any size, any level) at start-up, before relying on it
 * and before any stream capture.
 * A, B, C: device pointers on the current device; cuda_stream: a
 * cudaStream_t (NULL = legacy default stream); level: FTGEMM_FT_OFF..BLOCK;
 * report: NULL, or as for ftgemm_gemm: at most 256 records are kept per
 * call, sorted as ftgemm_report_fetch sorts them before the first
 * `capacity` are copied; the call then synchronises the stream.  Bounded
 * device waits that gave up stay counted in the array until a call with a
 * report reads the count: that call returns FTGEMM_ERR_TIMEOUT and clears
 * it, so a give-up in an earlier call without a report is reported there. */
int ftgemm_gemm_noalloc(int64_t m, int64_t n, int64_t k, double alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, double beta, float* C,
                        int64_t ldc, ftgemm_ft_level ft_level, void* cuda_stream,
                        ftgemm_report* report);

/* Text of a status code.  (No counterpart in the paper.) */
const char* ftgemm_status_string(int status);
/* Text of the last error raised on the calling thread ("" if none).  (No
 * counterpart in the paper.) */
const char* ftgemm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FTGEMM_H */
