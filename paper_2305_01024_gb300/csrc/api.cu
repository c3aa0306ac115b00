// api.cu -- the C ABI of libftgemm (include/ftgemm.h): handle, argument
// checks, schedule choice, fault table, workspaces, dispatch and report.
// Each entry point implements the passage its declaration in ftgemm.h cites
// (Eq. 1-4 and Sections 4.1-4.2 for the GEMMs, Section 5.3 for injection,
// Section 5.5 for the offline scheme, Section 6 for DGEMM / ZGEMM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "fp64.cuh"

namespace ftg {
using SimtLaunch = cudaError_t (*)(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_small(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_medium(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_large(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_tall(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_huge(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_huge16(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_wide(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_wide32(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_wide32_detect(const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t launch_transpose(const float*, long long, int, int, float*, long long, cudaStream_t);
cudaError_t launch_transpose_encode(const float* A, long long lda, int M, int K, float* At, long long ldt, int m_u,
                                    float* V, long long ldv, float* nrm, float* scratch, int* launches,
                                    cudaStream_t st);
cudaError_t launch_copy_pad(const float*, long long, int, int, float*, long long, cudaStream_t);
long long kmajor_scratch_floats(int K, int L);
cudaError_t launch_encode_rowmajor(const float* A, long long lda, int M, int K, int m_u, float* V, long long ldv,
                                   float* nA, float* scratch, int* launches, cudaStream_t st);
cudaError_t launch_encode_kmajor(const float*, long long, int, int, int, float*, long long, float*,
                                 float*, int*, cudaStream_t);
cudaError_t launch_splitk_reduce(const float*, int, int, int, float, float, float*, long long,
                                 cudaStream_t);
void tc_prep_blocks(const TcProblem& P, int dt, int out[P_KINDS]);
int tc_nb_parts(int dt, long long K);
cudaError_t launch_tc_bind(TcProblem* probs, TcProbMaps* maps, const int* pos, const ftgemm_problem* in, int count,
                           int dt, DevReport* rep, cudaStream_t st);
cudaError_t launch_tc_prep(int dt, bool abft, const TcBatch& b, const int total[P_KINDS],
                           const int* const* bmap, int* launches, cudaStream_t st);
cudaError_t launch_tc_gemm(int dt, bool abft, bool pair, const TcBatch& b, const TcMapsBatch& mb, const TcRun& run, int grid,
                           cudaStream_t st);
cudaError_t launch_quantize(int dt, const float* x, long long n, void* y, unsigned int* amax_bits, float* scale,
                            int* launches, cudaStream_t st);
cudaError_t launch_fault_bits(const Fault* f, int n, uint32_t* bits, size_t words, cudaStream_t st);
cudaError_t launch_wait_selftest(DevReport* rep, long long limit_cycles, cudaStream_t st);
cudaError_t launch_nonfused_inject(const Fault* f, int nf, int ks_lo, int ks_hi, int tiles_n, float* acc,
                                   long long ldacc, float* Cc, long long ldcc, float* CrT, long long ldcr,
                                   cudaStream_t st);
cudaError_t launch_block_coherence(const float* V, const float* W, long long ldv, int K, const float* nA,
                                   const float* nB, int M, int N, int m_u, int n_u, float* coA, float* coB,
                                   cudaStream_t st);
cudaError_t launch_nonfused_verify(float* acc, long long ldacc, int M, int N, float* Cc, long long ldcc,
                                   float* CrT, long long ldcr, const float* nA, const float* nB, float lam_u,
                                   float grow, int kstep, DevReport* rep, ftgemm_fault_record* recs,
                                   cudaStream_t st);
cudaError_t launch_nonfused_epilogue(const float* acc, long long ldacc, int M, int N, float alpha, float beta,
                                     float* C, long long ldc, cudaStream_t st);
int mlp_grad_blocks(long long nb);
cudaError_t launch_mlp_grad(const float* X, const float* t, long long s0, int nb, const float* theta, float inv_n,
                            float* part, int nblk, cudaStream_t st);
cudaError_t launch_mlp_reduce(const float* part, int nblk, float* grad_out, float* theta, float* m, float* v, int step,
                              float lr, float inv_n, float* loss_out, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* X, long long n, const float* theta, float* y, cudaStream_t st);

// The compiled SIMT tile tuples: the five kernel setups of Table 1, plus the
// large tile with a 16-wide k-step in two thread layouts (8 x 8 fragments on
// 256 threads, and 16 x 8 fragments on 128 threads, the GB300 default for
// big problems: fewer shared-memory wavefronts per FMA).
struct SimtConfig {
  const char* name;
  int m_tb, n_tb, k_tb, m_w, n_w, m_t, n_t;
  SimtLaunch launch;
};
static const SimtConfig kSimtConfigs[] = {
    {"wide", 128, 128, 16, 64, 64, 16, 8, simt_launch_wide},
    {"wide32", 128, 128, 32, 64, 64, 16, 8, simt_launch_wide32},
    {"huge16", 128, 128, 16, 32, 64, 8, 8, simt_launch_huge16},
    {"huge", 128, 128, 8, 32, 64, 8, 8, simt_launch_huge},
    {"large", 64, 64, 8, 32, 64, 8, 8, simt_launch_large},
    {"tall", 32, 128, 8, 16, 64, 4, 8, simt_launch_tall},
    {"medium", 32, 32, 8, 16, 32, 4, 4, simt_launch_medium},
    {"small", 16, 16, 16, 8, 16, 2, 2, simt_launch_small},
};

static const SimtConfig* find_simt(const ftgemm_schedule& s) {
  for (const auto& c : kSimtConfigs)
    if (c.m_tb == s.m_tb && c.n_tb == s.n_tb && c.k_tb == s.k_tb && c.m_w == s.m_w &&
        c.n_w == s.n_w && c.m_t == s.m_t && c.n_t == s.n_t)
      return &c;
  return nullptr;
}

static thread_local std::string g_last_error;

// Lets other translation units report through ftgemm_last_error().
void set_last_error(const char* msg) { g_last_error = msg; }

}  // namespace ftg

using namespace ftg;

// Scale of the threshold's checksum-growth term mu * u * sqrt(k) * |c| (the
// analytic reading of the "predetermined threshold" of Section 2.2), on the
// CUDA cores and on the tensor cores alike.
constexpr double kMu = 8.0;

struct ftgemm_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  // workspace (floats), grown on demand
  float* ws = nullptr;
  size_t ws_floats = 0;
  // report
  DevReport* rep = nullptr;
  ftgemm_fault_record* recs = nullptr;
  int rep_cap = 1 << 16;
  // fault table
  Fault* d_faults = nullptr;
  Fault* h_faults = nullptr;  // pinned staging
  int faults_cap = 0;
  uint32_t* d_fbits = nullptr;  // tensor-core path: one bit per tile with a fault
  size_t fbits_words = 0;
  cudaEvent_t faults_free = nullptr;
  // settings
  bool has_sched = false;
  ftgemm_schedule sched{};
  double lambda = 32.0;
  double lambda_tc[2] = {32.0, 32.0};  // bf16, e4m3
  int tc_pair = -1;                      // tensor-core GEMMs on 2-CTA pairs (cta_group::2): 1 always,
                                         // 0 never, -1 automatic (bf16 only)
  // checksum-growth term of the analytic threshold, mu * u * sqrt(k) * |c|
  double mu = kMu;
  float fp8_sa = 1.f, fp8_sb = 1.f;
  float* qscratch = nullptr;  // amax bits + scale of ftgemm_quantize
  // learned threshold (tensor-core path)
  float* mlp_theta = nullptr;  // device, FTGEMM_MLP_PARAMS floats
  bool mlp_on = false;
  float mlp_scale = 1.f;
  float* mlp_ws = nullptr;     // training: block partials, Adam moments, step losses
  size_t mlp_ws_floats = 0;
  // autotuned SIMT schedules: (m, n, k, requested level) -> (schedule, level to run)
  std::map<std::tuple<int64_t, int64_t, int64_t, int>, std::pair<ftgemm_schedule, int>> tuned;
  // autotuned tensor-core schedules: (m, n, k, dtype, level) -> 1 CTA pairs, 0 single CTAs
  std::map<std::tuple<int64_t, int64_t, int64_t, int, int>, int> tc_tuned;
  // second workspace (non-fused baseline: its buffers live across the GEMM calls it makes)
  float* ws2 = nullptr;
  size_t ws2_floats = 0;
  // fp64 complex path: Im of (delta, residual_r, residual_c) per record slot
  double* zimag = nullptr;
  // residual sink (tensor-core path)
  float* sink_lam = nullptr;
  float* sink_x = nullptr;
  int64_t sink_cap = 0;
  // instrumentation
  int64_t launches = 0;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending, pool;
  int64_t timed = 0;
  double kernel_ms = 0.0;
};

#define FAIL(code, ...)                                                         \
  do {                                                                          \
    char _b[512];                                                               \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                                      \
    g_last_error = _b;                                                          \
    return (code);                                                              \
  } while (0)

#define CK(call)                                                                \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess)                                                      \
      FAIL(FTGEMM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(_e));    \
  } while (0)

static int ensure_ws(ftgemm_ctx* h, size_t floats) {
  if (floats <= h->ws_floats) return FTGEMM_OK;
  if (h->ws) {
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaFree(h->ws));
    h->ws = nullptr;
    h->ws_floats = 0;
  }
  size_t want = std::max(floats, h->ws_floats * 3 / 2);
  CK(cudaMalloc(&h->ws, want * sizeof(float)));
  h->ws_floats = want;
  return FTGEMM_OK;
}

static int ensure_faults(ftgemm_ctx* h, int n) {
  if (n <= h->faults_cap) return FTGEMM_OK;
  CK(cudaStreamSynchronize(h->stream));
  if (h->d_faults) CK(cudaFree(h->d_faults));
  if (h->h_faults) CK(cudaFreeHost(h->h_faults));
  h->d_faults = nullptr;
  h->h_faults = nullptr;
  const int cap = std::max(n, 2 * h->faults_cap);
  h->faults_cap = 0;  // nothing usable until both buffers exist
  CK(cudaMalloc(&h->d_faults, sizeof(Fault) * cap));
  CK(cudaHostAlloc(&h->h_faults, sizeof(Fault) * cap, cudaHostAllocDefault));
  h->faults_cap = cap;
  return FTGEMM_OK;
}

static size_t align64(size_t x) { return (x + 63) & ~size_t(63); }

static int default_schedule(const ftgemm_ctx* h, int64_t m, int64_t n, int64_t k, int level,
                            ftgemm_schedule* s) {
  const int sms = h->num_sms > 0 ? h->num_sms : 152;
  const SimtConfig* pick = nullptr;
  for (const auto& c : kSimtConfigs) {
    // the k_tb=8 variant and the k_tb=32 one only on request (or
    // through the autotuner): the latter wins only for long K at block level
    if (c.launch == simt_launch_huge || c.launch == simt_launch_wide32) continue;
    // on the 128 x 128 tile, 16 x 8 fragments win with checksums (fewer
    // shared-memory wavefronts per FMA leave room for the checksum loads),
    // 8 x 8 fragments without
    if (c.launch == simt_launch_wide && level == FTGEMM_FT_OFF) continue;
    if (c.launch == simt_launch_huge16 && level != FTGEMM_FT_OFF) continue;
    int64_t tiles = ((m + c.m_tb - 1) / c.m_tb) * ((n + c.n_tb - 1) / c.n_tb);
    if (tiles >= sms) { pick = &c; break; }
  }
  int split = 1;
  if (!pick) {
    // no tuple fills the GPU with output tiles alone: the big tile with split-K
    // when K is long, else the smallest tile.
    const SimtConfig& big = kSimtConfigs[0];
    int64_t tiles = ((m + big.m_tb - 1) / big.m_tb) * ((n + big.n_tb - 1) / big.n_tb);
    int64_t ksteps = (k + big.k_tb - 1) / big.k_tb;
    if (ksteps >= 256) {
      pick = &big;
      split = (int)std::min<int64_t>((2 * sms + tiles - 1) / tiles, ksteps / 64);
      split = std::max(split, 1);
    } else {
      pick = &kSimtConfigs[sizeof(kSimtConfigs) / sizeof(kSimtConfigs[0]) - 1];
    }
  }
  s->m_tb = pick->m_tb; s->n_tb = pick->n_tb; s->k_tb = pick->k_tb;
  s->m_w = pick->m_w; s->n_w = pick->n_w; s->m_t = pick->m_t; s->n_t = pick->n_t;
  s->cadence = std::max(1, 256 / pick->k_tb);  // period K_s = 256 (Section 5.3)
  s->split_k = split;
  return FTGEMM_OK;
}

// The schedule and level an F32 call runs with: the handle's forced
// schedule, else an autotuned one for this shape and requested level, else
// the default.  FTGEMM_FT_AUTO without a tuned entry runs BLOCK.
static void choose_schedule(const ftgemm_ctx* h, int64_t m, int64_t n, int64_t k, ftgemm_ft_level level,
                            ftgemm_schedule* s, ftgemm_ft_level* run_level) {
  *run_level = level == FTGEMM_FT_AUTO ? FTGEMM_FT_BLOCK : level;
  if (h->has_sched) {
    *s = h->sched;
    return;
  }
  auto it = h->tuned.find(std::make_tuple(m, n, k, (int)level));
  if (it != h->tuned.end()) {
    *s = it->second.first;
    *run_level = (ftgemm_ft_level)it->second.second;
    return;
  }
  default_schedule(h, m, n, k, (int)*run_level, s);
}

static int simt_gemm(ftgemm_ctx* h, int64_t m, int64_t n, int64_t k, double alpha, const float* A, int64_t lda,
                     const float* B, int64_t ldb, double beta, float* C, int64_t ldc, ftgemm_ft_level level,
                     const ftgemm_schedule& s, const ftgemm_inject_spec* inject, ftgemm_report* report,
                     const float* At_given = nullptr, int64_t ldat = 0, bool detect = false);

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D fp32 tensor map: dims {inner, outer}, row stride in elements, box {bi, bo}.
// Out-of-range box elements read as zero.
static int make_map_2d(CUtensorMap* m, const float* base, uint64_t inner, uint64_t outer,
                       uint64_t ld, uint32_t bi, uint32_t bo) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) FAIL(FTGEMM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * sizeof(float)};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    FAIL(FTGEMM_ERR_ALIGN, "cuTensorMapEncodeTiled failed (%d) for dims {%llu,%llu} ld %llu box {%u,%u}",
         (int)r, (unsigned long long)inner, (unsigned long long)outer, (unsigned long long)ld, bi, bo);
  return FTGEMM_OK;
}

// Validate an injection spec against the tiling, resolve k-step -1, sort by
// (tile, k-step) and upload it; *nf receives the number of faults.
static int upload_faults(ftgemm_ctx* h, const ftgemm_inject_spec* inject, const ftgemm_schedule& s, int M,
                         int N, int ksteps, int tiles_m, int tiles_n, ftgemm_ft_level level, int* nf_out,
                         bool imag_targets = false) {
  int nf = inject ? inject->n : 0;
  *nf_out = 0;
  if (nf < 0) FAIL(FTGEMM_ERR_ARG, "inject->n < 0");
  if (nf == 0) return FTGEMM_OK;
  if (!inject->tile_m || !inject->tile_n || !inject->kstep || !inject->row || !inject->col || !inject->delta)
    FAIL(FTGEMM_ERR_ARG, "inject: NULL array");
  int rc = ensure_faults(h, nf);
  if (rc) return rc;
  CK(cudaEventSynchronize(h->faults_free));  // staging buffer no longer read by a prior copy
  std::vector<Fault> fv(nf);
  for (int i = 0; i < nf; ++i) {
    const int tm = inject->tile_m[i], tn = inject->tile_n[i];
    int ks = inject->kstep[i];
    const int r = inject->row[i], c = inject->col[i];
    const int tg = inject->target ? inject->target[i] : 0;
    if (tm < 0 || tm >= tiles_m || tn < 0 || tn >= tiles_n)
      FAIL(FTGEMM_ERR_ARG, "inject[%d]: tile (%d,%d) outside the %dx%d tile grid", i, tm, tn, tiles_m, tiles_n);
    if (ks == -1) ks = ksteps - 1;
    if (ks < 0 || ks >= ksteps) FAIL(FTGEMM_ERR_ARG, "inject[%d]: k-step %d outside [0,%d)", i, ks, ksteps);
    const int rows = std::min(s.m_tb, M - tm * s.m_tb), cols = std::min(s.n_tb, N - tn * s.n_tb);
    if (r < 0 || r >= rows || c < 0 || c >= cols)
      FAIL(FTGEMM_ERR_ARG, "inject[%d]: element (%d,%d) outside tile (%d x %d)", i, r, c, rows, cols);
    const int tb = imag_targets ? (tg & ~FTGEMM_TARGET_IMAG) : tg;
    if (tg < 0 || tb > 2) FAIL(FTGEMM_ERR_ARG, "inject[%d]: target %d", i, tg);
    if (level == FTGEMM_FT_OFF && tb != 0) FAIL(FTGEMM_ERR_ARG, "inject[%d]: no checksums at level OFF", i);
    fv[i] = Fault{tm * tiles_n + tn, ks, r, c, tg, inject->delta[i]};
  }
  std::stable_sort(fv.begin(), fv.end(), [](const Fault& a, const Fault& b) {
    return a.tile != b.tile ? a.tile < b.tile : a.kstep < b.kstep;
  });
  memcpy(h->h_faults, fv.data(), sizeof(Fault) * nf);
  CK(cudaMemcpyAsync(h->d_faults, h->h_faults, sizeof(Fault) * nf, cudaMemcpyHostToDevice, h->stream));
  CK(cudaEventRecord(h->faults_free, h->stream));
  *nf_out = nf;
  return FTGEMM_OK;
}

// 2-D tensor map of 1- or 2-byte elements with the 128-byte swizzle (the
// K-major operand tiles of the tensor-core kernel).
static int make_map_sw128(CUtensorMap* m, const void* base, int elem, uint64_t inner, uint64_t outer,
                          uint64_t ld, uint32_t bi, uint32_t bo) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) FAIL(FTGEMM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * (uint64_t)elem};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    FAIL(FTGEMM_ERR_ALIGN, "cuTensorMapEncodeTiled (swizzled) failed (%d): dims {%llu,%llu} ld %llu box {%u,%u}",
         (int)r, (unsigned long long)inner, (unsigned long long)outer, (unsigned long long)ld, bi, bo);
  return FTGEMM_OK;
}

static int take_events(ftgemm_ctx* h, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
  if (!h->pool.empty()) {
    *ev = h->pool.back();
    h->pool.pop_back();
    return FTGEMM_OK;
  }
  CK(cudaEventCreate(&ev->first));
  CK(cudaEventCreate(&ev->second));
  return FTGEMM_OK;
}

static int drain_events(ftgemm_ctx* h) {
  if (h->pending.empty()) return FTGEMM_OK;
  CK(cudaStreamSynchronize(h->stream));
  for (auto& e : h->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e.first, e.second));
    h->kernel_ms += ms;
    h->timed += 1;
    h->pool.push_back(e);
  }
  h->pending.clear();
  return FTGEMM_OK;
}

static int clear_report(ftgemm_ctx* h) {
  CK(cudaMemsetAsync(h->rep, 0, offsetof(DevReport, capacity), h->stream));
  CK(cudaMemsetAsync(&h->rep->timeouts, 0, 2 * sizeof(int), h->stream));  // timeouts, bind_errors
  return FTGEMM_OK;
}
extern "C" int ftgemm_report_fetch(ftgemm_handle_t h, ftgemm_report* out);

// ---- tensor-core path: problem layout shared by ftgemm_gemm and groups ----

// CTA pairs for this operand type.  Automatic: bf16 on pairs (each SM moves a
// third fewer operand bytes per k-block: 7-11% faster kernels measured at
// 8192^3 and 16384^3, with or without checksums), e4m3 on single CTAs (its
// operands are half the bytes per flop; pairs measured level without
// checksums and 4% slower with them).
// A shape tuned by ftgemm_autotune_tc takes the schedule measured fastest.
static bool tc_use_pair(const ftgemm_ctx* h, int dt, int64_t m = 0, int64_t n = 0, int64_t k = 0, int level = 0) {
  if (h->tc_pair >= 0) return h->tc_pair != 0;
  const auto it = h->tc_tuned.find(std::make_tuple(m, n, k, dt, level));
  if (it != h->tc_tuned.end()) return it->second != 0;
  return dt == 0;
}

// Shape, tiling and epilogue fields of a tensor-core problem.
static void tc_set_problem(TcProblem& P, int dt, bool abft, int M, int N, int K, const void* A, int64_t lda,
                           const void* B, int64_t ldb, float* C, int64_t ldc, double alpha, double beta,
                           float acc_scale, float lam_u, double mu) {
  memset(&P, 0, sizeof(P));
  // checksum-growth term of the analytic threshold at the one verification, k = K
  P.grow = (float)(mu * std::ldexp(1.0, -24) * std::sqrt((double)K));
  const int dm = tc_dm(dt, abft), dn = tc_dn(dt, abft);
  const int kblk = dt == 0 ? 64 : 128;
  P.M = M; P.N = N; P.K = K;
  P.tiles_m = (M + dm - 1) / dm;
  P.tiles_n = (N + dn - 1) / dn;
  P.nkb = (K + kblk - 1) / kblk;
  P.A = A; P.lda = lda; P.B = B; P.ldb = ldb;
  P.ldk = (K + 127) / 128 * 128;  // elements; a 16-byte multiple for both types
  P.b_mn = tc_b_in_place(dt, abft, B, ldb);
  P.C = C; P.ldc = ldc;
  P.c_vec = (ldc % 4 == 0) && (((uintptr_t)C & 15) == 0);
  P.alpha = (float)alpha; P.beta = (float)beta;
  P.acc_scale = acc_scale;
  P.lam_u = lam_u;
}

// Encode buffers of one problem laid out from `ws` (floats); with ws null
// only the size is computed.  Returns the floats used.
static size_t tc_layout(TcProblem& P, int dt, bool abft, float* ws) {
  const size_t eb = dt == 0 ? 2 : 1, ns = TC_TAIL;
  const size_t tm = P.tiles_m, tn = P.tiles_n, K = P.K;
  auto fl = [&](size_t bytes) { return (bytes + 3) / 4; };
  size_t o = 0;
  auto take = [&](size_t floats) {
    const size_t at = o;
    o = align64(o + floats);
    return ws ? ws + at : nullptr;
  };
  P.Bt = P.b_mn ? nullptr : take(fl(eb * (size_t)P.N * P.ldk));
  if (abft) {
    P.Vf = take(tm * P.ldk);
    P.Wf = take(tn * P.ldk);
    P.Vt = take(fl(eb * tm * ns * P.ldk));
    P.Wt = take(fl(eb * tn * ns * P.ldk));
    P.vscale = take(tm * ns);
    P.wscale = take(tn * ns);
    P.s0v = take(tm);
    P.s0w = take(tn);
    P.nA = take(P.M);
    P.nB = take(P.N);
    P.nA_part = take((size_t)((K + 255) / 256) * P.M);
    P.nB_part = take((size_t)tc_nb_parts(dt, K) * P.N);
    P.froA = take(tm);
    P.froB = take(tn);
    P.coA = take(tm);
    P.coB = take(tn);
  }
  return o;
}

static int tc_make_maps(TcProbMaps& mp, const TcProblem& P, int dt, bool abft, bool pair) {
  const int elem = dt == 0 ? 2 : 1, BK = 128 / elem;
  // main boxes: every row of the MMA tile, or with checksums all but the
  // 8-row tail (the tile's last data rows and its pieces, from V / W)
  const int am = abft ? TC_AROWS : TC_BM, bn = abft ? TC_BROWS : TC_BN;
  const uint32_t ns = TC_TAIL;
  memset(&mp, 0, sizeof(mp));
  int rc = make_map_sw128(&mp.A, P.A, elem, P.K, P.M, P.lda, BK, am);
  if (!rc) {
    if (P.b_mn) {
      rc = make_map_sw128(&mp.B, P.B, elem, P.N, P.K, P.ldb, 64, BK);  // 64-column boxes
    } else if (pair) {  // the two halves of a pair's 256-column MMA tile
      rc = make_map_sw128(&mp.B, P.Bt, elem, P.K, P.N, P.ldk, BK, 128);
      if (!rc) rc = make_map_sw128(&mp.B1, P.Bt, elem, P.K, P.N, P.ldk, BK, bn - 128);
    } else {
      rc = make_map_sw128(&mp.B, P.Bt, elem, P.K, P.N, P.ldk, BK, bn);
    }
  }
  if (!rc && abft) rc = make_map_sw128(&mp.W, P.Wt, elem, P.K, (uint64_t)P.tiles_n * ns, P.ldk, BK, ns);
  if (!rc && abft) rc = make_map_sw128(&mp.V, P.Vt, elem, P.K, (uint64_t)P.tiles_m * ns, P.ldk, BK, ns);
  if (rc) return rc;
  if (!abft) { mp.W = mp.A; mp.V = mp.A; }
  if (!pair || P.b_mn) mp.B1 = mp.B;  // not used
  return FTGEMM_OK;
}

static int tc_check_operand_a(const void* A, int64_t lda, int elem, const char* who) {
  if (((uintptr_t)A & 15) || (lda * elem) % 16)
    FAIL(FTGEMM_ERR_ALIGN, "%s: A needs a 16-byte aligned base and row stride for TMA", who);
  return FTGEMM_OK;
}

// Tensor-core path of ftgemm_gemm (BF16 / E4M3 operands, levels OFF and TILE):
// one problem passed inline to the batched encode and the persistent GEMM.
static int tc_gemm(ftgemm_ctx* h, int64_t m, int64_t n, int64_t k, double alpha, const void* A, int64_t lda,
                   const void* B, int64_t ldb, double beta, float* C, int64_t ldc, ftgemm_dtype dtype,
                   ftgemm_ft_level level, const ftgemm_inject_spec* inject, ftgemm_report* report) {
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: bf16/e4m3 take level OFF or TILE, not %d", (int)level);
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1;
  {
    int rc = tc_check_operand_a(A, lda, dt == 0 ? 2 : 1, "ftgemm_gemm");
    if (rc) return rc;
  }
  CK(cudaSetDevice(h->device));
  const bool abft = level == FTGEMM_FT_TILE;
  TcBatch b;
  memset(&b, 0, sizeof(b));
  TcProblem& P = b.one;
  tc_set_problem(P, dt, abft, (int)m, (int)n, (int)k, A, lda, B, ldb, C, ldc, alpha, beta,
                 dt == 1 ? h->fp8_sa * h->fp8_sb : 1.f, (float)(h->lambda_tc[dt] * std::ldexp(1.0, -24)),
                 h->mu);
  P.mlp = h->mlp_on ? h->mlp_theta : nullptr;
  P.mlp_scale = h->mlp_scale;
  b.table = nullptr;
  b.nprob = 1;
  const bool pair = tc_use_pair(h, dt, m, n, k, (int)level);
  const int ntiles = P.tiles_m * P.tiles_n;
  // the raster's tiles: a pair's tile is two tile rows high
  b.total_tiles = pair ? ((P.tiles_m + 1) / 2) * P.tiles_n : ntiles;
  int nf = 0;
  {
    const int dm = tc_dm(dt, abft), dn = tc_dn(dt, abft);
    ftgemm_schedule tcs{dm, dn, dt == 0 ? 64 : 128, dm, dn, dm, dn, 0, 1};
    int rc = upload_faults(h, inject, tcs, P.M, P.N, P.nkb, P.tiles_m, P.tiles_n, level, &nf);
    if (rc) return rc;
  }
  {
    int rc = ensure_ws(h, tc_layout(P, dt, abft, nullptr));
    if (rc) return rc;
  }
  tc_layout(P, dt, abft, h->ws);
  if (report) {
    int rc = clear_report(h);
    if (rc) return rc;
  }
  int total[P_KINDS];
  tc_prep_blocks(P, dt, total);
  int launches = 0;
  CK(launch_tc_prep(dt, abft, b, total, nullptr, &launches, h->stream));
  TcMapsBatch mb;
  memset(&mb, 0, sizeof(mb));
  {
    int rc = tc_make_maps(mb.one, P, dt, abft, pair);
    if (rc) return rc;
  }
  if (h->sink_lam && abft && ntiles > h->sink_cap)
    FAIL(FTGEMM_ERR_ARG, "residual sink holds %lld tiles, the call has %d", (long long)h->sink_cap, ntiles);
  const uint32_t* fbits = nullptr;
  if (nf > 0) {
    const size_t words = ((size_t)ntiles + 31) / 32;
    if (words > h->fbits_words) {
      CK(cudaStreamSynchronize(h->stream));
      if (h->d_fbits) CK(cudaFree(h->d_fbits));
      h->d_fbits = nullptr;
      h->fbits_words = 0;
      CK(cudaMalloc(&h->d_fbits, words * sizeof(uint32_t)));
      h->fbits_words = words;
    }
    CK(launch_fault_bits(h->d_faults, nf, h->d_fbits, words, h->stream));
    ++launches;
    fbits = h->d_fbits;
  }
  TcRun run{nf > 0 ? h->d_faults : nullptr, nf, fbits, h->rep, h->recs, abft ? h->sink_lam : nullptr,
            abft ? h->sink_x : nullptr};
  const int sms = h->num_sms > 0 ? h->num_sms : 148;
  const int grid = pair ? 2 * std::max(1, std::min(b.total_tiles, sms / 2)) : std::max(1, std::min(b.total_tiles, sms));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (h->timing) {
    int rc = take_events(h, &ev);
    if (rc) return rc;
    CK(cudaEventRecord(ev.first, h->stream));
  }
  CK(launch_tc_gemm(dt, abft, pair, b, mb, run, grid, h->stream));
  ++launches;
  if (h->timing) {
    CK(cudaEventRecord(ev.second, h->stream));
    h->pending.push_back(ev);
  }
  h->launches += launches;
  if (report) return ftgemm_report_fetch(h, report);
  return FTGEMM_OK;
}

// A prepared group of tensor-core problems (ftgemm_group_create): device
// problem table in schedule order, tensor maps, encode workspace, faults.
struct ftgemm_group {
  ftgemm_ctx* h = nullptr;
  int dt = 0;
  bool abft = false;
  int count = 0;
  std::vector<TcProblem> probs;  // schedule order
  std::vector<int> pos;          // user index -> schedule position
  TcProblem* d_probs = nullptr;
  TcProbMaps* d_maps = nullptr;
  int4* d_tiles = nullptr;      // the schedule: per-CTA tile lists, concatenated
  int* d_cta_start = nullptr;   // [ncta + 1]
  int* d_bmap = nullptr;        // encode launches: the problem of every block, kinds concatenated
  int* d_pos = nullptr;         // caller index -> schedule position (device-array rebinding)
  bool pair = false;            // 2-CTA pairs (the handle's setting at creation)
  const int* bmap[P_KINDS] = {};
  int ncta = 0;
  float* ws = nullptr;
  int total[P_KINDS] = {};
  int total_tiles = 0;
  Fault* d_faults = nullptr;
  uint32_t* d_fbits = nullptr;  // one bit per tile with a fault
  int nfaults = 0;
};

// Static schedule of a group's tiles over `ncta` persistent CTAs: tiles in
// order (problems longest-K first, each in the kernel's raster), each given
// to the CTA with the least work so far (longest-processing-time greedy).
// A tile's cost is its k-blocks, but at least kEpilogueKb: with the
// accumulator double-buffered a CTA's time per tile is about the larger of
// its main loop and its epilogue.
static void tc_schedule(const std::vector<TcProblem>& probs, int ncta, std::vector<int4>& tiles,
                        std::vector<int>& cta_start, bool pair = false) {
  constexpr long long kEpilogueKb = 6;
  std::vector<std::vector<int4>> per(ncta);
  // min-heap of (load, cta)
  std::vector<std::pair<long long, int>> heap;
  for (int c = 0; c < ncta; ++c) heap.push_back({0, c});
  auto cmp = [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) { return a > b; };
  std::make_heap(heap.begin(), heap.end(), cmp);
  for (int pi = 0; pi < (int)probs.size(); ++pi) {
    const TcProblem& P = probs[pi];
    const long long cost = std::max<long long>(P.nkb, kEpilogueKb);
    // a pair's tile (the worker is a CTA pair) is two tile rows high
    const int rows = pair ? (P.tiles_m + 1) / 2 : P.tiles_m, gm = pair ? TC_GROUP_M / 2 : TC_GROUP_M;
    const int ntile = rows * P.tiles_n, per_group = gm * P.tiles_n;
    for (int id = 0; id < ntile; ++id) {
      const int first_m = (id / per_group) * gm;
      const int gsize = std::min(rows - first_m, gm);
      const int tm = first_m + (id % per_group) % gsize, tn = (id % per_group) / gsize;
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto& top = heap.back();
      per[top.second].push_back(make_int4(pi, tm, tn, P.nkb));
      top.first += cost;
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  tiles.clear();
  cta_start.assign(ncta + 1, 0);
  for (int c = 0; c < ncta; ++c) {
    cta_start[c] = (int)tiles.size();
    tiles.insert(tiles.end(), per[c].begin(), per[c].end());
  }
  cta_start[ncta] = (int)tiles.size();
}

// The order in which a group's problems are laid out and scheduled: longer
// K first (stable), so each CTA's static tile list ends on the cheap tiles.
template <class KOf>
static std::vector<int> longest_k_first(int count, KOf k_of) {
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return k_of(a) > k_of(c); });
  return order;
}

static void group_free(ftgemm_group* g) {
  if (!g) return;
  if (g->d_probs) cudaFree(g->d_probs);
  if (g->d_maps) cudaFree(g->d_maps);
  if (g->d_tiles) cudaFree(g->d_tiles);
  if (g->d_cta_start) cudaFree(g->d_cta_start);
  if (g->d_bmap) cudaFree(g->d_bmap);
  if (g->d_pos) cudaFree(g->d_pos);
  if (g->ws) cudaFree(g->ws);
  if (g->d_faults) cudaFree(g->d_faults);
  if (g->d_fbits) cudaFree(g->d_fbits);
  delete g;
}

static int group_enqueue(ftgemm_ctx* h, ftgemm_group* g);

extern "C" {

int ftgemm_group_create(ftgemm_handle_t h, int32_t count, const ftgemm_problem* pr, ftgemm_dtype dtype,
                        ftgemm_ft_level level, ftgemm_group_t* out) {
  if (!h || !pr || !out || count <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_create: bad argument");
  *out = nullptr;
  if (dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_group_create: bf16 or e4m3 operands only");
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_group_create: level OFF or TILE, not %d", (int)level);
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1, elem = dt == 0 ? 2 : 1;
  const bool abft = level == FTGEMM_FT_TILE;
  for (int i = 0; i < count; ++i) {
    const ftgemm_problem& q = pr[i];
    if (q.m <= 0 || q.n <= 0 || q.k <= 0 || q.m > INT32_MAX || q.n > INT32_MAX || q.k > INT32_MAX)
      FAIL(FTGEMM_ERR_ARG, "problem %d: sizes %lld x %lld x %lld", i, (long long)q.m, (long long)q.n,
           (long long)q.k);
    if (!q.A || !q.B || !q.C || q.lda < q.k || q.ldb < q.n || q.ldc < q.n)
      FAIL(FTGEMM_ERR_ARG, "problem %d: NULL operand or leading dimension too small", i);
    if (dt == 1 && !(q.scale_a > 0.f && q.scale_b > 0.f))
      FAIL(FTGEMM_ERR_ARG, "problem %d: e4m3 scales must be positive", i);
    char who[48];
    snprintf(who, sizeof(who), "problem %d", i);
    int rc = tc_check_operand_a(q.A, q.lda, elem, who);
    if (rc) return rc;
  }
  CK(cudaSetDevice(h->device));
  ftgemm_group* g = new ftgemm_group;
  g->h = h; g->dt = dt; g->abft = abft; g->count = count;
  const std::vector<int> order = longest_k_first(count, [&](int i) { return pr[i].k; });
  g->probs.resize(count);
  g->pos.resize(count);
  const float lam_u = (float)(h->lambda_tc[dt] * std::ldexp(1.0, -24));
  long long tiles = 0, blocks[P_KINDS] = {};
  size_t ws_floats = 0;
  std::vector<size_t> ws_at(count);
  for (int q = 0; q < count; ++q) {
    const ftgemm_problem& u = pr[order[q]];
    TcProblem& P = g->probs[q];
    tc_set_problem(P, dt, abft, (int)u.m, (int)u.n, (int)u.k, u.A, u.lda, u.B, u.ldb, u.C, u.ldc, u.alpha, u.beta,
                   dt == 1 ? u.scale_a * u.scale_b : 1.f, lam_u, h->mu);
    P.id = order[q];
    P.mlp = h->mlp_on ? h->mlp_theta : nullptr;
    P.mlp_scale = h->mlp_scale;
    g->pos[order[q]] = q;
    P.tile_start = (int)tiles;
    tiles += (long long)P.tiles_m * P.tiles_n;
    int nb[P_KINDS];
    tc_prep_blocks(P, dt, nb);
    for (int kd = 0; kd < P_KINDS; ++kd) {
      P.blk_start[kd] = (int)blocks[kd];
      blocks[kd] += nb[kd];
    }
    ws_at[q] = ws_floats;
    ws_floats += tc_layout(P, dt, abft, nullptr);
    if (tiles > INT32_MAX) { group_free(g); FAIL(FTGEMM_ERR_ARG, "ftgemm_group_create: too many tiles"); }
  }
  for (int kd = 0; kd < P_KINDS; ++kd) {
    if (blocks[kd] > INT32_MAX) { group_free(g); FAIL(FTGEMM_ERR_ARG, "ftgemm_group_create: group too large"); }
    g->total[kd] = (int)blocks[kd];
  }
  g->total_tiles = (int)tiles;
  cudaError_t e = cudaMalloc(&g->ws, ws_floats * sizeof(float));
  if (e != cudaSuccess) {
    group_free(g);
    FAIL(FTGEMM_ERR_CUDA, "ftgemm_group_create: %zu bytes of workspace: %s", ws_floats * sizeof(float),
         cudaGetErrorString(e));
  }
  std::vector<TcProbMaps> maps(count);
  for (int q = 0; q < count; ++q) {
    tc_layout(g->probs[q], dt, abft, g->ws + ws_at[q]);
    int rc = tc_make_maps(maps[q], g->probs[q], dt, abft, tc_use_pair(h, dt));
    if (rc) { group_free(g); return rc; }
  }
  g->pair = tc_use_pair(h, dt);
  {
    // workers: CTAs, or CTA pairs
    long long wtiles = 0;
    for (const TcProblem& P : g->probs) wtiles += (long long)(g->pair ? (P.tiles_m + 1) / 2 : P.tiles_m) * P.tiles_n;
    const int sms = h->num_sms > 0 ? h->num_sms : 148;
    g->ncta = (int)std::max<long long>(1, std::min<long long>(wtiles, g->pair ? sms / 2 : sms));
  }
  std::vector<int4> sched;
  std::vector<int> cta_start;
  tc_schedule(g->probs, g->ncta, sched, cta_start, g->pair);
  e = cudaMalloc(&g->d_probs, sizeof(TcProblem) * count);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_maps, sizeof(TcProbMaps) * count);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_tiles, sizeof(int4) * sched.size());
  if (e == cudaSuccess) e = cudaMalloc(&g->d_cta_start, sizeof(int) * cta_start.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_probs, g->probs.data(), sizeof(TcProblem) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_maps, maps.data(), sizeof(TcProbMaps) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_tiles, sched.data(), sizeof(int4) * sched.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_cta_start, cta_start.data(), sizeof(int) * cta_start.size(), cudaMemcpyHostToDevice);
  // the problem of every block of each encode launch (no search on the device)
  std::vector<int> bmap;
  size_t at[P_KINDS];
  for (int kd = 0; kd < P_KINDS; ++kd) {
    at[kd] = bmap.size();
    for (int q = 0; q < count; ++q) {
      int nb[P_KINDS];
      tc_prep_blocks(g->probs[q], dt, nb);
      bmap.insert(bmap.end(), (size_t)nb[kd], q);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->d_pos, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_pos, g->pos.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !bmap.empty()) e = cudaMalloc(&g->d_bmap, sizeof(int) * bmap.size());
  if (e == cudaSuccess && !bmap.empty())
    e = cudaMemcpy(g->d_bmap, bmap.data(), sizeof(int) * bmap.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    group_free(g);
    FAIL(FTGEMM_ERR_CUDA, "ftgemm_group_create: %s", cudaGetErrorString(e));
  }
  for (int kd = 0; kd < P_KINDS; ++kd) g->bmap[kd] = g->d_bmap ? g->d_bmap + at[kd] : nullptr;
  *out = g;
  return FTGEMM_OK;
}

int ftgemm_tc_tile(ftgemm_dtype dtype, ftgemm_ft_level level, int32_t* rows, int32_t* cols) {
  if (!rows || !cols) FAIL(FTGEMM_ERR_ARG, "ftgemm_tc_tile: NULL argument");
  if (dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_tc_tile: bf16 or e4m3 operands only");
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_tc_tile: level OFF or TILE, not %d", (int)level);
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1;
  *rows = tc_dm(dt, level == FTGEMM_FT_TILE);
  *cols = tc_dn(dt, level == FTGEMM_FT_TILE);
  return FTGEMM_OK;
}

int ftgemm_group_plan(int32_t count, const int64_t* m, const int64_t* n, const int64_t* k, ftgemm_dtype dtype,
                      ftgemm_ft_level level, int32_t ncta, int32_t* tiles, int32_t* cta_start,
                      int32_t* total_tiles) {
  if (count <= 0 || !m || !n || !k || ncta <= 0 || !total_tiles)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_group_plan: bad argument");
  if (dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_group_plan: bf16 or e4m3 operands only");
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_group_plan: level OFF or TILE, not %d", (int)level);
  for (int i = 0; i < count; ++i)
    if (m[i] <= 0 || n[i] <= 0 || k[i] <= 0 || m[i] > INT32_MAX || n[i] > INT32_MAX || k[i] > INT32_MAX)
      FAIL(FTGEMM_ERR_ARG, "problem %d: sizes %lld x %lld x %lld", i, (long long)m[i], (long long)n[i],
           (long long)k[i]);
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1;
  const bool abft = level == FTGEMM_FT_TILE;
  // the same problem order, tile grid and schedule as ftgemm_group_create
  const std::vector<int> order = longest_k_first(count, [&](int i) { return k[i]; });
  std::vector<TcProblem> probs(count);
  long long total = 0;
  for (int q = 0; q < count; ++q) {
    const int i = order[q];
    tc_set_problem(probs[q], dt, abft, (int)m[i], (int)n[i], (int)k[i], nullptr, k[i], nullptr, n[i], nullptr,
                   n[i], 1.0, 0.0, 1.f, 0.f, 0.0);
    total += (long long)probs[q].tiles_m * probs[q].tiles_n;
    if (total > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_plan: too many tiles");
  }
  *total_tiles = (int32_t)total;
  if (!tiles && !cta_start) return FTGEMM_OK;  // size query
  std::vector<int4> sched;
  std::vector<int> start;
  tc_schedule(probs, ncta, sched, start);
  if (tiles)
    for (size_t j = 0; j < sched.size(); ++j) {
      tiles[4 * j + 0] = order[sched[j].x];  // the caller's problem index
      tiles[4 * j + 1] = sched[j].y;
      tiles[4 * j + 2] = sched[j].z;
      tiles[4 * j + 3] = sched[j].w;
    }
  if (cta_start)
    for (int c = 0; c <= ncta; ++c) cta_start[c] = start[c];
  return FTGEMM_OK;
}

int ftgemm_group_tiles(ftgemm_group_t g, int32_t* tiles_m, int32_t* tiles_n) {
  if (!g || !tiles_m || !tiles_n) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_tiles: NULL argument");
  for (int i = 0; i < g->count; ++i) {
    const TcProblem& P = g->probs[g->pos[i]];
    tiles_m[i] = P.tiles_m;
    tiles_n[i] = P.tiles_n;
  }
  return FTGEMM_OK;
}

int ftgemm_group_set_faults(ftgemm_group_t g, const int32_t* problem, const ftgemm_inject_spec* inject) {
  if (!g) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_set_faults: NULL group");
  const int nf = inject ? inject->n : 0;
  if (nf < 0) FAIL(FTGEMM_ERR_ARG, "inject->n < 0");
  if (nf > 0 && (!problem || !inject->tile_m || !inject->tile_n || !inject->kstep || !inject->row || !inject->col ||
                 !inject->delta))
    FAIL(FTGEMM_ERR_ARG, "ftgemm_group_set_faults: NULL array");
  std::vector<Fault> fv(nf);
  const int dm = tc_dm(g->dt, g->abft), dn = tc_dn(g->dt, g->abft);
  for (int i = 0; i < nf; ++i) {
    const int pi = problem[i];
    if (pi < 0 || pi >= g->count) FAIL(FTGEMM_ERR_ARG, "inject[%d]: problem %d outside [0,%d)", i, pi, g->count);
    const TcProblem& P = g->probs[g->pos[pi]];
    const int tm = inject->tile_m[i], tn = inject->tile_n[i], r = inject->row[i], c = inject->col[i];
    const int tg = inject->target ? inject->target[i] : 0;
    int ks = inject->kstep[i];
    if (tm < 0 || tm >= P.tiles_m || tn < 0 || tn >= P.tiles_n)
      FAIL(FTGEMM_ERR_ARG, "inject[%d]: tile (%d,%d) outside problem %d's %dx%d grid", i, tm, tn, pi, P.tiles_m,
           P.tiles_n);
    if (ks == -1) ks = P.nkb - 1;
    if (ks < 0 || ks >= P.nkb) FAIL(FTGEMM_ERR_ARG, "inject[%d]: k-step %d outside [0,%d)", i, ks, P.nkb);
    const int rows = std::min(dm, P.M - tm * dm), cols = std::min(dn, P.N - tn * dn);
    if (r < 0 || r >= rows || c < 0 || c >= cols)
      FAIL(FTGEMM_ERR_ARG, "inject[%d]: element (%d,%d) outside tile (%d x %d)", i, r, c, rows, cols);
    if (tg < 0 || tg > 2) FAIL(FTGEMM_ERR_ARG, "inject[%d]: target %d", i, tg);
    if (!g->abft && tg != 0) FAIL(FTGEMM_ERR_ARG, "inject[%d]: no checksums at level OFF", i);
    fv[i] = Fault{P.tile_start + tm * P.tiles_n + tn, ks, r, c, tg, inject->delta[i]};
  }
  std::stable_sort(fv.begin(), fv.end(), [](const Fault& a, const Fault& b) {
    return a.tile != b.tile ? a.tile < b.tile : a.kstep < b.kstep;
  });
  CK(cudaSetDevice(g->h->device));
  CK(cudaStreamSynchronize(g->h->stream));  // a launch in flight may read the old table
  if (g->d_faults) cudaFree(g->d_faults);
  if (g->d_fbits) cudaFree(g->d_fbits);
  g->d_faults = nullptr;
  g->d_fbits = nullptr;
  g->nfaults = 0;
  if (nf > 0) {
    std::vector<uint32_t> bits(((size_t)g->total_tiles + 31) / 32, 0u);
    for (const Fault& f : fv) bits[f.tile >> 5] |= 1u << (f.tile & 31);
    CK(cudaMalloc(&g->d_faults, sizeof(Fault) * nf));
    CK(cudaMalloc(&g->d_fbits, sizeof(uint32_t) * bits.size()));
    CK(cudaMemcpy(g->d_faults, fv.data(), sizeof(Fault) * nf, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g->d_fbits, bits.data(), sizeof(uint32_t) * bits.size(), cudaMemcpyHostToDevice));
  }
  g->nfaults = nf;
  return FTGEMM_OK;
}

int ftgemm_grouped_gemm(ftgemm_handle_t h, ftgemm_group_t g) {
  if (!h || !g) FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm: NULL argument");
  if (g->h != h) FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm: the group was created on another handle");
  CK(cudaSetDevice(h->device));
  return group_enqueue(h, g);
}

int ftgemm_grouped_gemm_dev(ftgemm_handle_t h, ftgemm_group_t g, int32_t count, const ftgemm_problem* problems) {
  if (!h || !g || !problems) FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm_dev: NULL argument");
  if (g->h != h) FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm_dev: the group was created on another handle");
  if (count != g->count)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm_dev: %d problems, the group has %d", (int)count, g->count);
  if ((uintptr_t)problems % alignof(ftgemm_problem))
    FAIL(FTGEMM_ERR_ARG, "ftgemm_grouped_gemm_dev: the problem array is not %zu-byte aligned",
         alignof(ftgemm_problem));
  if (h->sink_lam && g->abft && g->total_tiles > h->sink_cap)
    FAIL(FTGEMM_ERR_ARG, "residual sink holds %lld tiles, the group has %d", (long long)h->sink_cap, g->total_tiles);
  CK(cudaSetDevice(h->device));
  CK(launch_tc_bind(g->d_probs, g->d_maps, g->d_pos, problems, g->count, g->dt, h->rep, h->stream));
  h->launches += 1;
  return group_enqueue(h, g);
}

int ftgemm_group_bind_rule(const ftgemm_problem* created, const ftgemm_problem* bound, ftgemm_dtype dtype,
                           ftgemm_ft_level level) {
  if (!created || !bound) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_bind_rule: NULL argument");
  if ((dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3) || (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE))
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_group_bind_rule: dtype %d, level %d", (int)dtype, (int)level);
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1;
  const int b_mn = tc_b_in_place(dt, level == FTGEMM_FT_TILE, created->B, created->ldb);
  return tc_bind_rule(created->m, created->n, created->k, created->lda, created->ldb, b_mn, dt, *bound);
}

}  // extern "C"

// The encode pass and the persistent launch of a group, on the handle's stream.
static int group_enqueue(ftgemm_ctx* h, ftgemm_group* g) {
  if (h->sink_lam && g->abft && g->total_tiles > h->sink_cap)
    FAIL(FTGEMM_ERR_ARG, "residual sink holds %lld tiles, the group has %d", (long long)h->sink_cap, g->total_tiles);
  TcBatch b;
  memset(&b, 0, sizeof(b));
  b.table = g->d_probs;
  b.tile_list = g->d_tiles;
  b.cta_start = g->d_cta_start;
  b.nprob = g->count;
  b.total_tiles = g->total_tiles;
  int launches = 0;
  CK(launch_tc_prep(g->dt, g->abft, b, g->total, g->bmap, &launches, h->stream));
  TcMapsBatch mb;
  memset(&mb, 0, sizeof(mb));
  mb.table = g->d_maps;
  TcRun run{g->nfaults > 0 ? g->d_faults : nullptr, g->nfaults, g->d_fbits, h->rep, h->recs,
            g->abft ? h->sink_lam : nullptr, g->abft ? h->sink_x : nullptr};
  const int grid = g->pair ? 2 * g->ncta : g->ncta;  // the schedule was built for this many workers
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(h->stream, &cs));
  const bool timed = h->timing && cs == cudaStreamCaptureStatusNone;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (timed) {
    int rc = take_events(h, &ev);
    if (rc) return rc;
    CK(cudaEventRecord(ev.first, h->stream));
  }
  CK(launch_tc_gemm(g->dt, g->abft, g->pair, b, mb, run, grid, h->stream));
  ++launches;
  if (timed) {
    CK(cudaEventRecord(ev.second, h->stream));
    h->pending.push_back(ev);
  }
  h->launches += launches;
  return FTGEMM_OK;
}

extern "C" {

int ftgemm_group_destroy(ftgemm_group_t g) {
  if (!g) return FTGEMM_OK;
  cudaSetDevice(g->h->device);
  cudaStreamSynchronize(g->h->stream);
  group_free(g);
  return FTGEMM_OK;
}

int ftgemm_set_tc_pair(ftgemm_handle_t h, int mode) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_tc_pair: NULL handle");
  if (mode < -1 || mode > 1) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_tc_pair: mode %d (1, 0 or -1)", mode);
  h->tc_pair = mode;
  return FTGEMM_OK;
}

int ftgemm_enable_timing(ftgemm_handle_t h, int enable) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_enable_timing: NULL handle");
  h->timing = enable != 0;
  return FTGEMM_OK;
}

int ftgemm_get_stats(ftgemm_handle_t h, ftgemm_stats* out, int reset) {
  if (!h || !out) FAIL(FTGEMM_ERR_ARG, "ftgemm_get_stats: NULL argument");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  int rc = drain_events(h);
  if (rc) return rc;
  out->launches = h->launches;
  out->timed_launches = h->timed;
  out->kernel_ms = h->kernel_ms;
  if (reset) {
    h->launches = 0;
    h->timed = 0;
    h->kernel_ms = 0.0;
  }
  return FTGEMM_OK;
}

const char* ftgemm_status_string(int status) {
  switch (status) {
    case FTGEMM_OK: return "ok";
    case FTGEMM_ERR_ARG: return "invalid argument";
    case FTGEMM_ERR_UNSUPPORTED: return "unsupported dtype / level / schedule";
    case FTGEMM_ERR_ALIGN: return "misaligned pointer or stride";
    case FTGEMM_ERR_CUDA: return "CUDA error";
    case FTGEMM_ERR_TIMEOUT: return "device wait timed out";
    case FTGEMM_ERR_UNRECOVERED: return "every offline attempt detected a fault";
    default: return "unknown status";
  }
}

const char* ftgemm_last_error(void) { return g_last_error.c_str(); }

int ftgemm_create(ftgemm_handle_t* handle, int device, void* cuda_stream) {
  if (!handle) FAIL(FTGEMM_ERR_ARG, "ftgemm_create: handle is NULL");
  *handle = nullptr;
  int count = 0;
  CK(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) FAIL(FTGEMM_ERR_ARG, "ftgemm_create: no device %d", device);
  CK(cudaSetDevice(device));
  ftgemm_ctx* h = new ftgemm_ctx();
  h->device = device;
  h->stream = (cudaStream_t)cuda_stream;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) h->num_sms = prop.multiProcessorCount;
  DevReport r{};
  r.capacity = h->rep_cap;
  cudaError_t e = cudaMalloc(&h->rep, sizeof(DevReport));
  if (e == cudaSuccess) e = cudaMalloc(&h->recs, sizeof(ftgemm_fault_record) * h->rep_cap);
  if (e == cudaSuccess) e = cudaMemcpy(h->rep, &r, sizeof(r), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->faults_free, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ftgemm_destroy(h);  // releases whatever was allocated
    FAIL(FTGEMM_ERR_CUDA, "ftgemm_create: cannot set up the report ring: %s", cudaGetErrorString(e));
  }
  *handle = h;
  return FTGEMM_OK;
}

int ftgemm_destroy(ftgemm_handle_t h) {
  if (!h) return FTGEMM_OK;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->ws) cudaFree(h->ws);
  if (h->rep) cudaFree(h->rep);
  if (h->recs) cudaFree(h->recs);
  if (h->zimag) cudaFree(h->zimag);
  if (h->d_faults) cudaFree(h->d_faults);
  if (h->h_faults) cudaFreeHost(h->h_faults);
  if (h->faults_free) cudaEventDestroy(h->faults_free);
  if (h->qscratch) cudaFree(h->qscratch);
  if (h->d_fbits) cudaFree(h->d_fbits);
  if (h->ws2) cudaFree(h->ws2);
  if (h->mlp_theta) cudaFree(h->mlp_theta);
  if (h->mlp_ws) cudaFree(h->mlp_ws);
  for (auto& e : h->pending) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  for (auto& e : h->pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  delete h;
  return FTGEMM_OK;
}

int ftgemm_set_stream(ftgemm_handle_t h, void* s) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_stream: NULL handle");
  h->stream = (cudaStream_t)s;
  return FTGEMM_OK;
}

int ftgemm_set_schedule(ftgemm_handle_t h, const ftgemm_schedule* s) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_schedule: NULL handle");
  if (!s) { h->has_sched = false; return FTGEMM_OK; }
  if (s->cadence < 0 || s->split_k < 1) FAIL(FTGEMM_ERR_ARG, "cadence must be >= 0 and split_k >= 1");
  if (!find_simt(*s))
    FAIL(FTGEMM_ERR_UNSUPPORTED, "tile tuple (%d,%d,%d,%d,%d,%d,%d) is not a compiled kernel",
         s->m_tb, s->n_tb, s->k_tb, s->m_w, s->n_w, s->m_t, s->n_t);
  h->sched = *s;
  h->has_sched = true;
  return FTGEMM_OK;
}

int ftgemm_get_schedule(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, ftgemm_dtype dtype,
                        ftgemm_ft_level level, ftgemm_schedule* out) {
  if (!h || !out || m <= 0 || n <= 0 || k <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_get_schedule: bad argument");
  if (dtype != FTGEMM_F32) FAIL(FTGEMM_ERR_UNSUPPORTED, "only FTGEMM_F32 has a SIMT schedule");
  ftgemm_ft_level run_level;
  choose_schedule(h, m, n, k, level, out, &run_level);
  return FTGEMM_OK;
}

int ftgemm_set_threshold(ftgemm_handle_t h, int mode, double lambda, const float* w, size_t nw) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_threshold: NULL handle");
  if (mode == 0) {
    if (lambda > 0) h->lambda = lambda;
    h->mlp_on = false;
    return FTGEMM_OK;
  }
  if (mode != 1) FAIL(FTGEMM_ERR_UNSUPPORTED, "threshold mode %d is not available", mode);
  if (!w || nw != (size_t)FTGEMM_MLP_PARAMS)
    FAIL(FTGEMM_ERR_ARG, "learned threshold: %d network parameters expected, got %zu", FTGEMM_MLP_PARAMS, nw);
  if (!(lambda > 0)) FAIL(FTGEMM_ERR_ARG, "learned threshold: the scale must be positive");
  for (size_t i = 0; i < nw; ++i)
    if (!std::isfinite(w[i])) FAIL(FTGEMM_ERR_ARG, "learned threshold: parameter %zu is not finite", i);
  CK(cudaSetDevice(h->device));
  if (!h->mlp_theta) CK(cudaMalloc(&h->mlp_theta, sizeof(float) * FTGEMM_MLP_PARAMS));
  CK(cudaStreamSynchronize(h->stream));  // a launch in flight may read the old parameters
  CK(cudaMemcpy(h->mlp_theta, w, sizeof(float) * FTGEMM_MLP_PARAMS, cudaMemcpyHostToDevice));
  h->mlp_on = true;
  h->mlp_scale = (float)lambda;
  return FTGEMM_OK;
}

int ftgemm_set_residual_sink(ftgemm_handle_t h, float* lam_needed, float* features, int64_t capacity) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_residual_sink: NULL handle");
  if (!lam_needed) {
    h->sink_lam = nullptr;
    h->sink_x = nullptr;
    h->sink_cap = 0;
    return FTGEMM_OK;
  }
  if (!features || capacity <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_residual_sink: bad argument");
  h->sink_lam = lam_needed;
  h->sink_x = features;
  h->sink_cap = capacity;
  return FTGEMM_OK;
}

static int ensure_mlp_ws(ftgemm_ctx* h, size_t floats) {
  if (floats <= h->mlp_ws_floats) return FTGEMM_OK;
  CK(cudaStreamSynchronize(h->stream));  // earlier launches may still read it
  if (h->mlp_ws) CK(cudaFree(h->mlp_ws));
  h->mlp_ws = nullptr;
  h->mlp_ws_floats = 0;
  CK(cudaMalloc(&h->mlp_ws, floats * sizeof(float)));
  h->mlp_ws_floats = floats;
  return FTGEMM_OK;
}

int ftgemm_mlp_forward(ftgemm_handle_t h, int64_t n, const float* X, const float* theta, float* y) {
  if (!h || !X || !theta || !y || n <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_mlp_forward: bad argument");
  CK(cudaSetDevice(h->device));
  CK(launch_mlp_forward(X, n, theta, y, h->stream));
  ++h->launches;
  return FTGEMM_OK;
}

int ftgemm_mlp_grad(ftgemm_handle_t h, int64_t n, const float* X, const float* t, const float* theta, float* grad,
                    float* loss) {
  if (!h || !X || !t || !theta || !grad || n <= 0 || n > INT32_MAX)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_mlp_grad: bad argument");
  CK(cudaSetDevice(h->device));
  const int nblk = mlp_grad_blocks(n);
  const size_t slot = FTGEMM_MLP_PARAMS + 1;
  int rc = ensure_mlp_ws(h, (size_t)nblk * slot + 1);
  if (rc) return rc;
  float* part = h->mlp_ws;
  float* dloss = h->mlp_ws + (size_t)nblk * slot;
  const float inv_n = (float)(1.0 / (double)n);
  CK(launch_mlp_grad(X, t, 0, (int)n, theta, inv_n, part, nblk, h->stream));
  CK(launch_mlp_reduce(part, nblk, grad, nullptr, nullptr, nullptr, 0, 0.f, inv_n, dloss, h->stream));
  h->launches += 2;
  if (loss) {
    CK(cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return FTGEMM_OK;
}

int ftgemm_mlp_train(ftgemm_handle_t h, int64_t n, const float* X, const float* t, int32_t epochs, int32_t batch,
                     float lr, float* theta, float* losses) {
  if (!h || !X || !t || !theta || n <= 0 || n > INT32_MAX || epochs <= 0 || batch <= 0 || !(lr > 0.f))
    FAIL(FTGEMM_ERR_ARG, "ftgemm_mlp_train: bad argument");
  CK(cudaSetDevice(h->device));
  const long long steps_per_epoch = (n + batch - 1) / batch;
  const long long steps = steps_per_epoch * epochs;
  const int nblk = mlp_grad_blocks(std::min<long long>(batch, n));
  const size_t slot = FTGEMM_MLP_PARAMS + 1;
  int rc = ensure_mlp_ws(h, (size_t)nblk * slot + 2 * (size_t)FTGEMM_MLP_PARAMS + (size_t)steps);
  if (rc) return rc;
  float* part = h->mlp_ws;
  float* m = part + (size_t)nblk * slot;
  float* v = m + FTGEMM_MLP_PARAMS;
  float* step_loss = v + FTGEMM_MLP_PARAMS;
  CK(cudaMemsetAsync(m, 0, sizeof(float) * 2 * FTGEMM_MLP_PARAMS, h->stream));
  long long step = 0;
  for (int e = 0; e < epochs; ++e) {
    for (long long s0 = 0; s0 < n; s0 += batch) {
      const int nb = (int)std::min<long long>(batch, n - s0);
      const float inv_n = (float)(1.0 / (double)nb);
      CK(launch_mlp_grad(X, t, s0, nb, theta, inv_n, part, nblk, h->stream));
      ++step;
      CK(launch_mlp_reduce(part, nblk, nullptr, theta, m, v, (int)step, lr, inv_n, step_loss + (step - 1),
                           h->stream));
    }
  }
  h->launches += 2 * steps;
  if (losses) {
    std::vector<float> sl((size_t)steps);
    CK(cudaMemcpyAsync(sl.data(), step_loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int e = 0; e < epochs; ++e) {
      double acc = 0.0;
      for (long long q = 0; q < steps_per_epoch; ++q) acc += sl[(size_t)(e * steps_per_epoch + q)];
      losses[e] = (float)(acc / (double)steps_per_epoch);
    }
  }
  return FTGEMM_OK;
}


int ftgemm_set_fp8_scales(ftgemm_handle_t h, float sa, float sb) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_fp8_scales: NULL handle");
  if (!(sa > 0.f) || !(sb > 0.f)) FAIL(FTGEMM_ERR_ARG, "fp8 scales must be positive");
  h->fp8_sa = sa;
  h->fp8_sb = sb;
  return FTGEMM_OK;
}

int ftgemm_quantize(ftgemm_handle_t h, int64_t n, const float* x, void* y, ftgemm_dtype dtype, float* scale_out) {
  if (!h || !x || !y || n <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_quantize: bad argument");
  if (dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3) FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_quantize: dtype %d", (int)dtype);
  CK(cudaSetDevice(h->device));
  if (!h->qscratch) CK(cudaMalloc(&h->qscratch, 2 * sizeof(float)));
  int launches = 0;
  CK(launch_quantize(dtype == FTGEMM_BF16 ? 0 : 1, x, n, y, reinterpret_cast<unsigned int*>(h->qscratch),
                     h->qscratch + 1, &launches, h->stream));
  h->launches += launches;
  if (scale_out) {
    if (dtype == FTGEMM_BF16) {
      *scale_out = 1.f;
    } else {
      CK(cudaMemcpyAsync(scale_out, h->qscratch + 1, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
  }
  return FTGEMM_OK;
}

int ftgemm_report_fetch(ftgemm_handle_t h, ftgemm_report* out) {
  if (!h || !out) FAIL(FTGEMM_ERR_ARG, "ftgemm_report_fetch: NULL argument");
  CK(cudaSetDevice(h->device));
  DevReport r;
  CK(cudaMemcpyAsync(&r, h->rep, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int n = std::min(r.n_records, h->rep_cap);
  std::vector<ftgemm_fault_record> v(n);
  if (n > 0) {
    CK(cudaMemcpyAsync(v.data(), h->recs, sizeof(ftgemm_fault_record) * n, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  std::sort(v.begin(), v.end(), [](const ftgemm_fault_record& a, const ftgemm_fault_record& b) {
    if (a.problem != b.problem) return a.problem < b.problem;
    if (a.tile_m != b.tile_m) return a.tile_m < b.tile_m;
    if (a.tile_n != b.tile_n) return a.tile_n < b.tile_n;
    if (a.kstep != b.kstep) return a.kstep < b.kstep;
    if (a.row != b.row) return a.row < b.row;
    if (a.col != b.col) return a.col < b.col;
    return a.kind < b.kind;
  });
  out->detected = (int64_t)r.detected;
  out->corrected = (int64_t)r.corrected;
  out->uncorrectable = (int64_t)r.uncorrectable;
  out->checksum_only = (int64_t)r.checksum_only;
  out->n_records = r.n_records;
  const int cap = std::max(0, out->capacity);
  const int w = std::min(cap, n);
  if (w > 0 && out->records) memcpy(out->records, v.data(), sizeof(ftgemm_fault_record) * w);
  out->overflow = (r.n_records > cap || r.n_records > h->rep_cap) ? 1 : 0;
  int rc = clear_report(h);
  if (rc) return rc;
  if (r.timeouts > 0) FAIL(FTGEMM_ERR_TIMEOUT, "%d bounded device waits gave up", r.timeouts);
  if (r.bind_errors > 0)
    FAIL(FTGEMM_ERR_ARG, "%d device-array entries broke a rebinding rule; their problems were skipped",
         r.bind_errors);
  return FTGEMM_OK;
}

int ftgemm_encode(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                  const float* B, int64_t ldb, int32_t m_u, int32_t n_u, float* V, float* W,
                  float* nA, float* nB) {
  if (!h || !A || !B || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || m_u < 2 || n_u < 2 ||
      m_u > 1024 || n_u > 1024 || (m_u & (m_u - 1)) || (n_u & (n_u - 1)) || m > INT32_MAX ||
      n > INT32_MAX || k > INT32_MAX)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_encode: bad argument (block sizes must be powers of two in [2,1024])");
  CK(cudaSetDevice(h->device));
  const int M = (int)m, N = (int)n, K = (int)k;
  // A is read once in place (no transpose); B is k-major already
  const size_t nScr = (size_t)std::max<long long>((long long)((K + 255) / 256) * M, kmajor_scratch_floats(K, N));
  int rc = ensure_ws(h, align64(nScr));
  if (rc) return rc;
  int launches = 0;
  if (V || nA) CK(launch_encode_rowmajor(A, lda, M, K, m_u, V, K, nA, h->ws, &launches, h->stream));
  if (W || nB)
    CK(launch_encode_kmajor(B, ldb, K, N, n_u, W, K, nB, h->ws, &launches, h->stream));
  h->launches += launches;
  return FTGEMM_OK;
}

int ftgemm_gemm(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, double alpha, const void* A,
                int64_t lda, const void* B, int64_t ldb, double beta, float* C, int64_t ldc,
                ftgemm_dtype dtype, ftgemm_ft_level level, const ftgemm_inject_spec* inject,
                ftgemm_report* report) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm: NULL handle");
  if (!A || !B || !C) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm: NULL matrix pointer");
  if (m <= 0 || n <= 0 || k <= 0) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm: m, n, k must be positive");
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm: size too large");
  if (lda < k || ldb < n || ldc < n) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm: leading dimension too small");
  if (dtype == FTGEMM_BF16 || dtype == FTGEMM_E4M3)
    return tc_gemm(h, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype, level, inject, report);
  if (dtype != FTGEMM_F32) FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: dtype %d", (int)dtype);
  if (level == FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: level TILE needs a tensor-core dtype");
  if (level < FTGEMM_FT_OFF || level > FTGEMM_FT_AUTO)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: level %d", (int)level);
  CK(cudaSetDevice(h->device));
  ftgemm_schedule s;
  ftgemm_ft_level run_level;
  choose_schedule(h, m, n, k, level, &s, &run_level);
  return simt_gemm(h, m, n, k, alpha, (const float*)A, lda, (const float*)B, ldb, beta, C, ldc, run_level, s,
                   inject, report);
}

}  // extern "C"

// The SIMT path of ftgemm_gemm with an explicit schedule and level.
// At_given (OFF only): A already k-major (K x M, row stride ldat, 16-byte
// aligned rows); the transpose pass is skipped.
// detect (level BLOCK, the 128 x 128 x 32 tuple with 16 x 8 fragments): the
// detector of the offline scheme -- column checksums only, one verification
// per split, detections reported and nothing corrected.
static int simt_gemm(ftgemm_ctx* h, int64_t m, int64_t n, int64_t k, double alpha, const float* A, int64_t lda,
                     const float* B, int64_t ldb, double beta, float* C, int64_t ldc, ftgemm_ft_level level,
                     const ftgemm_schedule& s, const ftgemm_inject_spec* inject, ftgemm_report* report,
                     const float* At_given, int64_t ldat, bool detect) {
  if (At_given && level != FTGEMM_FT_OFF) FAIL(FTGEMM_ERR_ARG, "internal: k-major A needs level OFF");
  const SimtConfig* cfg = find_simt(s);
  if (!cfg) FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: schedule is not a compiled kernel");
  if (detect && (level != FTGEMM_FT_BLOCK || cfg->launch != simt_launch_wide32))
    FAIL(FTGEMM_ERR_ARG, "internal: the detector runs the 128 x 128 x 32 tuple at block level");

  const int M = (int)m, N = (int)n, K = (int)k;
  const int ksteps = (K + s.k_tb - 1) / s.k_tb;
  int split = std::max(1, std::min(s.split_k, ksteps));
  const int ks_per_split = (ksteps + split - 1) / split;
  split = (ksteps + ks_per_split - 1) / ks_per_split;
  const int cadence = (s.cadence > 0 && !detect) ? s.cadence : ks_per_split;
  const int tiles_m = (M + s.m_tb - 1) / s.m_tb, tiles_n = (N + s.n_tb - 1) / s.n_tb;

  const float* Af = A;
  const float* Bf = B;
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };

  // ---- faults: validate, resolve, sort, upload -----------------------------
  int nf = 0;
  {
    int rc = upload_faults(h, inject, s, M, N, ksteps, tiles_m, tiles_n, level, &nf);
    if (rc) return rc;
  }

  if (report) {
    int rc = clear_report(h);
    if (rc) return rc;
  }

  // ---- workspace: k-major operands, encoded vectors, norms, partials -----
  const bool abft = level != FTGEMM_FT_OFF;
  int m_u = 1, n_u = 1;
  bool need_vw = false;
  if (level == FTGEMM_FT_WARP) { m_u = s.m_w; n_u = s.n_w; need_vw = true; }
  if (level == FTGEMM_FT_BLOCK) { m_u = s.m_tb; n_u = s.n_tb; need_vw = true; }
  const int NV = level == FTGEMM_FT_WARP ? s.m_tb / s.m_w : 1;
  const int NW = level == FTGEMM_FT_WARP ? s.n_tb / s.n_w : 1;
  const long long ldt = At_given ? ldat : (M + 3) / 4 * 4;  // A^T row stride (16-byte multiple)
  const long long ldv = (K + 3) / 4 * 4;  // encoded-vector row stride
  const bool b_ok = (ldb % 4 == 0) && al16(B);
  const long long ldbp = b_ok ? ldb : (N + 3) / 4 * 4;
  const int nvb = (M + m_u - 1) / m_u, nwb = (N + n_u - 1) / n_u;
  const size_t nAt = At_given ? 0 : (size_t)K * ldt;
  const size_t nBp = b_ok ? 0 : (size_t)K * ldbp;
  const size_t nV = need_vw ? (size_t)nvb * ldv : 0;
  const size_t nW = (need_vw && !detect) ? (size_t)nwb * ldv : 0;  // the detector keeps no B e
  const size_t nNa = abft ? (size_t)M : 0, nNb = abft ? (size_t)N : 0;
  const size_t nScr = abft ? (size_t)std::max<long long>((long long)((K + 31) / 32) * M,
                                                         kmajor_scratch_floats(K, N))
                           : 0;
  const size_t nPart = split > 1 ? (size_t)split * M * N : 0;
  // learned threshold and residual sink (block level): block coherences
  const bool learned = level == FTGEMM_FT_BLOCK && h->mlp_on && !detect;
  const bool sink = level == FTGEMM_FT_BLOCK && h->sink_lam != nullptr && !detect;
  if (sink && (long long)tiles_m * tiles_n > h->sink_cap)
    FAIL(FTGEMM_ERR_ARG, "residual sink: %lld tiles, capacity %lld", (long long)tiles_m * tiles_n,
         (long long)h->sink_cap);
  const size_t nCo = (learned || sink) ? (size_t)(tiles_m + tiles_n) : 0;
  const size_t oAt = 0, oBp = align64(oAt + nAt), oV = align64(oBp + nBp), oW = align64(oV + nV),
               oNa = align64(oW + nW), oNb = align64(oNa + nNa), oScr = align64(oNb + nNb),
               oPart = align64(oScr + nScr), oCo = align64(oPart + nPart), total = align64(oCo + nCo);
  {
    int rc = ensure_ws(h, total);
    if (rc) return rc;
  }
  float* ws = h->ws;
  int launches = 0;
  // A^T, with the A side of the encoding (block sums, row norms) in the same pass
  const float* At = At_given ? At_given : ws + oAt;
  if (!At_given)
    CK(launch_transpose_encode(Af, lda, M, K, ws + oAt, ldt, m_u, need_vw ? ws + oV : nullptr, ldv,
                               abft ? ws + oNa : nullptr, ws + oScr, &launches, h->stream));
  const float* Bk = Bf;
  if (!b_ok) {
    CK(launch_copy_pad(Bf, ldb, K, N, ws + oBp, ldbp, h->stream));
    ++launches;
    Bk = ws + oBp;
  }
  if (abft) {
    CK(launch_encode_kmajor(Bk, ldbp, K, N, (need_vw && !detect) ? n_u : 2,
                            (need_vw && !detect) ? ws + oW : nullptr, ldv, ws + oNb, ws + oScr, &launches,
                            h->stream));
  }
  if (learned || sink) {
    CK(launch_block_coherence(ws + oV, ws + oW, ldv, K, ws + oNa, ws + oNb, M, N, m_u, n_u, ws + oCo,
                              ws + oCo + tiles_m, h->stream));
    ++launches;
  }
  if (sink) CK(cudaMemsetAsync(h->sink_lam, 0, sizeof(float) * (size_t)tiles_m * tiles_n, h->stream));

  SimtMaps maps;
  {
    int rc = make_map_2d(&maps.A, At, M, K, ldt, s.m_tb, s.k_tb);
    if (!rc) rc = make_map_2d(&maps.B, Bk, N, K, ldbp, s.n_tb, s.k_tb);
    if (!rc && need_vw) rc = make_map_2d(&maps.V, ws + oV, K, nvb, ldv, s.k_tb, NV);
    if (!rc && need_vw && !detect) rc = make_map_2d(&maps.W, ws + oW, K, nwb, ldv, s.k_tb, NW);
    if (rc) return rc;
    if (!need_vw) { maps.V = maps.A; maps.W = maps.A; }
    if (detect) maps.W = maps.V;  // not read
  }

  SimtParams p;
  p.M = M; p.N = N; p.K = K;
  p.C = C; p.ldc = ldc;
  p.c_vec = (ldc % 4 == 0) && al16(C);
  p.alpha = (float)alpha; p.beta = (float)beta;
  p.nA = abft ? ws + oNa : nullptr;
  p.nB = abft ? ws + oNb : nullptr;
  p.lam_u = (float)(h->lambda * std::ldexp(1.0, -24));
  p.mu_u = (float)(h->mu * std::ldexp(1.0, -24));
  p.cadence = std::max(1, cadence);
  p.ksteps = ksteps;
  p.ks_per_split = ks_per_split;
  p.partial = split > 1 ? ws + oPart : nullptr;
  p.faults = nf > 0 ? h->d_faults : nullptr;
  p.nfaults = nf;
  p.rep = h->rep;
  p.recs = h->recs;
  p.tiles_m = tiles_m;
  p.tiles_n = tiles_n;
  p.group_m = std::min(tiles_m, 16);
  p.mlp = learned ? h->mlp_theta : nullptr;
  p.mlp_scale = h->mlp_scale;
  p.coA = (learned || sink) ? ws + oCo : nullptr;
  p.coB = (learned || sink) ? ws + oCo + tiles_m : nullptr;
  p.sink_lam = sink ? h->sink_lam : nullptr;
  p.sink_x = sink ? h->sink_x : nullptr;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (h->timing) {
    int rc = take_events(h, &ev);
    if (rc) return rc;
    CK(cudaEventRecord(ev.first, h->stream));
  }
  if (detect) CK(simt_launch_wide32_detect(maps, p, split, h->stream));
  else CK(cfg->launch((int)level, maps, p, split, h->stream));
  ++launches;
  if (h->timing) {
    CK(cudaEventRecord(ev.second, h->stream));
    h->pending.push_back(ev);
  }
  if (split > 1) {
    CK(launch_splitk_reduce(ws + oPart, split, M, N, (float)alpha, (float)beta, C, ldc, h->stream));
    ++launches;
  }
  h->launches += launches;

  if (report) return ftgemm_report_fetch(h, report);
  return FTGEMM_OK;
}

// ---- autotuner (Section 3.2's parameter selection, done by measurement) ----

int ftgemm_autotune(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                    const float* B, int64_t ldb, float* C, int64_t ldc, ftgemm_ft_level level, int32_t reps,
                    ftgemm_schedule* out, ftgemm_ft_level* level_out) {
  if (!h || !A || !B || !C || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || ldc < n)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_autotune: bad argument");
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "ftgemm_autotune: size too large");
  if (level < FTGEMM_FT_OFF || level > FTGEMM_FT_AUTO || level == FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_autotune: level %d (F32 SIMT levels and AUTO only)", (int)level);
  CK(cudaSetDevice(h->device));
  reps = std::max(1, reps);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool timing = h->timing;
  h->timing = false;
  // time one candidate: a warm-up run, then `reps` runs between two events
  auto time_it = [&](const ftgemm_schedule& s, ftgemm_ft_level lv, float* ms) -> int {
    int rc = simt_gemm(h, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, lv, s, nullptr, nullptr);
    if (rc) return rc;
    CK(cudaEventRecord(e0, h->stream));
    for (int r = 0; r < reps; ++r) {
      rc = simt_gemm(h, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, lv, s, nullptr, nullptr);
      if (rc) return rc;
    }
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= reps;
    return FTGEMM_OK;
  };
  std::vector<ftgemm_ft_level> levels;
  if (level == FTGEMM_FT_AUTO) levels = {FTGEMM_FT_BLOCK, FTGEMM_FT_WARP, FTGEMM_FT_THREAD};
  else levels = {level};
  float best_ms = 1e30f;
  ftgemm_schedule best{};
  ftgemm_ft_level best_lv = levels[0];
  int rc = FTGEMM_OK;
  for (ftgemm_ft_level lv : levels) {
    // 1. the tile tuple, with the default cadence and no split-K (and the
    //    default schedule itself)
    std::vector<std::pair<float, ftgemm_schedule>> tried;
    ftgemm_schedule d;
    default_schedule(h, m, n, k, (int)lv, &d);
    for (int c = -1; c < (int)(sizeof(kSimtConfigs) / sizeof(kSimtConfigs[0])); ++c) {
      ftgemm_schedule s = d;
      if (c >= 0) {
        const SimtConfig& q = kSimtConfigs[c];
        s = ftgemm_schedule{q.m_tb, q.n_tb, q.k_tb, q.m_w, q.n_w, q.m_t, q.n_t, std::max(1, 256 / q.k_tb), 1};
        if (s.m_tb == d.m_tb && s.n_tb == d.n_tb && s.k_tb == d.k_tb && s.m_w == d.m_w && s.n_w == d.n_w &&
            s.m_t == d.m_t && s.n_t == d.n_t && d.split_k == 1)
          continue;  // the same as the default
      }
      float ms;
      if ((rc = time_it(s, lv, &ms))) break;
      tried.push_back({ms, s});
    }
    if (rc) break;
    std::sort(tried.begin(), tried.end(), [](const std::pair<float, ftgemm_schedule>& a,
                                             const std::pair<float, ftgemm_schedule>& b) { return a.first < b.first; });
    // 2. split-K for every tuple (a large tile with few tiles can be the
    //    fastest once split) while each split keeps >= 8 k-steps and the
    //    CTAs stay within 16 per SM; not only powers of two, so that
    //    tiles x splits can fill the SMs without a nearly empty last wave
    static const int kSplits[] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 48, 64, 96, 128};
    const size_t top = tried.size();
    const int64_t max_ctas = 16LL * (h->num_sms > 0 ? h->num_sms : 148);
    for (size_t q = 0; q < top && !rc; ++q) {
      const ftgemm_schedule base = tried[q].second;
      const int64_t ksteps = (k + base.k_tb - 1) / base.k_tb;
      const int64_t tiles = ((m + base.m_tb - 1) / base.m_tb) * ((n + base.n_tb - 1) / base.n_tb);
      for (int split : kSplits) {
        if (ksteps / split < 8 || tiles * split > max_ctas) break;
        ftgemm_schedule s = base;
        s.split_k = split;
        float ms;
        if ((rc = time_it(s, lv, &ms))) break;
        tried.push_back({ms, s});
      }
    }
    if (rc) break;
    std::sort(tried.begin(), tried.end(), [](const std::pair<float, ftgemm_schedule>& a,
                                             const std::pair<float, ftgemm_schedule>& b) { return a.first < b.first; });
    // 3. the verification cadence of the fastest: the paper's K_s = 256
    //    against once per split (checksums still accumulated every k-step)
    if (lv != FTGEMM_FT_OFF) {
      ftgemm_schedule s = tried[0].second;
      s.cadence = 0;  // once, after the last k-step of each split
      float ms;
      if ((rc = time_it(s, lv, &ms))) break;
      tried.push_back({ms, s});
      std::sort(tried.begin(), tried.end(), [](const std::pair<float, ftgemm_schedule>& a,
                                               const std::pair<float, ftgemm_schedule>& b) { return a.first < b.first; });
    }
    if (tried[0].first < best_ms) {
      best_ms = tried[0].first;
      best = tried[0].second;
      best_lv = lv;
    }
  }
  h->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  h->tuned[std::make_tuple(m, n, k, (int)level)] = {best, (int)best_lv};
  if (out) *out = best;
  if (level_out) *level_out = best_lv;
  return FTGEMM_OK;
}

// ---- tensor-core autotuner: single CTAs or CTA pairs, by measurement ----

// Best of `reps` timings of `call` (after one warm-up) on the handle's stream.
template <class F>
static int time_best(ftgemm_ctx* h, F call, int reps, float* best_ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    FAIL(FTGEMM_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  int rc = call();
  float best = 3.4e38f;
  for (int r = 0; rc == FTGEMM_OK && r < reps; ++r) {
    e = cudaEventRecord(a, h->stream);
    if (e == cudaSuccess) rc = call();
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventRecord(b, h->stream);
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess && rc == FTGEMM_OK) rc = FTGEMM_ERR_CUDA;
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  *best_ms = best;
  return FTGEMM_OK;
}

// Best time of two candidates over `reps` rounds, timed interleaved (one
// call of each per round, the order alternating) so that a drift of the
// clocks or of the memory system during the tuning weighs on both alike;
// each candidate is called once, untimed, first.
template <class F0, class F1>
static int time_best_pair(ftgemm_ctx* h, F0 call0, F1 call1, int reps, float* ms0, float* ms1) {
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    FAIL(FTGEMM_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  int rc = call0();
  if (rc == FTGEMM_OK) rc = call1();
  float best[2] = {3.4e38f, 3.4e38f};
  for (int r = 0; rc == FTGEMM_OK && r < 2 * reps; ++r) {
    const int c = (r & 1) ^ ((r >> 1) & 1);  // 0 1 1 0 0 1 1 0 ...
    e = cudaEventRecord(a, h->stream);
    if (e == cudaSuccess) rc = c ? call1() : call0();
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventRecord(b, h->stream);
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess && rc == FTGEMM_OK) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess && rc == FTGEMM_OK) rc = FTGEMM_ERR_CUDA;
    best[c] = std::min(best[c], ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  *ms0 = best[0];
  *ms1 = best[1];
  return FTGEMM_OK;
}

int ftgemm_autotune_tc(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                       const void* B, int64_t ldb, float* C, int64_t ldc, ftgemm_dtype dtype,
                       ftgemm_ft_level level, int32_t reps, int32_t* pair_out) {
  if (!h || !A || !B || !C || m <= 0 || n <= 0 || k <= 0 || reps < 1 || m > INT32_MAX || n > INT32_MAX ||
      k > INT32_MAX || lda < k || ldb < n || ldc < n)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_autotune_tc: bad argument");
  if (dtype != FTGEMM_BF16 && dtype != FTGEMM_E4M3)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_autotune_tc: bf16 or e4m3 operands only");
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_TILE)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_autotune_tc: level OFF or TILE, not %d", (int)level);
  CK(cudaSetDevice(h->device));
  const int saved = h->tc_pair;
  float ms[2] = {0.f, 0.f};
  auto run = [&](int p) {
    h->tc_pair = p;
    return tc_gemm(h, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, dtype, level, nullptr, nullptr);
  };
  const int rc = time_best_pair(h, [&]() { return run(0); }, [&]() { return run(1); }, reps, &ms[0], &ms[1]);
  h->tc_pair = saved;
  if (rc) return rc;
  const int pick = ms[1] < ms[0] ? 1 : 0;
  const int dt = dtype == FTGEMM_BF16 ? 0 : 1;
  h->tc_tuned[std::make_tuple(m, n, k, dt, (int)level)] = pick;
  if (pair_out) *pair_out = pick;
  return FTGEMM_OK;
}

int ftgemm_group_autotune(ftgemm_handle_t h, int32_t count, const ftgemm_problem* problems, ftgemm_dtype dtype,
                          ftgemm_ft_level level, int32_t reps, ftgemm_group_t* out, int32_t* pair_out) {
  if (!h || !problems || !out || count <= 0 || reps < 1) FAIL(FTGEMM_ERR_ARG, "ftgemm_group_autotune: bad argument");
  *out = nullptr;
  const int saved = h->tc_pair;
  ftgemm_group_t g[2] = {nullptr, nullptr};
  float ms[2] = {0.f, 0.f};
  int rc = FTGEMM_OK;
  for (int p = 0; p < 2 && rc == FTGEMM_OK; ++p) {
    h->tc_pair = p;
    rc = ftgemm_group_create(h, count, problems, dtype, level, &g[p]);
  }
  h->tc_pair = saved;
  if (rc == FTGEMM_OK)
    rc = time_best_pair(h, [&]() { return ftgemm_grouped_gemm(h, g[0]); },
                        [&]() { return ftgemm_grouped_gemm(h, g[1]); }, reps, &ms[0], &ms[1]);
  if (rc) {
    for (int p = 0; p < 2; ++p) ftgemm_group_destroy(g[p]);
    return rc;
  }
  const int pick = ms[1] < ms[0] ? 1 : 0;
  ftgemm_group_destroy(g[1 - pick]);
  *out = g[pick];
  if (pair_out) *pair_out = pick;
  return FTGEMM_OK;
}

int ftgemm_selftest_wait(ftgemm_handle_t h, int64_t limit_cycles) {
  if (!h || limit_cycles <= 0 || limit_cycles > (1ll << 34))
    FAIL(FTGEMM_ERR_ARG, "ftgemm_selftest_wait: bad argument");
  CK(cudaSetDevice(h->device));
  int rc = clear_report(h);
  if (rc) return rc;
  CK(launch_wait_selftest(h->rep, limit_cycles, h->stream));
  ++h->launches;
  ftgemm_report r;
  memset(&r, 0, sizeof(r));
  return ftgemm_report_fetch(h, &r);  // FTGEMM_ERR_TIMEOUT when the wait gave up
}

// ---- non-fused ABFT baseline (Section 5.3's comparison scheme) --------------

int ftgemm_gemm_nonfused(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, double alpha, const float* A,
                         int64_t lda, const float* B, int64_t ldb, double beta, float* C, int64_t ldc, int32_t ks,
                         const ftgemm_inject_spec* inject, ftgemm_report* report) {
  if (!h || !A || !B || !C || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || ldc < n)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm_nonfused: bad argument");
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm_nonfused: size too large");
  if (ks <= 0) ks = 256;
  if (ks % 16) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm_nonfused: the step K_s must be a multiple of 16");
  CK(cudaSetDevice(h->device));
  const int M = (int)m, N = (int)n, K = (int)k, T = 128;
  const int tiles_m = (M + T - 1) / T, tiles_n = (N + T - 1) / T, ksteps = (K + 15) / 16;
  const ftgemm_schedule unit{T, T, 16, 64, 64, 16, 8, ks / 16, 1};  // the tiling faults refer to
  int nf = 0;
  {
    int rc = upload_faults(h, inject, unit, M, N, ksteps, tiles_m, tiles_n, FTGEMM_FT_BLOCK, &nf);
    if (rc) return rc;
  }
  if (report) {
    int rc = clear_report(h);
    if (rc) return rc;
  }
  // workspace (its own buffer: the GEMM calls below use the handle's)
  auto r4 = [](long long x) { return (x + 3) / 4 * 4; };
  const long long ldt = r4(M), ldv = r4(K), ldvt = r4(tiles_m), ldwt = r4(tiles_n), ldacc = r4(N);
  size_t o = 0;
  auto take = [&](size_t floats) { const size_t at = o; o = align64(o + floats); return at; };
  const size_t oAt = take((size_t)K * ldt), oV = take((size_t)tiles_m * ldv), oW = take((size_t)tiles_n * ldv),
               oVt = take((size_t)K * ldvt), oWt = take((size_t)K * ldwt), oNa = take(M), oNb = take(N),
               oScr = take((size_t)std::max<long long>((long long)((K + 31) / 32) * M, kmajor_scratch_floats(K, N))),
               oAcc = take((size_t)M * ldacc), oCc = take((size_t)tiles_m * ldacc), oCr = take((size_t)tiles_n * ldt);
  if (o > h->ws2_floats) {
    CK(cudaStreamSynchronize(h->stream));
    if (h->ws2) CK(cudaFree(h->ws2));
    h->ws2 = nullptr;
    h->ws2_floats = 0;
    CK(cudaMalloc(&h->ws2, o * sizeof(float)));
    h->ws2_floats = o;
  }
  float* w = h->ws2;
  float *At = w + oAt, *V = w + oV, *W = w + oW, *Vt = w + oVt, *Wt = w + oWt, *nA = w + oNa, *nB = w + oNb,
        *Acc = w + oAcc, *Cc = w + oCc, *CrT = w + oCr;
  int launches = 0;
  // encode (Eq. 1-2): A^T with e^T A per 128-row block and row norms; B e per
  // 128-column block and column norms; the checksum vectors k-major
  CK(launch_transpose_encode(A, lda, M, K, At, ldt, T, V, ldv, nA, w + oScr, &launches, h->stream));
  CK(launch_encode_kmajor(B, ldb, K, N, T, W, ldv, nB, w + oScr, &launches, h->stream));
  CK(launch_transpose(V, ldv, tiles_m, K, Vt, ldvt, h->stream));
  CK(launch_transpose(W, ldv, tiles_n, K, Wt, ldwt, h->stream));
  launches += 2;
  const float lam_u = (float)(h->lambda * std::ldexp(1.0, -24));
  const bool timing = h->timing;
  h->timing = false;
  int rc = FTGEMM_OK;
  for (int k0 = 0; k0 < K && !rc; k0 += ks) {
    const int kl = std::min(ks, K - k0);
    const double b0 = k0 == 0 ? 0.0 : 1.0;
    ftgemm_schedule sa, sb, sc;
    default_schedule(h, M, N, kl, FTGEMM_FT_OFF, &sa);
    default_schedule(h, tiles_m, N, kl, FTGEMM_FT_OFF, &sb);
    default_schedule(h, tiles_n, M, kl, FTGEMM_FT_OFF, &sc);
    // the step's product and the updates of the two checksums (Eq. 4)
    rc = simt_gemm(h, M, N, kl, 1.0, nullptr, 0, B + (long long)k0 * ldb, ldb, b0, Acc, ldacc, FTGEMM_FT_OFF, sa,
                   nullptr, nullptr, At + (long long)k0 * ldt, ldt);
    if (!rc)
      rc = simt_gemm(h, tiles_m, N, kl, 1.0, nullptr, 0, B + (long long)k0 * ldb, ldb, b0, Cc, ldacc, FTGEMM_FT_OFF,
                     sb, nullptr, nullptr, Vt + (long long)k0 * ldvt, ldvt);
    if (!rc)
      rc = simt_gemm(h, tiles_n, M, kl, 1.0, nullptr, 0, At + (long long)k0 * ldt, ldt, b0, CrT, ldt, FTGEMM_FT_OFF,
                     sc, nullptr, nullptr, Wt + (long long)k0 * ldwt, ldwt);
    if (rc) break;
    // faults scheduled inside this step, then the verification after it
    const int ks_lo = k0 / 16, ks_hi = (k0 + kl + 15) / 16;
    CK(launch_nonfused_inject(nf > 0 ? h->d_faults : nullptr, nf, ks_lo, ks_hi, tiles_n, Acc, ldacc, Cc, ldacc, CrT,
                              ldt, h->stream));
    // growth term after the k0 + kl elements of K accumulated so far
    const float grow = (float)(h->mu * std::ldexp(1.0, -24) * std::sqrt((double)(k0 + kl)));
    CK(launch_nonfused_verify(Acc, ldacc, M, N, Cc, ldacc, CrT, ldt, nA, nB, lam_u, grow, ks_hi - 1, h->rep,
                              h->recs, h->stream));
    launches += (nf > 0 ? 1 : 0) + 1;
  }
  h->timing = timing;
  if (rc) return rc;
  CK(launch_nonfused_epilogue(Acc, ldacc, M, N, (float)alpha, (float)beta, C, ldc, h->stream));
  ++launches;
  h->launches += launches;
  if (report) return ftgemm_report_fetch(h, report);
  return FTGEMM_OK;
}

// ---- offline (detect-only, recompute) ABFT (Section 5.5) --------------------

int ftgemm_gemm_offline(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, double alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, double beta, float* C, int64_t ldc,
                        const ftgemm_inject_spec* const* injects, int32_t max_runs, int32_t* runs_out,
                        ftgemm_report* report) {
  if (runs_out) *runs_out = 0;
  if (!h || !A || !B || !C || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || ldc < n || max_runs <= 0)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm_offline: bad argument");
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "ftgemm_gemm_offline: size too large");
  CK(cudaSetDevice(h->device));
  // detector: the detect-only kernel on the 128 x 128 x 32 tile -- column
  // checksums only, one verification after the last k-step, no correction
  const ftgemm_schedule det{128, 128, 32, 64, 64, 16, 8, 0, 1};
  // C_in is kept for the recomputation when beta reads it
  float* cin = nullptr;
  const size_t cin_floats = (size_t)m * (size_t)n;
  if (beta != 0.0) {
    if (cin_floats > h->ws2_floats) {
      CK(cudaStreamSynchronize(h->stream));
      if (h->ws2) CK(cudaFree(h->ws2));
      h->ws2 = nullptr;
      h->ws2_floats = 0;
      CK(cudaMalloc(&h->ws2, cin_floats * sizeof(float)));
      h->ws2_floats = cin_floats;
    }
    cin = h->ws2;
    CK(cudaMemcpy2DAsync(cin, n * sizeof(float), C, ldc * sizeof(float), n * sizeof(float), m,
                         cudaMemcpyDeviceToDevice, h->stream));
  }
  int rc = clear_report(h);
  if (rc) return rc;
  unsigned long long before = 0;
  for (int r = 0; r < max_runs; ++r) {
    if (cin && r > 0)
      CK(cudaMemcpy2DAsync(C, ldc * sizeof(float), cin, n * sizeof(float), n * sizeof(float), m,
                           cudaMemcpyDeviceToDevice, h->stream));
    rc = simt_gemm(h, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, FTGEMM_FT_BLOCK, det,
                   injects ? injects[r] : nullptr, nullptr, nullptr, 0, true);
    if (rc) return rc;
    // the detection count so far (the report accumulates over attempts)
    unsigned long long det_now = 0;
    CK(cudaMemcpyAsync(&det_now, &h->rep->detected, sizeof(det_now), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (runs_out) *runs_out = r + 1;
    if (det_now == before) {
      if (report) return ftgemm_report_fetch(h, report);
      return FTGEMM_OK;
    }
    before = det_now;
  }
  if (report) {
    rc = ftgemm_report_fetch(h, report);
    if (rc) return rc;
  }
  FAIL(FTGEMM_ERR_UNRECOVERED, "ftgemm_gemm_offline: all %d attempts detected a fault", max_runs);
}

// ---- double and double complex (Section 6: DGEMM / ZGEMM) -------------------

static int f64_gemm(ftgemm_ctx* h, bool cplx, int64_t m, int64_t n, int64_t k, const double* alpha,
                    const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                    int64_t ldc, ftgemm_ft_level level, int32_t cadence, const ftgemm_inject_spec* inject,
                    ftgemm_report* report, double* imag) {
  const char* who = cplx ? "ftgemm_zgemm" : "ftgemm_dgemm";
  if (!h || !A || !B || !C || !alpha || !beta || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || ldc < n)
    FAIL(FTGEMM_ERR_ARG, "%s: bad argument", who);
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) FAIL(FTGEMM_ERR_ARG, "%s: size too large", who);
  if (level == FTGEMM_FT_AUTO) level = FTGEMM_FT_BLOCK;
  if (level != FTGEMM_FT_OFF && level != FTGEMM_FT_BLOCK)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "%s: checksum level %d (OFF or BLOCK only)", who, (int)level);
  const size_t esz = cplx ? 16 : 8;
  if ((uintptr_t)A % esz || (uintptr_t)B % esz || (uintptr_t)C % esz)
    FAIL(FTGEMM_ERR_ALIGN, "%s: operands must be aligned to their element size (%zu bytes)", who, esz);
  CK(cudaSetDevice(h->device));
  const int M = (int)m, N = (int)n, K = (int)k, T = f64_tile(cplx);
  const int tiles_m = (M + T - 1) / T, tiles_n = (N + T - 1) / T, ksteps = (K + FTGEMM_F64_KSTEP - 1) / FTGEMM_F64_KSTEP;
  if (tiles_m > 65535) FAIL(FTGEMM_ERR_ARG, "%s: m too large for the tile grid", who);
  const bool abft = level == FTGEMM_FT_BLOCK;
  const ftgemm_schedule unit{T, T, FTGEMM_F64_KSTEP, T, T, T / 16, T / 16, 1, 1};  // the tiling faults refer to
  int nf = 0;
  {
    int rc = upload_faults(h, inject, unit, M, N, ksteps, tiles_m, tiles_n, level, &nf, cplx);
    if (rc) return rc;
  }
  if (report) {
    int rc = clear_report(h);
    if (rc) return rc;
  }
  if (cplx && !h->zimag) CK(cudaMalloc(&h->zimag, sizeof(double) * 3 * (size_t)h->rep_cap));
  int launches = 0;
  // workspace: V[tiles_m][K], W[tiles_n][K] (operand type), nA[M], nB[N]
  const size_t ev = esz / 4;  // floats per element
  size_t o = 0;
  auto take = [&](size_t floats) { const size_t at = o; o = align64(o + floats); return at; };
  const size_t oV = take(ev * (size_t)tiles_m * K), oW = take(ev * (size_t)tiles_n * K), oNa = take(2 * (size_t)M),
               oNb = take(2 * (size_t)N);
  if (abft) {
    int rc = ensure_ws(h, o);
    if (rc) return rc;
    CK(launch_f64_encode(cplx, A, lda, B, ldb, M, N, K, h->ws + oV, h->ws + oW, (double*)(h->ws + oNa),
                         (double*)(h->ws + oNb), &launches, h->stream));
  }
  F64Params p{};
  p.M = M; p.N = N; p.K = K;
  p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
  p.alpha_re = alpha[0]; p.alpha_im = cplx ? alpha[1] : 0.0;
  p.beta_re = beta[0]; p.beta_im = cplx ? beta[1] : 0.0;
  p.beta_zero = p.beta_re == 0.0 && p.beta_im == 0.0;
  if (abft) {
    p.V = h->ws + oV; p.W = h->ws + oW;
    p.nA = (const double*)(h->ws + oNa); p.nB = (const double*)(h->ws + oNb);
  }
  p.lam_u = h->lambda * std::ldexp(1.0, -53);
  p.mu_u = h->mu * std::ldexp(1.0, -53);
  p.cadence = cadence > 0 ? cadence : ksteps;
  p.faults = nf > 0 ? h->d_faults : nullptr;
  p.nfaults = nf;
  p.rep = h->rep;
  p.recs = h->recs;
  p.imag = cplx ? h->zimag : nullptr;
  std::pair<cudaEvent_t, cudaEvent_t> ev2;
  if (h->timing) {
    int rc = take_events(h, &ev2);
    if (rc) return rc;
    CK(cudaEventRecord(ev2.first, h->stream));
  }
  CK(launch_f64_gemm(cplx, abft, p, h->stream));
  ++launches;
  if (h->timing) {
    CK(cudaEventRecord(ev2.second, h->stream));
    h->pending.push_back(ev2);
  }
  h->launches += launches;
  if (!report) return FTGEMM_OK;
  int rc = ftgemm_report_fetch(h, report);
  if (rc) return rc;
  // pair each returned record with its imaginary parts through its slot
  const int w = std::min(std::max(0, report->capacity), std::min(report->n_records, h->rep_cap));
  if (cplx && imag && w > 0 && report->records) {
    const int slots = std::min(report->n_records, h->rep_cap);
    std::vector<double> im(3 * (size_t)slots);
    CK(cudaMemcpy(im.data(), h->zimag, sizeof(double) * im.size(), cudaMemcpyDeviceToHost));
    for (int q = 0; q < w; ++q) {
      const int sl = report->records[q].reserved;
      for (int e = 0; e < 3; ++e) imag[3 * q + e] = (sl >= 0 && sl < slots) ? im[3 * (size_t)sl + e] : 0.0;
    }
  }
  for (int q = 0; q < w && report->records; ++q) report->records[q].reserved = 0;
  return FTGEMM_OK;
}

int ftgemm_dgemm(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double beta, double* C, int64_t ldc, ftgemm_ft_level ft_level,
                 int32_t cadence, const ftgemm_inject_spec* inject, ftgemm_report* report) {
  const double al[2] = {alpha, 0.0}, be[2] = {beta, 0.0};
  return f64_gemm(h, false, m, n, k, al, A, lda, B, ldb, be, C, ldc, ft_level, cadence, inject, report, nullptr);
}

int ftgemm_zgemm(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, const double* alpha, const double* A,
                 int64_t lda, const double* B, int64_t ldb, const double* beta, double* C, int64_t ldc,
                 ftgemm_ft_level ft_level, int32_t cadence, const ftgemm_inject_spec* inject, ftgemm_report* report,
                 double* imag) {
  return f64_gemm(h, true, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ft_level, cadence, inject, report, imag);
}
