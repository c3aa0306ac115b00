// api.cu -- the C ABI of libftgemm (include/ftgemm.h): handle, argument
// checks, schedule choice, fault table, workspaces, dispatch and report.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ftg {
cudaError_t simt_launch_small(int, bool, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_medium(int, bool, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_large(int, bool, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_tall(int, bool, const SimtParams&, int, cudaStream_t);
cudaError_t simt_launch_huge(int, bool, const SimtParams&, int, cudaStream_t);
cudaError_t launch_encode(const float*, long long, const float*, long long, int, int, int, int, int,
                          float*, float*, float*, float*, float*, cudaStream_t);
long long colnorm_scratch_floats(int K, int N);
cudaError_t launch_splitk_reduce(const float*, int, int, int, float, float, float*, long long,
                                 cudaStream_t);

using SimtLaunch = cudaError_t (*)(int, bool, const SimtParams&, int, cudaStream_t);

// The compiled SIMT tile tuples: the five kernel setups of Table 1.
struct SimtConfig {
  const char* name;
  int m_tb, n_tb, k_tb, m_w, n_w, m_t, n_t;
  SimtLaunch launch;
};
static const SimtConfig kSimtConfigs[] = {
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

}  // namespace ftg

using namespace ftg;

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
  cudaEvent_t faults_free = nullptr;
  // settings
  bool has_sched = false;
  ftgemm_schedule sched{};
  double lambda = 32.0;
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
  int cap = std::max(n, 2 * h->faults_cap);
  CK(cudaMalloc(&h->d_faults, sizeof(Fault) * cap));
  CK(cudaHostAlloc(&h->h_faults, sizeof(Fault) * cap, cudaHostAllocDefault));
  h->faults_cap = cap;
  return FTGEMM_OK;
}

static size_t align64(size_t x) { return (x + 63) & ~size_t(63); }

static int default_schedule(const ftgemm_ctx* h, int64_t m, int64_t n, int64_t k,
                            ftgemm_schedule* s) {
  const int sms = h->num_sms > 0 ? h->num_sms : 152;
  const SimtConfig* pick = nullptr;
  for (const auto& c : kSimtConfigs) {
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

extern "C" {

const char* ftgemm_status_string(int status) {
  switch (status) {
    case FTGEMM_OK: return "ok";
    case FTGEMM_ERR_ARG: return "invalid argument";
    case FTGEMM_ERR_UNSUPPORTED: return "unsupported dtype / level / schedule";
    case FTGEMM_ERR_ALIGN: return "misaligned pointer or stride";
    case FTGEMM_ERR_CUDA: return "CUDA error";
    case FTGEMM_ERR_TIMEOUT: return "device wait timed out";
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
  if (cudaMalloc(&h->rep, sizeof(DevReport)) != cudaSuccess ||
      cudaMalloc(&h->recs, sizeof(ftgemm_fault_record) * h->rep_cap) != cudaSuccess ||
      cudaMemset(h->rep, 0, sizeof(DevReport)) != cudaSuccess) {
    delete h;
    FAIL(FTGEMM_ERR_CUDA, "ftgemm_create: cannot allocate the report ring");
  }
  DevReport r{};
  r.capacity = h->rep_cap;
  CK(cudaMemcpy(h->rep, &r, sizeof(r), cudaMemcpyHostToDevice));
  CK(cudaEventCreateWithFlags(&h->faults_free, cudaEventDisableTiming));
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
  if (h->d_faults) cudaFree(h->d_faults);
  if (h->h_faults) cudaFreeHost(h->h_faults);
  if (h->faults_free) cudaEventDestroy(h->faults_free);
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
  (void)level;
  if (h->has_sched) { *out = h->sched; return FTGEMM_OK; }
  return default_schedule(h, m, n, k, out);
}

int ftgemm_set_threshold(ftgemm_handle_t h, int mode, double lambda, const float* w, size_t nw) {
  if (!h) FAIL(FTGEMM_ERR_ARG, "ftgemm_set_threshold: NULL handle");
  (void)w; (void)nw;
  if (mode != 0) FAIL(FTGEMM_ERR_UNSUPPORTED, "threshold mode %d is not available", mode);
  if (lambda > 0) h->lambda = lambda;
  return FTGEMM_OK;
}

static int clear_report(ftgemm_ctx* h) {
  CK(cudaMemsetAsync(h->rep, 0, offsetof(DevReport, capacity), h->stream));
  CK(cudaMemsetAsync(&h->rep->timeouts, 0, sizeof(int), h->stream));
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
  return FTGEMM_OK;
}

int ftgemm_encode(ftgemm_handle_t h, int64_t m, int64_t n, int64_t k, const float* A, int64_t lda,
                  const float* B, int64_t ldb, int32_t m_u, int32_t n_u, float* V, float* W,
                  float* nA, float* nB) {
  if (!h || !A || !B || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || m_u <= 0 || n_u <= 0 ||
      m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
    FAIL(FTGEMM_ERR_ARG, "ftgemm_encode: bad argument");
  CK(cudaSetDevice(h->device));
  float* scratch = nullptr;
  if (nB) {
    int rc = ensure_ws(h, (size_t)colnorm_scratch_floats((int)k, (int)n));
    if (rc) return rc;
    scratch = h->ws;
  }
  CK(launch_encode(A, lda, B, ldb, (int)m, (int)n, (int)k, m_u, n_u, V, W, nA, nB, scratch,
                   h->stream));
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
  if (dtype != FTGEMM_F32)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: dtype %d is not available in this build", (int)dtype);
  if (level < FTGEMM_FT_OFF || level > FTGEMM_FT_BLOCK)
    FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: level %d needs a tensor-core dtype", (int)level);
  CK(cudaSetDevice(h->device));

  ftgemm_schedule s;
  if (h->has_sched) s = h->sched;
  else default_schedule(h, m, n, k, &s);
  const SimtConfig* cfg = find_simt(s);
  if (!cfg) FAIL(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm: schedule is not a compiled kernel");

  const int M = (int)m, N = (int)n, K = (int)k;
  const int ksteps = (K + s.k_tb - 1) / s.k_tb;
  int split = std::max(1, std::min(s.split_k, ksteps));
  const int ks_per_split = (ksteps + split - 1) / split;
  split = (ksteps + ks_per_split - 1) / ks_per_split;
  const int cadence = s.cadence > 0 ? s.cadence : ks_per_split;
  const int tiles_m = (M + s.m_tb - 1) / s.m_tb, tiles_n = (N + s.n_tb - 1) / s.n_tb;

  const float* Af = (const float*)A;
  const float* Bf = (const float*)B;
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && (ldc % 4 == 0) && (K % 4 == 0) &&
                   (N % 4 == 0) && al16(A) && al16(B) && al16(C);

  // ---- faults: validate, resolve, sort, upload -----------------------------
  int nf = inject ? inject->n : 0;
  if (nf < 0) FAIL(FTGEMM_ERR_ARG, "inject->n < 0");
  if (nf > 0) {
    if (!inject->tile_m || !inject->tile_n || !inject->kstep || !inject->row || !inject->col ||
        !inject->delta)
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
      if (tg < 0 || tg > 2) FAIL(FTGEMM_ERR_ARG, "inject[%d]: target %d", i, tg);
      if (level == FTGEMM_FT_OFF && tg != 0) FAIL(FTGEMM_ERR_ARG, "inject[%d]: no checksums at level OFF", i);
      fv[i] = Fault{tm * tiles_n + tn, ks, r, c, tg, inject->delta[i]};
    }
    std::stable_sort(fv.begin(), fv.end(), [](const Fault& a, const Fault& b) {
      return a.tile != b.tile ? a.tile < b.tile : a.kstep < b.kstep;
    });
    memcpy(h->h_faults, fv.data(), sizeof(Fault) * nf);
    CK(cudaMemcpyAsync(h->d_faults, h->h_faults, sizeof(Fault) * nf, cudaMemcpyHostToDevice, h->stream));
    CK(cudaEventRecord(h->faults_free, h->stream));
  }

  if (report) {
    int rc = clear_report(h);
    if (rc) return rc;
  }

  // ---- workspace ----------------------------------------------------------
  const bool abft = level != FTGEMM_FT_OFF;
  int m_u = 1, n_u = 1;
  bool need_vw = false;
  if (level == FTGEMM_FT_WARP) { m_u = s.m_w; n_u = s.n_w; need_vw = true; }
  if (level == FTGEMM_FT_BLOCK) { m_u = s.m_tb; n_u = s.n_tb; need_vw = true; }
  const size_t nV = need_vw ? (size_t)((M + m_u - 1) / m_u) * K : 0;
  const size_t nW = need_vw ? (size_t)((N + n_u - 1) / n_u) * K : 0;
  const size_t nNa = abft ? (size_t)M : 0, nNb = abft ? (size_t)N : 0;
  const size_t nScr = abft ? (size_t)colnorm_scratch_floats(K, N) : 0;
  const size_t nPart = split > 1 ? (size_t)split * M * N : 0;
  const size_t oV = 0, oW = align64(oV + nV), oNa = align64(oW + nW), oNb = align64(oNa + nNa),
               oScr = align64(oNb + nNb), oPart = align64(oScr + nScr), total = align64(oPart + nPart);
  if (total > 0) {
    int rc = ensure_ws(h, total);
    if (rc) return rc;
  }
  float* ws = h->ws;

  if (abft) {
    CK(launch_encode(Af, lda, Bf, ldb, M, N, K, m_u, n_u, need_vw ? ws + oV : nullptr,
                     need_vw ? ws + oW : nullptr, ws + oNa, ws + oNb, ws + oScr, h->stream));
  }

  SimtParams p;
  p.M = M; p.N = N; p.K = K;
  p.A = Af; p.lda = lda; p.B = Bf; p.ldb = ldb; p.C = C; p.ldc = ldc;
  p.alpha = (float)alpha; p.beta = (float)beta;
  p.V = need_vw ? ws + oV : nullptr;
  p.Wt = need_vw ? ws + oW : nullptr;
  p.nA = abft ? ws + oNa : nullptr;
  p.nB = abft ? ws + oNb : nullptr;
  p.lam_u = (float)(h->lambda * std::ldexp(1.0, -24));
  p.cadence = std::max(1, cadence);
  p.ksteps = ksteps;
  p.ks_per_split = ks_per_split;
  p.partial = split > 1 ? ws + oPart : nullptr;
  p.faults = nf > 0 ? h->d_faults : nullptr;
  p.nfaults = nf;
  p.rep = h->rep;
  p.recs = h->recs;
  p.tiles_n = tiles_n;
  CK(cfg->launch((int)level, vec, p, split, h->stream));
  if (split > 1)
    CK(launch_splitk_reduce(ws + oPart, split, M, N, (float)alpha, (float)beta, C, ldc, h->stream));

  if (report) return ftgemm_report_fetch(h, report);
  return FTGEMM_OK;
}

}  // extern "C"
