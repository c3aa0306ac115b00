// noalloc.cu -- ftgemm_gemm_noalloc: the fp32 fused-ABFT GEMM without any
// device allocation, for callers that may not call cudaMalloc (no
// counterpart in the paper; the checksum levels are those of Section 4.2).
//
// Some callers cannot allocate device memory at the moment they need a GEMM:
// a framework whose caching allocator already owns the whole device, code
// that must not trigger the device-wide synchronisation cudaMalloc and
// cudaFree can cause, or recovery code running after an out-of-memory error.
// This entry point serves them: it needs no handle (creating one allocates)
// and keeps every temporary -- the transposed A, the encoded vectors, the
// norms and the event report -- in one fixed array compiled into the
// library, kNoallocBytes bytes in size.  Every GPU that loads the library
// holds that array until the process exits.
//
// The array is shared by all calls: each call clears what must start at
// zero (the report counters) and overwrites the rest.  Calls that overlap on
// the GPU (on different streams, or from several host threads at once) use
// the same bytes and race; serialise them.  The first call on each device
// sets the device up while it is current: it looks up the array's device
// address with cudaGetSymbolAddress and loads every kernel any later call
// can launch.  Under lazy module loading (CUDA's default) both steps can
// allocate device memory, so the no-allocation promise holds from the
// second call on: make one call (any size) at start-up, before relying on it
// and before any stream capture.
//
// Bounded device waits that give up are counted in the array and stay there
// until a call with a report reads them: that call returns
// FTGEMM_ERR_TIMEOUT and clears the count, so a give-up in a call without a
// report is not lost.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace ftg {
cudaError_t simt_launch_huge16(int, const SimtMaps&, const SimtParams&, int, cudaStream_t);
cudaError_t launch_transpose(const float*, long long, int, int, float*, long long, cudaStream_t);
cudaError_t launch_copy_pad(const float*, long long, int, int, float*, long long, cudaStream_t);
long long kmajor_scratch_floats(int K, int L);
cudaError_t launch_encode_kmajor(const float*, long long, int, int, int, float*, long long, float*,
                                 float*, int*, cudaStream_t);
void set_last_error(const char* msg);
cudaError_t preload_kmajor_kernels();
cudaError_t simt_preload_huge16();

constexpr size_t kNoallocBytes = (size_t)FTGEMM_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocRecords = 256;  // event records kept per call

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

int fail(int code, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof(b), fmt, ap);
  va_end(ap);
  set_last_error(b);
  return code;
}

// Zero the event counters and set the record capacity; the count of waits
// that gave up is left for the next call with a report to read.
__global__ void noalloc_reset_kernel(DevReport* rep, int capacity) {
  rep->detected = 0ull;
  rep->corrected = 0ull;
  rep->uncorrectable = 0ull;
  rep->checksum_only = 0ull;
  rep->n_records = 0;
  rep->capacity = capacity;
}

// Per-device set-up, done once with that device current: the array's device
// address (host code only knows a host-side stand-in for the symbol) and the
// loading of every kernel a call can launch.
void* scratch_address(int device, cudaError_t* err) {
  static std::mutex mu;
  static std::vector<void*> addr;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)addr.size() <= device) addr.resize(device + 1, nullptr);
  if (!addr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    cudaFuncAttributes a;
    *err = cudaFuncGetAttributes(&a, noalloc_reset_kernel);
    if (*err == cudaSuccess) *err = preload_kmajor_kernels();
    if (*err == cudaSuccess) *err = simt_preload_huge16();
    if (*err != cudaSuccess) return nullptr;
    addr[device] = p;
  }
  *err = cudaSuccess;
  return addr[device];
}

// The order ftgemm_report_fetch returns records in.
bool record_before(const ftgemm_fault_record& a, const ftgemm_fault_record& b) {
  if (a.problem != b.problem) return a.problem < b.problem;
  if (a.tile_m != b.tile_m) return a.tile_m < b.tile_m;
  if (a.tile_n != b.tile_n) return a.tile_n < b.tile_n;
  if (a.kstep != b.kstep) return a.kstep < b.kstep;
  if (a.row != b.row) return a.row < b.row;
  if (a.col != b.col) return a.col < b.col;
  return a.kind < b.kind;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool map2d(CUtensorMap* m, const float* base, uint64_t inner, uint64_t outer, uint64_t ld,
           uint32_t bi, uint32_t bo) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = (EncodeTiledFn)p;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {ld * sizeof(float)};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace ftg

using namespace ftg;

extern "C" int ftgemm_gemm_noalloc(int64_t m, int64_t n, int64_t k, double alpha, const float* A,
                                   int64_t lda, const float* B, int64_t ldb, double beta, float* C,
                                   int64_t ldc, ftgemm_ft_level level, void* cuda_stream,
                                   ftgemm_report* report) {
  if (!A || !B || !C) return fail(FTGEMM_ERR_ARG, "ftgemm_gemm_noalloc: NULL matrix pointer");
  if (m <= 0 || n <= 0 || k <= 0 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
    return fail(FTGEMM_ERR_ARG, "ftgemm_gemm_noalloc: bad size %lld x %lld x %lld", (long long)m,
                (long long)n, (long long)k);
  if (lda < k || ldb < n || ldc < n)
    return fail(FTGEMM_ERR_ARG, "ftgemm_gemm_noalloc: leading dimension too small");
  if (level < FTGEMM_FT_OFF || level > FTGEMM_FT_BLOCK)
    return fail(FTGEMM_ERR_UNSUPPORTED, "ftgemm_gemm_noalloc: level %d is not an fp32 level", (int)level);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(FTGEMM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));

  // the 128 x 128 x 16 tile, verification every 256 of K, no split-K
  const int MT = 128, NT = 128, KT = 16, WM = 32, WN = 64;
  const int M = (int)m, N = (int)n, K = (int)k;
  const bool abft = level != FTGEMM_FT_OFF;
  const bool vw = level == FTGEMM_FT_WARP || level == FTGEMM_FT_BLOCK;
  const int m_u = level == FTGEMM_FT_WARP ? WM : MT, n_u = level == FTGEMM_FT_WARP ? WN : NT;
  const int NV = level == FTGEMM_FT_WARP ? MT / WM : 1, NW = level == FTGEMM_FT_WARP ? NT / WN : 1;
  const long long ldt = (M + 3) / 4 * 4, ldv = (K + 3) / 4 * 4;
  const bool b_ok = (ldb % 4 == 0) && (((uintptr_t)B & 15) == 0);
  const long long ldbp = b_ok ? ldb : (N + 3) / 4 * 4;
  const int nvb = (M + m_u - 1) / m_u, nwb = (N + n_u - 1) / n_u;

  // byte layout inside the array
  const size_t oRep = 0;
  const size_t oRec = up256(oRep + sizeof(DevReport));
  const size_t oAt = up256(oRec + sizeof(ftgemm_fault_record) * kNoallocRecords);
  const size_t oBp = up256(oAt + sizeof(float) * (size_t)K * ldt);
  const size_t oV = up256(oBp + (b_ok ? 0 : sizeof(float) * (size_t)K * ldbp));
  const size_t oW = up256(oV + (vw ? sizeof(float) * (size_t)nvb * ldv : 0));
  const size_t oNa = up256(oW + (vw ? sizeof(float) * (size_t)nwb * ldv : 0));
  const size_t oNb = up256(oNa + (abft ? sizeof(float) * M : 0));
  const size_t oScr = up256(oNb + (abft ? sizeof(float) * N : 0));
  const size_t need = up256(oScr + (abft ? sizeof(float) * (size_t)std::max(kmajor_scratch_floats(K, M),
                                                                              kmajor_scratch_floats(K, N))
                                         : 0));
  if (need > kNoallocBytes)
    return fail(FTGEMM_ERR_ARG,
                "ftgemm_gemm_noalloc: %lld x %lld x %lld needs %zu bytes of scratch, more than the "
                "library's fixed %zu bytes; use ftgemm_gemm for this size",
                (long long)m, (long long)n, (long long)k, need, kNoallocBytes);

  unsigned char* base = (unsigned char*)scratch_address(dev, &e);
  if (!base) return fail(FTGEMM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  DevReport* rep = (DevReport*)(base + oRep);
  ftgemm_fault_record* recs = (ftgemm_fault_record*)(base + oRec);
  float* At = (float*)(base + oAt);
  float* Bp = (float*)(base + oBp);
  float* V = (float*)(base + oV);
  float* W = (float*)(base + oW);
  float* nA = (float*)(base + oNa);
  float* nB = (float*)(base + oNb);
  float* scr = (float*)(base + oScr);

#define NA_CK(call)                                                                          \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) return fail(FTGEMM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

  // what must start at zero: the event counters (capacity is rewritten too)
  noalloc_reset_kernel<<<1, 1, 0, st>>>(rep, kNoallocRecords);
  NA_CK(cudaGetLastError());

  int launches = 0;
  NA_CK(launch_transpose(A, lda, M, K, At, ldt, st));
  const float* Bk = B;
  if (!b_ok) {
    NA_CK(launch_copy_pad(B, ldb, K, N, Bp, ldbp, st));
    Bk = Bp;
  }
  if (abft) {
    NA_CK(launch_encode_kmajor(At, ldt, K, M, vw ? m_u : 2, vw ? V : nullptr, ldv, nA, scr, &launches, st));
    NA_CK(launch_encode_kmajor(Bk, ldbp, K, N, vw ? n_u : 2, vw ? W : nullptr, ldv, nB, scr, &launches, st));
  }
  SimtMaps maps;
  if (!map2d(&maps.A, At, M, K, ldt, MT, KT) || !map2d(&maps.B, Bk, N, K, ldbp, NT, KT) ||
      (vw && (!map2d(&maps.V, V, K, nvb, ldv, KT, NV) || !map2d(&maps.W, W, K, nwb, ldv, KT, NW))))
    return fail(FTGEMM_ERR_ALIGN, "ftgemm_gemm_noalloc: cannot build the TMA descriptors");
  if (!vw) { maps.V = maps.A; maps.W = maps.A; }

  SimtParams p;
  memset(&p, 0, sizeof(p));
  p.M = M; p.N = N; p.K = K;
  p.C = C; p.ldc = ldc;
  p.c_vec = (ldc % 4 == 0) && (((uintptr_t)C & 15) == 0);
  p.alpha = (float)alpha; p.beta = (float)beta;
  p.nA = abft ? nA : nullptr;
  p.nB = abft ? nB : nullptr;
  p.lam_u = (float)(32.0 * std::ldexp(1.0, -24));
  p.mu_u = (float)(8.0 * std::ldexp(1.0, -24));
  p.ksteps = (K + KT - 1) / KT;
  p.ks_per_split = p.ksteps;
  p.cadence = 256 / KT;
  p.partial = nullptr;
  p.faults = nullptr;
  p.nfaults = 0;
  p.rep = rep;
  p.recs = recs;
  p.tiles_m = (M + MT - 1) / MT;
  p.tiles_n = (N + NT - 1) / NT;
  p.group_m = std::min(p.tiles_m, 16);
  NA_CK(simt_launch_huge16((int)level, maps, p, 1, st));

  if (report) {
    DevReport r;
    NA_CK(cudaMemcpyAsync(&r, rep, sizeof(r), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    const int have = std::min(r.n_records, kNoallocRecords);
    const int w = std::min(have, std::max(0, report->capacity));
    if (w > 0 && report->records) {
      // all kept records, sorted as ftgemm_report_fetch sorts them, then the
      // first `capacity` of them (host stack memory, 16 KB)
      ftgemm_fault_record v[kNoallocRecords];
      NA_CK(cudaMemcpyAsync(v, recs, sizeof(ftgemm_fault_record) * have, cudaMemcpyDeviceToHost, st));
      NA_CK(cudaStreamSynchronize(st));
      std::sort(v, v + have, record_before);
      memcpy(report->records, v, sizeof(ftgemm_fault_record) * w);
    }
    report->detected = (int64_t)r.detected;
    report->corrected = (int64_t)r.corrected;
    report->uncorrectable = (int64_t)r.uncorrectable;
    report->checksum_only = (int64_t)r.checksum_only;
    report->n_records = r.n_records;
    report->overflow = (r.n_records > w) ? 1 : 0;
    if (r.timeouts > 0) {
      NA_CK(cudaMemsetAsync(&rep->timeouts, 0, sizeof(int), st));
      NA_CK(cudaStreamSynchronize(st));
      return fail(FTGEMM_ERR_TIMEOUT, "%d bounded device waits gave up (this call or an earlier one "
                  "without a report)", r.timeouts);
    }
  }
#undef NA_CK
  return FTGEMM_OK;
}
