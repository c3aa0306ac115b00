// selftest.cu -- self-test of the bounded device waits (no counterpart in
// the paper).
//
// Every wait of the GEMM kernels on an mbarrier gives up after a time limit,
// records the give-up in the report and lets the kernel return, so that a
// lost TMA transaction or MMA completion ends in an error status instead of
// a hung GPU.  This kernel exercises that path on purpose and safely: it
// waits on a barrier nothing will ever arrive on, with a short limit.
#include "internal.cuh"
#include "ptx.cuh"

namespace ftg {

__global__ void wait_selftest_kernel(DevReport* rep, long long limit_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing arrives: phase 0 never completes
    if (!mbar_wait_limit(&bar, 0u, limit_cycles)) atomicAdd(&rep->timeouts, 1);
  }
  __syncthreads();
}

cudaError_t launch_wait_selftest(DevReport* rep, long long limit_cycles, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(rep, limit_cycles);
  return cudaGetLastError();
}

}  // namespace ftg
