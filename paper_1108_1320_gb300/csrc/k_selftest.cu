// k_selftest.cu - self-test of the library's failure detection: every wait
// a kernel makes on another agent (a TMA copy landing in an mbarrier phase)
// is bounded, and a wait that gives up is reported to the host instead of
// hanging the device.  Here one thread waits, with the same bounded wait the
// sketch kernels use, on an mbarrier phase that nothing completes (no thread
// arrives and no copy is issued); the wait gives up after its limit and the
// kernel records that, which the host reads back.
#include "cms_internal.h"
#include "warp_fft.cuh"

namespace cms {
namespace {

// 0: not run, 1: the wait gave up (the designed outcome), 2: it completed
__device__ uint32_t g_selftest_word = 0;

__global__ void k_selftest_wait() {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    wfft::mbar_init(&bar, 1);
    // phase 0 of a fresh barrier with one expected arrival: it completes
    // only on an arrival, and none is made
    const bool done = wfft::mbar_wait_bounded(&bar, 0);
    g_selftest_word = done ? 2u : 1u;
    wfft::mbar_inval(&bar);
  }
}

}  // namespace

cudaError_t run_selftest_wait(cudaStream_t s, uint32_t* outcome) {
  const uint32_t zero = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_selftest_word, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof_scope("k_selftest_wait", s);
    k_selftest_wait<<<1, 32, 0, s>>>();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyFromSymbolAsync(outcome, g_selftest_word, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace cms
