// cms_noalloc.cu - cms_sketch_product_noalloc: the fused sketch with its
// scratch memory in a fixed, library-owned device array instead of a
// caller-provided workspace.
//
// Some callers cannot call cudaMalloc or hand the library a workspace
// buffer: code embedded in a host application whose own allocator owns all
// device memory (a database extension, a plug-in inside a serving process),
// or code on a path that must not allocate because cudaMalloc/cudaFree may
// synchronise the device and their latency is unbounded.  This entry point
// lets them compute a sketch with only their inputs and output.
//
// The scratch is one file-scope device array of kNoallocScratchBytes.  Every
// GPU that loads this library holds it until the process exits.  All calls
// on a device share it and it keeps the last call's contents; nothing in it
// has to start at zero (each call writes every scratch byte it later
// reads), but two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it and give wrong results.
#include <mutex>
#include <vector>

#include "cms_internal.h"

namespace cms {
namespace {

constexpr size_t kNoallocScratchBytes = 32u << 20;   // 32 MiB

// Host code must not use this name as a device address: on the host it is a
// stand-in.  Its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct ScratchAddr {
  bool ready = false;
  void* ptr = nullptr;
};

std::mutex g_noalloc_mu;
std::vector<ScratchAddr> g_noalloc_addr;   // one per device ordinal

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev >= static_cast<int>(g_noalloc_addr.size())) g_noalloc_addr.resize(dev + 1);
  ScratchAddr& s = g_noalloc_addr[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    s.ptr = p;
    s.ready = true;
  }
  *out = s.ptr;
  return cudaSuccess;
}

}  // namespace
}  // namespace cms

using namespace cms;

extern "C" {

cms_status cms_sketch_product_noalloc(const void* A, int64_t lda, const void* B, int64_t ldb,
                                      int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                      const cms_hashes* h, float* c, void* stream) {
  const int chk = check_dense_call(h, A, lda, B, ldb, n1, n2, n3, dt, c);
  if (chk != CMS_OK) return static_cast<cms_status>(chk);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return CMS_ERR_CUDA; }
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  SketchPlan plan;
  std::string why;
  const int r = make_sketch_plan(h, n1, n2, n3, dt, sms > 0 ? sms : 1,
                                 optin > 0 ? static_cast<size_t>(optin) : 48 * 1024, &plan, &why,
                                 A, lda, B, ldb);
  if (r != CMS_OK) { set_error(why); return static_cast<cms_status>(r); }
  if (plan.ws_bytes > kNoallocScratchBytes) {
    set_error("cms_sketch_product_noalloc: this shape needs " + std::to_string(plan.ws_bytes) +
              " bytes of scratch, above the fixed " + std::to_string(kNoallocScratchBytes) +
              "-byte array; use cms_sketch_product with a workspace");
    return CMS_ERR_WORKSPACE;
  }
  void* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    return CMS_ERR_CUDA;
  }
  e = launch_sketch(plan, h, A, lda, B, ldb, n1, n2, n3, dt, c, static_cast<char*>(scratch),
                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_error(std::string("cms_sketch_product_noalloc: ") + cudaGetErrorString(e));
    return CMS_ERR_CUDA;
  }
  return CMS_OK;
}

}  // extern "C"
