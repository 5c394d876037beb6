// cms_api.cu - the C ABI declared in include/cms.h: argument checking,
// the hash-set object, planning, and the launch sequences.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cms_internal.h"

namespace cms {

namespace {
thread_local std::string g_last_error;

// splitmix64 (Steele, Lea, Flood 2014): state += golden gamma, then the
// variant-13 finaliser.
uint64_t splitmix64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Coefficient draw of the hash family: per repetition, (a, c) of h1, s1,
// h2, s2 in that order, a = 1 + (r mod (p-1)), c = r mod p.
void draw_coeffs(uint64_t seed, int d, Coeffs* co) {
  std::memset(co, 0, sizeof(*co));
  uint64_t st = seed;
  for (int t = 0; t < d; ++t) {
    for (int f = 0; f < 4; ++f) {
      const uint64_t ra = splitmix64_next(&st);
      const uint64_t rc = splitmix64_next(&st);
      co->v[t][2 * f + 0] = static_cast<uint32_t>(1 + ra % (kP31 - 1));
      co->v[t][2 * f + 1] = static_cast<uint32_t>(rc % kP31);
    }
  }
}

struct DeviceProps {
  int sms = 0;
  size_t smem_optin = 0;
};

DeviceProps device_props(int dev) {
  static std::mutex mu;
  static std::vector<DeviceProps> cache;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= static_cast<int>(cache.size())) cache.resize(dev + 1);
  if (cache[dev].sms == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev].sms = v > 0 ? v : 1;
    v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cache[dev].smem_optin = v > 0 ? static_cast<size_t>(v) : 48 * 1024;
  }
  return cache[dev];
}

cms_status fail(cms_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

cms_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return CMS_ERR_CUDA;
}

cms_status check_device(const cms_hashes* h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != h->device)
    return fail(CMS_ERR_INVALID_ARG, "current device differs from the device the hashes were made on");
  return CMS_OK;
}

cms_status alloc_tables(cms_hashes* h) {
  const size_t cells = static_cast<size_t>(h->d) * 2 * static_cast<size_t>(h->n);
  cudaError_t e = cudaMalloc(&h->d_hs, cells * sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(hash tables)");
  if (h->C > 0) {
    e = cudaMalloc(&h->d_perm, cells * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(bucket lists)");
    e = cudaMalloc(&h->d_off, static_cast<size_t>(h->d) * 2 * (h->C + 1) * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(bucket offsets)");
  }
  if (fe_pq(h->C, nullptr, nullptr) && h->n <= 65535) {
    h->fe_ecap = static_cast<uint32_t>(h->n + 32 * kFeCap);
    const size_t ts = static_cast<size_t>(h->d) * 2;
    const size_t C = static_cast<size_t>(h->C);
    const size_t groups = (C + 31) / 32;
    if ((e = cudaMalloc(&h->d_fe_x, ts * h->fe_ecap * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_hs, ts * h->fe_ecap * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_grp, ts * groups * 2 * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_dest, ts * groups * 32 * 2)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_ovf_off, ts * (C + 1) * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_ovf_x, ts * h->n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_assign, ts * (kFeC / 32))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_fe_ovf_hs, ts * h->n * 4)) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(front-end records)");
  }
  return CMS_OK;
}

void free_tables(cms_hashes* h) {
  if (h->d_hs) cudaFree(h->d_hs);
  if (h->d_perm) cudaFree(h->d_perm);
  if (h->d_off) cudaFree(h->d_off);
  h->d_hs = h->d_perm = nullptr;
  h->d_off = nullptr;
  for (uint32_t** q : {&h->d_fe_x, &h->d_fe_hs, &h->d_fe_grp, &h->d_fe_ovf_off, &h->d_fe_ovf_x, &h->d_fe_ovf_hs}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  if (h->d_fe_dest) cudaFree(h->d_fe_dest);
  h->d_fe_dest = nullptr;
  if (h->d_fe_assign) cudaFree(h->d_fe_assign);
  h->d_fe_assign = nullptr;

  h->fe_ecap = 0;
}

cms_status fill_tables(cms_hashes* h, cudaStream_t s, bool hash) {
  cudaError_t e = cudaSuccess;
  if (hash) {
    e = launch_hash_tables(h->coef, h->d, h->n, h->b, h->d_hs, s);
    if (e != cudaSuccess) return cuda_fail(e, "hash table kernel");
  }
  if (h->C > 0) {
    e = launch_bucket_sort(h->d_hs, h->d, h->n, h->C, h->d_perm, h->d_off, s);
    if (e != cudaSuccess) return cuda_fail(e, "bucket sort kernel");
  }
  if (h->fe_ecap > 0) {
    e = launch_frontend_tables(h->d_hs, h->d_perm, h->d_off, h->d, h->n, h->C, h->fe_ecap, h->d_fe_x, h->d_fe_hs,
                               h->d_fe_grp, h->d_fe_dest, h->d_fe_ovf_off, h->d_fe_ovf_x, h->d_fe_assign,
                               h->d_fe_ovf_hs, s);
    if (e != cudaSuccess) return cuda_fail(e, "front-end table kernel");
  }
  return CMS_OK;
}

bool valid_dtype(int dt) { return dt == CMS_F32 || dt == CMS_BF16 || dt == CMS_F64; }

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace cms

using namespace cms;

extern "C" {

const char* cms_status_string(cms_status s) {
  switch (s) {
    case CMS_OK: return "CMS_OK";
    case CMS_ERR_INVALID_ARG: return "CMS_ERR_INVALID_ARG";
    case CMS_ERR_UNSUPPORTED: return "CMS_ERR_UNSUPPORTED";
    case CMS_ERR_CUDA: return "CMS_ERR_CUDA";
    case CMS_ERR_WORKSPACE: return "CMS_ERR_WORKSPACE";
    case CMS_ERR_TIMEOUT: return "CMS_ERR_TIMEOUT";
    case CMS_ERR_DEVICE: return "CMS_ERR_DEVICE";
  }
  return "CMS_ERR_UNKNOWN";
}

const char* cms_last_error(void) { return g_last_error.c_str(); }

cms_status cms_make_hashes(uint64_t seed, int64_t n, int64_t b, int32_t d, cms_hashes** out) {
  NvtxRange nvtx_range("cms_make_hashes");
  if (!out) return fail(CMS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > (1LL << 24)) return fail(CMS_ERR_INVALID_ARG, "n must be in [1, 2^24]");
  if (b < 1 || b > (1LL << 24)) return fail(CMS_ERR_INVALID_ARG, "b must be in [1, 2^24]");
  if (d < 1 || d > kMaxD) return fail(CMS_ERR_INVALID_ARG, "d must be in [1, 64]");
  cms_hashes* h = new cms_hashes();
  h->n = n; h->b = b; h->d = d; h->seed = seed;
  choose_factorisation(b, &h->R, &h->C);
  cudaGetDevice(&h->device);
  draw_coeffs(seed, d, &h->coef);
  cms_status st = alloc_tables(h);
  if (st == CMS_OK) st = fill_tables(h, nullptr, true);
  if (st == CMS_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "cms_make_hashes");
  }
  if (st != CMS_OK) { free_tables(h); delete h; return st; }
  *out = h;
  return CMS_OK;
}

cms_status cms_reseed_hashes(cms_hashes* h, uint64_t seed, void* stream) {
  NvtxRange nvtx_range("cms_reseed_hashes");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (h->from_tables) return fail(CMS_ERR_INVALID_ARG, "hashes built from tables cannot be reseeded");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  h->seed = seed;
  draw_coeffs(seed, h->d, &h->coef);
  return fill_tables(h, static_cast<cudaStream_t>(stream), true);
}

cms_status cms_make_hashes_from_tables(int64_t n, int64_t b, int32_t d, const uint32_t* h1,
                                       const int8_t* s1, const uint32_t* h2, const int8_t* s2,
                                       cms_hashes** out) {
  NvtxRange nvtx_range("cms_make_hashes_from_tables");
  if (!out) return fail(CMS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!h1 || !s1 || !h2 || !s2) return fail(CMS_ERR_INVALID_ARG, "table pointer is NULL");
  if (n < 1 || n > (1LL << 24)) return fail(CMS_ERR_INVALID_ARG, "n must be in [1, 2^24]");
  if (b < 1 || b > (1LL << 24)) return fail(CMS_ERR_INVALID_ARG, "b must be in [1, 2^24]");
  if (d < 1 || d > kMaxD) return fail(CMS_ERR_INVALID_ARG, "d must be in [1, 64]");
  std::vector<uint32_t> packed(static_cast<size_t>(d) * 2 * n);
  for (int t = 0; t < d; ++t) {
    for (int64_t x = 0; x < n; ++x) {
      const size_t q = static_cast<size_t>(t) * n + x;
      if (h1[q] >= b || h2[q] >= b) return fail(CMS_ERR_INVALID_ARG, "table bucket >= b");
      if ((s1[q] != 1 && s1[q] != -1) || (s2[q] != 1 && s2[q] != -1))
        return fail(CMS_ERR_INVALID_ARG, "table sign not +-1");
      packed[(static_cast<size_t>(2 * t) * n) + x] = h1[q] | (s1[q] < 0 ? 0x80000000u : 0u);
      packed[(static_cast<size_t>(2 * t + 1) * n) + x] = h2[q] | (s2[q] < 0 ? 0x80000000u : 0u);
    }
  }
  cms_hashes* h = new cms_hashes();
  h->n = n; h->b = b; h->d = d; h->from_tables = true;
  choose_factorisation(b, &h->R, &h->C);
  cudaGetDevice(&h->device);
  cms_status st = alloc_tables(h);
  if (st == CMS_OK) {
    cudaError_t e = cudaMemcpy(h->d_hs, packed.data(), packed.size() * sizeof(uint32_t),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy(tables)");
  }
  if (st == CMS_OK) st = fill_tables(h, nullptr, false);
  if (st == CMS_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "cms_make_hashes_from_tables");
  }
  if (st != CMS_OK) { free_tables(h); delete h; return st; }
  *out = h;
  return CMS_OK;
}

cms_status cms_free_hashes(cms_hashes* h) {
  if (!h) return CMS_OK;
  cudaDeviceSynchronize();
  free_tables(h);
  delete h;
  return CMS_OK;
}

cms_status cms_hashes_info(const cms_hashes* h, int64_t* n, int64_t* b, int32_t* d, int64_t* R,
                           int64_t* C) {
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (n) *n = h->n;
  if (b) *b = h->b;
  if (d) *d = h->d;
  if (R) *R = h->R;
  if (C) *C = h->C;
  return CMS_OK;
}

cms_status cms_hashes_coeffs(const cms_hashes* h, int32_t t, uint32_t out[8]) {
  if (!h || !out) return fail(CMS_ERR_INVALID_ARG, "NULL argument");
  if (t < 0 || t >= h->d) return fail(CMS_ERR_INVALID_ARG, "t out of range");
  for (int q = 0; q < 8; ++q) out[q] = h->coef.v[t][q];
  return CMS_OK;
}

cms_status cms_hashes_tables(const cms_hashes* h, uint32_t* h1, int8_t* s1, uint32_t* h2,
                             int8_t* s2) {
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  std::vector<uint32_t> packed(static_cast<size_t>(h->d) * 2 * h->n);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(packed.data(), h->d_hs, packed.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cms_hashes_tables");
  for (int t = 0; t < h->d; ++t) {
    for (int64_t x = 0; x < h->n; ++x) {
      const size_t q = static_cast<size_t>(t) * h->n + x;
      const uint32_t wa = packed[static_cast<size_t>(2 * t) * h->n + x];
      const uint32_t wb = packed[static_cast<size_t>(2 * t + 1) * h->n + x];
      if (h1) h1[q] = wa & kBucketMask;
      if (s1) s1[q] = (wa >> 31) ? -1 : 1;
      if (h2) h2[q] = wb & kBucketMask;
      if (s2) s2[q] = (wb >> 31) ? -1 : 1;
    }
  }
  return CMS_OK;
}

static cms_status check_shapes(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3,
                               int64_t lda, int64_t ldb) {
  if (n1 < 0 || n2 < 0 || n3 < 0) return fail(CMS_ERR_INVALID_ARG, "negative dimension");
  if (n2 > (1LL << 31) - 1) return fail(CMS_ERR_INVALID_ARG, "n2 too large (inner indices are 32-bit)");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (n1 > h->n || n3 > h->n) return fail(CMS_ERR_INVALID_ARG, "n1 and n3 must be <= the hash domain n");
  if (lda < std::max<int64_t>(n1, 1)) return fail(CMS_ERR_INVALID_ARG, "lda < n1");
  if (ldb < std::max<int64_t>(n3, 1)) return fail(CMS_ERR_INVALID_ARG, "ldb < n3");
  return CMS_OK;
}

}  // extern "C"

namespace cms {
int check_dense_call(const cms_hashes* h, const void* A, int64_t lda, const void* B, int64_t ldb,
                     int64_t n1, int64_t n2, int64_t n3, int32_t dt, const float* c) {
  cms_status st = check_shapes(h, n1, n2, n3, lda, ldb);
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (!c) return fail(CMS_ERR_INVALID_ARG, "c is NULL");
  if (n2 > 0 && ((n1 > 0 && !A) || (n3 > 0 && !B))) return fail(CMS_ERR_INVALID_ARG, "A or B is NULL");
  return check_device(h);
}
}  // namespace cms

extern "C" {

cms_status cms_hashes_buckets(const cms_hashes* h, int32_t t, int32_t side, uint32_t* perm, uint32_t* off) {
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (t < 0 || t >= h->d || side < 0 || side > 1) return fail(CMS_ERR_INVALID_ARG, "t or side out of range");
  if (h->C <= 0 || !h->d_perm || !h->d_off) return fail(CMS_ERR_UNSUPPORTED, "no bucket lists (b is not 5-smooth)");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  const size_t ts = static_cast<size_t>(t) * 2 + static_cast<size_t>(side);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && perm)
    e = cudaMemcpy(perm, h->d_perm + ts * h->n, static_cast<size_t>(h->n) * sizeof(uint32_t),
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && off)
    e = cudaMemcpy(off, h->d_off + ts * (h->C + 1), static_cast<size_t>(h->C + 1) * sizeof(uint32_t),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cms_hashes_buckets");
  return CMS_OK;
}

cms_status cms_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                              size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  cms_status st = check_shapes(h, n1, n2, n3, std::max<int64_t>(n1, 1), std::max<int64_t>(n3, 1));
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  DeviceProps dp = device_props(h->device);
  SketchPlan plan;
  std::string why;
  // the kernel is chosen per call (pointer alignment); cover both plans
  int r = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &plan, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  SketchPlan generic;
  r = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &generic, &why, nullptr, 0, nullptr, 0,
                       false);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  *bytes = std::max(plan.ws_bytes, generic.ws_bytes);
  if (n1 == n3) {
    // A and B the same bytes (A = X^T, B = X): the register-FFT and cluster
    // kernels stage each row once, so their plans can differ from the
    // two-operand one (leading dimensions in whole 16-byte units of FP32
    // and of BF16 cover both storage types)
    const void* same = reinterpret_cast<const void*>(static_cast<uintptr_t>(256));
    for (int64_t unit : {4, 8}) {
      const int64_t ld = std::max<int64_t>((n1 + unit - 1) / unit * unit, unit);
      SketchPlan alias;
      r = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &alias, &why, same, ld, same, ld);
      if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
      *bytes = std::max(*bytes, alias.ws_bytes);
    }
  }
  return CMS_OK;
}

cms_status cms_plan_kernel(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                           int64_t n3, int32_t dt, const cms_hashes* h, int32_t* kernel_out) {
  if (!kernel_out) return fail(CMS_ERR_INVALID_ARG, "kernel_out is NULL");
  cms_status st = check_shapes(h, n1, n2, n3, lda, ldb);
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  DeviceProps dp = device_props(h->device);
  SketchPlan plan;
  std::string why;
  int r = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &plan, &why, A, lda, B, ldb);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  *kernel_out = plan.wide ? CMS_KERNEL_CLUSTER
                          : plan.ws ? CMS_KERNEL_WARP_SPECIALISED
                                    : plan.fast ? (plan.tmem_rec ? CMS_KERNEL_LOCKSTEP_TMEM : CMS_KERNEL_LOCKSTEP)
                                                : CMS_KERNEL_SHARED_MEMORY;
  return CMS_OK;
}

cms_status cms_sketch_product(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                              int64_t n2, int64_t n3, int32_t dt, const cms_hashes* h, float* c,
                              void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_sketch_product");
  cms_status st = static_cast<cms_status>(cms::check_dense_call(h, A, lda, B, ldb, n1, n2, n3, dt, c));
  if (st != CMS_OK) return st;
  DeviceProps dp = device_props(h->device);
  SketchPlan plan;
  std::string why;
  int r = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &plan, &why, A, lda, B, ldb);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  if (!ws || ws_bytes < plan.ws_bytes)
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaError_t e = launch_sketch(plan, h, A, lda, B, ldb, n1, n2, n3, dt, c, static_cast<char*>(ws),
                                static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product");
  return CMS_OK;
}

cms_status cms_sparse_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3,
                                     size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  cms_status st = check_shapes(h, n1, n2, n3, std::max<int64_t>(n1, 1), std::max<int64_t>(n3, 1));
  if (st != CMS_OK) return st;
  DeviceProps dp = device_props(h->device);
  SketchPlan plan;
  size_t off_klist = 0;
  std::string why;
  int r = make_sparse_plan(h, n2, -1, dp.sms, dp.smem_optin, &plan, &off_klist, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  *bytes = plan.ws_bytes;
  return CMS_OK;
}

cms_status cms_sketch_product_csr(const int64_t* a_colptr, const int32_t* a_rowidx, const void* a_val,
                                  const int64_t* b_rowptr, const int32_t* b_colidx, const void* b_val,
                                  int64_t n1, int64_t n2, int64_t n3, int32_t dt, const cms_hashes* h,
                                  float* c, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_sketch_product_csr");
  cms_status st = check_shapes(h, n1, n2, n3, std::max<int64_t>(n1, 1), std::max<int64_t>(n3, 1));
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (!c) return fail(CMS_ERR_INVALID_ARG, "c is NULL");
  if (n2 > 0 && (!a_colptr || !b_rowptr)) return fail(CMS_ERR_INVALID_ARG, "pointer array is NULL");
  if (n2 >= (1LL << 31) - 1) return fail(CMS_ERR_INVALID_ARG, "n2 too large for int32 inner indices");
  st = check_device(h);
  if (st != CMS_OK) return st;
  DeviceProps dp = device_props(h->device);
  SketchPlan worst;
  size_t off_klist = 0;
  std::string why;
  int r = make_sparse_plan(h, n2, -1, dp.sms, dp.smem_optin, &worst, &off_klist, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  if (!ws || ws_bytes < worst.ws_bytes)
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_sparse_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  int32_t* klist = reinterpret_cast<int32_t*>(w + off_klist);
  int32_t* dlist = reinterpret_cast<int32_t*>(w + worst.off_dlist);
  int32_t* counts = dlist + std::max<int64_t>(n2, 1);
  // the list of nonempty inner indices and its length stay on the device:
  // the FFT route runs the plan's worst-case chunking and reads the length
  // there, so the call returns without waiting for the GPU
  cudaError_t e = launch_nonempty_split(a_colptr, b_rowptr, n2, -1, klist, dlist, counts, counts + 2, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product_csr (nonempty inner indices)");
  const SketchPlan& plan = worst;
  float2* partial = reinterpret_cast<float2*>(w + plan.off_partial);
  float2* V = reinterpret_cast<float2*>(w + plan.off_V);
  float2* twC = reinterpret_cast<float2*>(w + plan.off_twC);
  float2* twR = reinterpret_cast<float2*>(w + plan.off_twR);
  SparseArgsHost in{a_colptr, a_rowidx, a_val, b_rowptr, b_colidx, b_val, static_cast<int>(n1),
                    static_cast<int>(n3)};
  e = launch_twiddle_tables(twC, static_cast<int>(plan.C), twR, static_cast<int>(plan.R), s);
  if (e == cudaSuccess) e = launch_sketch_sparse(plan, h, in, dt, klist, counts, 0, partial, s);
  if (e == cudaSuccess) e = launch_inverse(plan, partial, V, twC, twR, c, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product_csr");
  return CMS_OK;
}

cms_status cms_sketch_product_csr_hybrid(const int64_t* a_colptr, const int32_t* a_rowidx, const void* a_val,
                                         const int64_t* b_rowptr, const int32_t* b_colidx, const void* b_val,
                                         int64_t n1, int64_t n2, int64_t n3, int32_t dt, const cms_hashes* h,
                                         int64_t direct_max_pairs, float* c, void* ws, size_t ws_bytes,
                                         void* stream) {
  NvtxRange nvtx_range("cms_sketch_product_csr_hybrid");
  cms_status st = check_shapes(h, n1, n2, n3, std::max<int64_t>(n1, 1), std::max<int64_t>(n3, 1));
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (!c) return fail(CMS_ERR_INVALID_ARG, "c is NULL");
  if (n2 > 0 && (!a_colptr || !b_rowptr)) return fail(CMS_ERR_INVALID_ARG, "pointer array is NULL");
  if (n2 >= (1LL << 31) - 1) return fail(CMS_ERR_INVALID_ARG, "n2 too large for int32 inner indices");
  st = check_device(h);
  if (st != CMS_OK) return st;
  DeviceProps dp = device_props(h->device);
  SketchPlan worst;
  size_t off_klist = 0;
  std::string why;
  int r = make_sparse_plan(h, n2, -1, dp.sms, dp.smem_optin, &worst, &off_klist, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  if (!ws || ws_bytes < worst.ws_bytes)
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_sparse_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  // default split: direct when the outer product has at most 5 b log2(b) / 64
  // terms (the FFT route costs about 5 b log2 b flops per inner index)
  const int64_t limit = direct_max_pairs >= 0
                            ? direct_max_pairs
                            : static_cast<int64_t>(5.0 * static_cast<double>(h->b) *
                                                   std::log2(static_cast<double>(std::max<int64_t>(h->b, 2))) / 64.0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  int32_t* flist = reinterpret_cast<int32_t*>(w + off_klist);
  int32_t* dlist = reinterpret_cast<int32_t*>(w + worst.off_dlist);
  int32_t* counts = dlist + std::max<int64_t>(n2, 1);
  double* cd = reinterpret_cast<double*>(w + worst.off_cd);
  // both lists and their lengths stay on the device (no host wait): the FFT
  // route and the inverse return at once when its list is empty, and the
  // direct scatter strides over the direct list's length
  cudaError_t e = launch_nonempty_split(a_colptr, b_rowptr, n2, limit, flist, dlist, counts, counts + 2, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product_csr_hybrid (inner-index split)");
  const SketchPlan& plan = worst;
  SparseArgsHost in{a_colptr, a_rowidx, a_val, b_rowptr, b_colidx, b_val, static_cast<int>(n1),
                    static_cast<int>(n3)};
  {
    float2* partial = reinterpret_cast<float2*>(w + plan.off_partial);
    float2* V = reinterpret_cast<float2*>(w + plan.off_V);
    float2* twC = reinterpret_cast<float2*>(w + plan.off_twC);
    float2* twR = reinterpret_cast<float2*>(w + plan.off_twR);
    e = launch_twiddle_tables(twC, static_cast<int>(plan.C), twR, static_cast<int>(plan.R), s);
    if (e == cudaSuccess) e = launch_sketch_sparse(plan, h, in, dt, flist, counts, 1, partial, s);
    if (e == cudaSuccess) e = launch_inverse(plan, partial, V, twC, twR, c, s, counts);
  }
  if (e == cudaSuccess) e = launch_direct_scatter(h, in, dt, dlist, counts, n2, cd, s);
  if (e == cudaSuccess) e = launch_add_direct(c, cd, static_cast<int64_t>(h->d) * h->b, counts, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product_csr_hybrid");
  return CMS_OK;
}

cms_status cms_plain_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3,
                                    size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  cms_status st = check_shapes(h, n1, n2, n3, std::max<int64_t>(n1, 1), std::max<int64_t>(n3, 1));
  if (st != CMS_OK) return st;
  PlainPlan plan;
  std::string why;
  int r = make_plain_plan(h, n2, &plan, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  *bytes = plan.ws_bytes;
  return CMS_OK;
}

cms_status cms_sketch_product_plain_f64(const double* A, int64_t lda, const double* B, int64_t ldb,
                                        int64_t n1, int64_t n2, int64_t n3, const cms_hashes* h,
                                        double* c, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_sketch_product_plain_f64");
  cms_status st = check_shapes(h, n1, n2, n3, lda, ldb);
  if (st != CMS_OK) return st;
  if (!c) return fail(CMS_ERR_INVALID_ARG, "c is NULL");
  if (n2 > 0 && ((n1 > 0 && !A) || (n3 > 0 && !B))) return fail(CMS_ERR_INVALID_ARG, "A or B is NULL");
  st = check_device(h);
  if (st != CMS_OK) return st;
  PlainPlan plan;
  std::string why;
  int r = make_plain_plan(h, n2, &plan, &why);
  if (r != CMS_OK) return fail(static_cast<cms_status>(r), why);
  if (!ws || ws_bytes < plan.ws_bytes)
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_plain_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaError_t e = launch_plain(plan, h, A, lda, B, ldb, n1, n2, n3, c, static_cast<char*>(ws),
                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_product_plain_f64");
  return CMS_OK;
}

cms_status cms_decode(const float* c, const cms_hashes* h, const int64_t* ij, int64_t q, float* out,
                      void* stream) {
  NvtxRange nvtx_range("cms_decode");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (q < 0) return fail(CMS_ERR_INVALID_ARG, "q < 0");
  if (q > 0 && (!c || !ij || !out)) return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_decode_pairs_f32(c, h, ij, q, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_decode");
  return CMS_OK;
}

cms_status cms_decode_f64(const double* c, const cms_hashes* h, const int64_t* ij, int64_t q,
                          double* out, void* stream) {
  NvtxRange nvtx_range("cms_decode_f64");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (q < 0) return fail(CMS_ERR_INVALID_ARG, "q < 0");
  if (q > 0 && (!c || !ij || !out)) return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_decode_pairs_f64(c, h, ij, q, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_decode_f64");
  return CMS_OK;
}

cms_status cms_decode_dense(const float* c, const cms_hashes* h, int64_t n1, int64_t n3, float* out,
                            int64_t ldo, void* stream) {
  NvtxRange nvtx_range("cms_decode_dense");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (n1 < 0 || n3 < 0 || n1 > h->n || n3 > h->n) return fail(CMS_ERR_INVALID_ARG, "bad n1 or n3");
  if (ldo < n3) return fail(CMS_ERR_INVALID_ARG, "ldo < n3");
  if (n1 > 0 && n3 > 0 && (!c || !out)) return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_decode_dense_f32(c, h, n1, n3, out, ldo, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_decode_dense");
  return CMS_OK;
}

cms_status cms_sketch_remove_diagonal(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                                      int64_t n2, int64_t n3, int32_t dt, const cms_hashes* h, float* c,
                                      void* stream) {
  NvtxRange nvtx_range("cms_sketch_remove_diagonal");
  cms_status st = check_shapes(h, n1, n2, n3, lda, ldb);
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (!c) return fail(CMS_ERR_INVALID_ARG, "c is NULL");
  if (n2 > 0 && std::min(n1, n3) > 0 && (!A || !B)) return fail(CMS_ERR_INVALID_ARG, "A or B is NULL");
  st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_remove_diagonal(A, lda, B, ldb, n1, n2, n3, dt, h, c, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_sketch_remove_diagonal");
  return CMS_OK;
}

cms_status cms_decode_threshold(const float* c, const cms_hashes* h, int64_t n1, int64_t n3, float tau,
                                int32_t skip_diagonal, int64_t* ij_out, float* val_out, int64_t capacity,
                                int64_t* count_out, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_decode_threshold");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (n1 < 0 || n3 < 0 || n1 > h->n || n3 > h->n) return fail(CMS_ERR_INVALID_ARG, "bad n1 or n3");
  if (capacity < 0) return fail(CMS_ERR_INVALID_ARG, "capacity < 0");
  if (!count_out || (n1 > 0 && n3 > 0 && !c) || (capacity > 0 && (!ij_out || !val_out)))
    return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  if (!(tau >= 0.f)) return fail(CMS_ERR_INVALID_ARG, "tau must be a number >= 0");
  if (!ws || ws_bytes < static_cast<size_t>(n1 + 1) * sizeof(int64_t))
    return fail(CMS_ERR_WORKSPACE, "workspace must hold 8 (n1 + 1) bytes");
  if (reinterpret_cast<uintptr_t>(ws) % 8 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 8-byte aligned");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_decode_threshold(c, h, n1, n3, tau, skip_diagonal ? 1 : 0, ij_out, val_out, capacity,
                                          count_out, static_cast<int64_t*>(ws), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_decode_threshold");
  return CMS_OK;
}

cms_status cms_frobenius_workspace_size(int64_t n1, int64_t n2, int64_t n3, int32_t d, size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  if (n1 < 0 || n2 < 0 || n3 < 0 || d < 1 || d > kMaxD) return fail(CMS_ERR_INVALID_ARG, "bad sizes or d");
  *bytes = frobenius_ws_bytes(n1, n2, n3, d);
  return CMS_OK;
}

cms_status cms_frobenius_estimate(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                                  int64_t n3, int32_t dt, uint64_t seed, int32_t d, double* est_out,
                                  double* bound_out, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_frobenius_estimate");
  if (n1 < 0 || n2 < 0 || n3 < 0 || n1 >= (1LL << 31) || n3 >= (1LL << 31))
    return fail(CMS_ERR_INVALID_ARG, "bad n1, n2 or n3");
  if (d < 1 || d > kMaxD) return fail(CMS_ERR_INVALID_ARG, "d must be in [1, 64]");
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (n2 > 1 && (lda < n1 || ldb < n3)) return fail(CMS_ERR_INVALID_ARG, "lda < n1 or ldb < n3");
  if (!est_out || !bound_out) return fail(CMS_ERR_INVALID_ARG, "est_out or bound_out is NULL");
  if (n2 > 0 && ((n1 > 0 && !A) || (n3 > 0 && !B))) return fail(CMS_ERR_INVALID_ARG, "A or B is NULL");
  if (!ws || ws_bytes < frobenius_ws_bytes(n1, n2, n3, d))
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_frobenius_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaError_t e = launch_frobenius(A, lda, B, ldb, n1, n2, n3, dt, seed, d, est_out, bound_out,
                                   static_cast<char*>(ws), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_frobenius_estimate");
  return CMS_OK;
}

cms_status cms_nnz_workspace_size(int32_t d, int64_t b_max, size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  if (d < 1 || d > kMaxD || b_max < 2 || b_max > (1LL << 30)) return fail(CMS_ERR_INVALID_ARG, "bad d or b_max");
  *bytes = nnz_ws_bytes(d, b_max);
  return CMS_OK;
}

cms_status cms_nnz_estimate(const int64_t* a_colptr, const int32_t* a_rowidx, const void* a_val,
                            const int64_t* b_rowptr, const int32_t* b_colidx, const void* b_val, int64_t n1,
                            int64_t n2, int64_t n3, int32_t dt, uint64_t seed, int32_t d, int64_t b_max,
                            int64_t* b_out, int64_t* buckets_out, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_nnz_estimate");
  if (!b_out || !buckets_out) return fail(CMS_ERR_INVALID_ARG, "b_out or buckets_out is NULL");
  if (n1 < 0 || n2 < 0 || n3 < 0 || n1 >= (1LL << 31) || n3 >= (1LL << 31) || n2 >= (1LL << 31) - 1)
    return fail(CMS_ERR_INVALID_ARG, "bad n1, n2 or n3");
  if (d < 1 || d > kMaxD || b_max < 2 || b_max > (1LL << 30)) return fail(CMS_ERR_INVALID_ARG, "bad d or b_max");
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (n2 > 0 && (!a_colptr || !b_rowptr)) return fail(CMS_ERR_INVALID_ARG, "pointer array is NULL");
  if (!ws || ws_bytes < nnz_ws_bytes(d, b_max))
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_nnz_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  Coeffs co;
  draw_coeffs(seed, d, &co);
  SparseArgsHost in{a_colptr, a_rowidx, a_val, b_rowptr, b_colidx, b_val, static_cast<int>(n1), static_cast<int>(n3)};
  cudaError_t e = run_nnz_doubling(in, dt, n2, co, seed, d, b_max, static_cast<char*>(ws), b_out, buckets_out,
                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_nnz_estimate");
  return CMS_OK;
}

namespace {
// Workspace of cms_find_significant: the sketch path's scratch, one masked
// operand, the 2 l sketches and the decode scratch.
struct SigLayout {
  size_t sk = 0, mask = 0, P = 0, dec = 0, total = 0;
  int ell = 0;
  int64_t ld0 = 0, ld1 = 0;
};

cms_status sig_layout(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3, int32_t dt, int32_t rho,
                      SigLayout* L) {
  auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  size_t sk = 0;
  cms_status st = cms_workspace_size(h, n1, n2, n3, dt, &sk);
  if (st != CMS_OK) return st;
  const size_t esz = dt == CMS_BF16 ? 2 : (dt == CMS_F64 ? 8 : 4);
  L->ell = significant_code_length(n1, n3, rho, nullptr);
  L->ld0 = std::max<int64_t>((n1 + 7) / 8 * 8, 8);
  L->ld1 = std::max<int64_t>((n3 + 7) / 8 * 8, 8);
  size_t o = 0;
  L->sk = o;   o += al(sk);
  L->mask = o; o += al(static_cast<size_t>(std::max(L->ld0, L->ld1)) * std::max<int64_t>(n2, 1) * esz);
  L->P = o;    o += al(static_cast<size_t>(2 * L->ell) * h->d * h->b * sizeof(float));
  L->dec = o;  o += al(significant_decode_ws_bytes(h->d, h->b));
  L->total = o;
  return CMS_OK;
}
}  // namespace

cms_status cms_significant_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                          int32_t rho, size_t* bytes) {
  if (!bytes) return fail(CMS_ERR_INVALID_ARG, "bytes is NULL");
  if (rho < 1 || rho > 8) return fail(CMS_ERR_INVALID_ARG, "rho must be in [1, 8]");
  SigLayout L;
  cms_status st = sig_layout(h, n1, n2, n3, dt, rho, &L);
  if (st != CMS_OK) return st;
  *bytes = L.total;
  return CMS_OK;
}

cms_status cms_decode_significant(const float* sketches, const cms_hashes* h, int64_t n1, int64_t n3, float delta,
                                  int32_t rho, int64_t* ij_out, int64_t capacity, int64_t* count_out, void* ws,
                                  size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("cms_decode_significant");
  if (!h) return fail(CMS_ERR_INVALID_ARG, "hashes is NULL");
  if (n1 < 1 || n3 < 1 || n1 > h->n || n3 > h->n) return fail(CMS_ERR_INVALID_ARG, "bad n1 or n3");
  if (rho < 1 || rho > 8) return fail(CMS_ERR_INVALID_ARG, "rho must be in [1, 8]");
  if (!(delta >= 0.f)) return fail(CMS_ERR_INVALID_ARG, "delta must be a number >= 0");
  if (capacity < 0 || !sketches || !count_out || (capacity > 0 && !ij_out))
    return fail(CMS_ERR_INVALID_ARG, "NULL pointer or capacity < 0");
  if (!ws || ws_bytes < significant_decode_ws_bytes(h->d, h->b))
    return fail(CMS_ERR_WORKSPACE, "workspace smaller than cms_significant_decode_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cms_status st = check_device(h);
  if (st != CMS_OK) return st;
  cudaError_t e = launch_decode_significant(sketches, h, n1, n3, delta, rho, ij_out, capacity, count_out,
                                            static_cast<char*>(ws), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_decode_significant");
  return CMS_OK;
}

cms_status cms_significant_decode_workspace_size(const cms_hashes* h, size_t* bytes) {
  if (!h || !bytes) return fail(CMS_ERR_INVALID_ARG, "NULL argument");
  *bytes = significant_decode_ws_bytes(h->d, h->b);
  return CMS_OK;
}

cms_status cms_find_significant(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                                int64_t n3, int32_t dt, const cms_hashes* h, float delta, int32_t rho,
                                int64_t* ij_out, int64_t capacity, int64_t* count_out, void* ws, size_t ws_bytes,
                                void* stream) {
  NvtxRange nvtx_range("cms_find_significant");
  cms_status st = check_shapes(h, n1, n2, n3, lda, ldb);
  if (st != CMS_OK) return st;
  if (!valid_dtype(dt)) return fail(CMS_ERR_INVALID_ARG, "unknown dtype");
  if (n1 < 1 || n3 < 1) return fail(CMS_ERR_INVALID_ARG, "n1 and n3 must be >= 1");
  if (rho < 1 || rho > 8) return fail(CMS_ERR_INVALID_ARG, "rho must be in [1, 8]");
  if (!(delta >= 0.f)) return fail(CMS_ERR_INVALID_ARG, "delta must be a number >= 0");
  if (capacity < 0 || !count_out || (capacity > 0 && !ij_out)) return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  if (n2 > 0 && (!A || !B)) return fail(CMS_ERR_INVALID_ARG, "A or B is NULL");
  st = check_device(h);
  if (st != CMS_OK) return st;
  SigLayout L;
  st = sig_layout(h, n1, n2, n3, dt, rho, &L);
  if (st != CMS_OK) return st;
  if (!ws || ws_bytes < L.total)
    return fail(CMS_ERR_WORKSPACE, "workspace missing or smaller than cms_significant_workspace_size()");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(CMS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  DeviceProps dp = device_props(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  void* M = w + L.mask;
  float* P = reinterpret_cast<float*>(w + L.P);
  const size_t per = static_cast<size_t>(h->d) * h->b;
  for (int r = 0; r < 2 * L.ell; ++r) {
    const bool side1 = r >= L.ell;
    const int rr = side1 ? r - L.ell : r;
    const void* Ao = side1 ? A : M;
    const void* Bo = side1 ? M : B;
    const int64_t la = side1 ? lda : L.ld0;
    const int64_t lb = side1 ? L.ld1 : ldb;
    cudaError_t e = side1 ? launch_mask_copy(B, ldb, M, L.ld1, n3, n2, rr, rho, dt, s)
                          : launch_mask_copy(A, lda, M, L.ld0, n1, n2, rr, rho, dt, s);
    if (e != cudaSuccess) return cuda_fail(e, "cms_find_significant (mask)");
    SketchPlan plan;
    std::string why;
    int rc = make_sketch_plan(h, n1, n2, n3, dt, dp.sms, dp.smem_optin, &plan, &why, Ao, la, Bo, lb);
    if (rc != CMS_OK) return fail(static_cast<cms_status>(rc), why);
    if (plan.ws_bytes > L.mask - L.sk) return fail(CMS_ERR_WORKSPACE, "internal: sketch scratch too small");
    e = launch_sketch(plan, h, Ao, la, Bo, lb, n1, n2, n3, dt, P + r * per, w + L.sk, s);
    if (e != cudaSuccess) return cuda_fail(e, "cms_find_significant (sketch)");
  }
  cudaError_t e = launch_decode_significant(P, h, n1, n3, delta, rho, ij_out, capacity, count_out, w + L.dec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_find_significant (decode)");
  return CMS_OK;
}

cms_status cms_merge(const float* const* parts, int32_t count, int32_t d, int64_t b, float* c_out,
                     void* stream) {
  NvtxRange nvtx_range("cms_merge");
  if (count < 0 || d < 1 || b < 1) return fail(CMS_ERR_INVALID_ARG, "bad count, d or b");
  if (!c_out || (count > 0 && !parts)) return fail(CMS_ERR_INVALID_ARG, "NULL pointer");
  for (int q = 0; q < count; ++q)
    if (!parts[q]) return fail(CMS_ERR_INVALID_ARG, "NULL part");
  cudaError_t e = launch_merge(parts, count, static_cast<int64_t>(d) * b, c_out,
                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_merge");
  return CMS_OK;
}

cms_status cms_selftest_wait(void* stream) {
  uint32_t outcome = 0;
  const cudaError_t e = run_selftest_wait(static_cast<cudaStream_t>(stream), &outcome);
  if (e != cudaSuccess) return cuda_fail(e, "cms_selftest_wait");
  if (outcome == 1) return fail(CMS_ERR_TIMEOUT, "the bounded wait gave up, as designed");
  return fail(CMS_ERR_DEVICE, "the self-test wait did not give up");
}

cms_status cms_check_async(void* stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cms_check_async");
  const uint32_t w = read_clear_error_decode();
  const uint32_t ws1 = read_clear_error_sketch();
  const uint32_t ws2 = read_clear_error_sketch_ws();
  const uint32_t ws3 = read_clear_error_sketch_wide();
  const uint32_t ws = ws1 | ws2 | ws3;
  if (w == 0xFFFFFFFFu || ws1 == 0xFFFFFFFFu || ws2 == 0xFFFFFFFFu || ws3 == 0xFFFFFFFFu)
    return fail(CMS_ERR_CUDA, "could not read the device error words");
  if (ws) return fail(CMS_ERR_TIMEOUT, "a fused-kernel wait for its TMA copies gave up");
  if (w) return fail(CMS_ERR_DEVICE, "decode saw an index pair outside the hash domain");
  return CMS_OK;
}

}  // extern "C"
