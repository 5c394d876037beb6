// k_decode.cu - DECOMPRESS of Fig. 1: X_t = s1_t(i) s2_t(j) c_t[(h1_t(i) +
// h2_t(j)) mod b], estimate = median over t (even d: mean of the two middle
// values).  Also the element-wise merge of partial sketches (linearity of
// the sketch in the outer products of eq. (1)).
#include <algorithm>
#include <cmath>

#include "cms_internal.h"

namespace cms {
namespace {

__device__ uint32_t g_decode_error = 0;   // set when a pair index is out of range

// Median of x[0..d) (d <= kMaxD): insertion sort in a per-thread array.
template <typename T>
__device__ __forceinline__ T median_of(T* x, int d) {
  for (int a = 1; a < d; ++a) {
    const T v = x[a];
    int q = a - 1;
    while (q >= 0 && x[q] > v) { x[q + 1] = x[q]; --q; }
    x[q + 1] = v;
  }
  const int mid = d >> 1;
  return (d & 1) ? x[mid] : static_cast<T>(0.5) * (x[mid - 1] + x[mid]);
}

// The same estimate for a compile-time d: the d values stay in registers
// and are sorted by odd-even transposition (d rounds of compare-exchange,
// the order an insertion sort gives for the same values).
template <typename T, int D>
__device__ __forceinline__ T estimate_fixed(const T* __restrict__ c, const uint32_t* __restrict__ hs,
                                            int64_t n, uint32_t b, int64_t i, int64_t j) {
  T x[D];
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const uint32_t wa = __ldg(hs + (static_cast<size_t>(2 * t) * n + i));
    const uint32_t wb = __ldg(hs + (static_cast<size_t>(2 * t + 1) * n + j));
    uint32_t z = (wa & kBucketMask) + (wb & kBucketMask);
    if (z >= b) z -= b;
    T v = __ldg(c + static_cast<size_t>(t) * b + z);
    if ((wa ^ wb) >> 31) v = -v;
    x[t] = v;
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int a = r & 1; a + 1 < D; a += 2) {
      const T lo = x[a], hi = x[a + 1];
      const bool sw = lo > hi;
      x[a] = sw ? hi : lo;
      x[a + 1] = sw ? lo : hi;
    }
  }
  constexpr int mid = D >> 1;
  return (D & 1) ? x[mid] : static_cast<T>(0.5) * (x[mid - 1] + x[mid]);
}

template <typename T>
__device__ __forceinline__ T estimate(const T* __restrict__ c, const uint32_t* __restrict__ hs,
                                      int64_t n, uint32_t b, int d, int64_t i, int64_t j) {
  switch (d) {
    case 1: return estimate_fixed<T, 1>(c, hs, n, b, i, j);
    case 2: return estimate_fixed<T, 2>(c, hs, n, b, i, j);
    case 3: return estimate_fixed<T, 3>(c, hs, n, b, i, j);
    case 4: return estimate_fixed<T, 4>(c, hs, n, b, i, j);
    case 5: return estimate_fixed<T, 5>(c, hs, n, b, i, j);
    case 6: return estimate_fixed<T, 6>(c, hs, n, b, i, j);
    case 7: return estimate_fixed<T, 7>(c, hs, n, b, i, j);
    case 8: return estimate_fixed<T, 8>(c, hs, n, b, i, j);
    default: break;
  }
  T x[kMaxD];
  for (int t = 0; t < d; ++t) {
    const uint32_t wa = __ldg(hs + (static_cast<size_t>(2 * t) * n + i));
    const uint32_t wb = __ldg(hs + (static_cast<size_t>(2 * t + 1) * n + j));
    uint32_t z = (wa & kBucketMask) + (wb & kBucketMask);
    if (z >= b) z -= b;
    T v = __ldg(c + static_cast<size_t>(t) * b + z);
    if ((wa ^ wb) >> 31) v = -v;
    x[t] = v;
  }
  return median_of(x, d);
}

template <typename T>
__global__ void k_decode_pairs(const T* __restrict__ c, const uint32_t* __restrict__ hs,
                               int64_t n, uint32_t b, int d, const int64_t* __restrict__ ij,
                               int64_t q, T* __restrict__ out) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= q) return;
  const int64_t i = ij[2 * p], j = ij[2 * p + 1];
  if (i < 0 || i >= n || j < 0 || j >= n) {
    out[p] = static_cast<T>(NAN);
    atomicOr(&g_decode_error, 1u);
    return;
  }
  out[p] = estimate(c, hs, n, b, d, i, j);
}

template <typename T>
__global__ void k_decode_dense(const T* __restrict__ c, const uint32_t* __restrict__ hs,
                               int64_t n, uint32_t b, int d, int64_t n1, int64_t n3,
                               T* __restrict__ out, int64_t ldo) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t i = blockIdx.y; i < n1; i += gridDim.y) {
    if (j < n3) out[i * ldo + j] = estimate(c, hs, n, b, d, i, j);
  }
}

// Thresholded decode (Fig. 2: the approximation is thresholded into a short
// list of candidates): pass 1 counts, per row i, the j with
// |estimate(i, j)| > tau (i != j when skip_diagonal); pass 2 turns the
// counts into row offsets; pass 3 recomputes the estimates and writes the
// hits of row i in increasing j from its offset (row-major order overall,
// independent of scheduling).
__device__ __forceinline__ bool thresh_hit(float v, float tau, int skip, int64_t i, int64_t j) {
  return fabsf(v) > tau && !(skip && i == j);
}

__global__ void __launch_bounds__(256)
k_thresh_count(const float* __restrict__ c, const uint32_t* __restrict__ hs, int64_t n, uint32_t b, int d,
               int64_t n1, int64_t n3, float tau, int skip, int64_t* __restrict__ rowcnt) {
  __shared__ int64_t part[8];
  for (int64_t i = blockIdx.x; i < n1; i += gridDim.x) {
    int64_t cnt = 0;
    for (int64_t j = threadIdx.x; j < n3; j += blockDim.x)
      cnt += thresh_hit(estimate(c, hs, n, b, d, i, j), tau, skip, i, j) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t s = 0;
      for (int w = 0; w < 8; ++w) s += part[w];
      rowcnt[i] = s;
    }
    __syncthreads();
  }
}

// exclusive scan of rowcnt[0..n1) in place; rowcnt[n1] and *total get the sum
__global__ void __launch_bounds__(1024) k_thresh_scan(int64_t* __restrict__ rowcnt, int64_t n1,
                                                      int64_t* __restrict__ total) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t running;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) running = 0;
  __syncthreads();
  for (int64_t base = 0; base < n1; base += 1024) {
    const int64_t i = base + tid;
    const int64_t v = i < n1 ? rowcnt[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (i < n1) rowcnt[i] = running + before + x - v;
    __syncthreads();
    if (tid == 0) {
      int64_t s = 0;
      for (int w = 0; w < 32; ++w) s += wsum[w];
      running += s;
    }
    __syncthreads();
  }
  if (tid == 0) {
    rowcnt[n1] = running;
    *total = running;
  }
}

__global__ void __launch_bounds__(256)
k_thresh_write(const float* __restrict__ c, const uint32_t* __restrict__ hs, int64_t n, uint32_t b, int d,
               int64_t n1, int64_t n3, float tau, int skip, const int64_t* __restrict__ rowoff,
               int64_t capacity, int64_t* __restrict__ ij, float* __restrict__ val) {
  __shared__ int wcnt[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n1; i += gridDim.x) {
    if (rowoff[i] == rowoff[i + 1]) continue;   // uniform over the block
    int64_t pos = rowoff[i];
    for (int64_t j0 = 0; j0 < n3; j0 += blockDim.x) {
      const int64_t j = j0 + threadIdx.x;
      float v = 0.f;
      bool hit = false;
      if (j < n3) {
        v = estimate(c, hs, n, b, d, i, j);
        hit = thresh_hit(v, tau, skip, i, j);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) wcnt[warp] = __popc(bal);
      __syncthreads();
      int64_t before = 0, tot = 0;
      for (int w = 0; w < 8; ++w) {
        if (w < warp) before += wcnt[w];
        tot += wcnt[w];
      }
      if (hit) {
        const int64_t q = pos + before + __popc(bal & ((1u << lane) - 1u));
        if (q < capacity) {
          ij[2 * q] = i;
          ij[2 * q + 1] = j;
          val[q] = v;
        }
      }
      pos += tot;
      __syncthreads();
    }
  }
}

struct PartPtrs {
  const float* p[32];
};

__global__ void k_merge(PartPtrs parts, int count, int64_t len, int accumulate,
                        float* __restrict__ out) {
  for (int64_t z = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; z < len;
       z += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = accumulate ? out[z] : 0.f;
    for (int q = 0; q < count; ++q) s += parts.p[q][z];
    out[z] = s;
  }
}

}  // namespace

uint32_t read_clear_error_decode() {
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_decode_error, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) cudaMemcpyToSymbol(g_decode_error, &zero, sizeof(zero));
  return v;
}

cudaError_t launch_decode_pairs_f32(const float* c, const cms_hashes* h, const int64_t* ij,
                                    int64_t q, float* out, cudaStream_t s) {
  if (q == 0) return cudaSuccess;
  {
    ProfScope prof_scope("k_decode_pairs", s);
    k_decode_pairs<float><<<static_cast<unsigned>((q + 255) / 256), 256, 0, s>>>(
        c, h->d_hs, h->n, static_cast<uint32_t>(h->b), h->d, ij, q, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode_pairs_f64(const double* c, const cms_hashes* h, const int64_t* ij,
                                    int64_t q, double* out, cudaStream_t s) {
  if (q == 0) return cudaSuccess;
  {
    ProfScope prof_scope("k_decode_pairs_f64", s);
    k_decode_pairs<double><<<static_cast<unsigned>((q + 255) / 256), 256, 0, s>>>(
        c, h->d_hs, h->n, static_cast<uint32_t>(h->b), h->d, ij, q, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode_dense_f32(const float* c, const cms_hashes* h, int64_t n1, int64_t n3,
                                    float* out, int64_t ldo, cudaStream_t s) {
  if (n1 == 0 || n3 == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>((n3 + 255) / 256),
            static_cast<unsigned>(std::min<int64_t>(n1, 65535)));
  {
    ProfScope prof_scope("k_decode_dense", s);
    k_decode_dense<float><<<grid, 256, 0, s>>>(c, h->d_hs, h->n, static_cast<uint32_t>(h->b), h->d,
                                               n1, n3, out, ldo);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode_threshold(const float* c, const cms_hashes* h, int64_t n1, int64_t n3, float tau,
                                    int skip_diagonal, int64_t* ij, float* val, int64_t capacity,
                                    int64_t* count, int64_t* rowcnt, cudaStream_t s) {
  if (n1 == 0 || n3 == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(n1, 65535));
  const uint32_t b = static_cast<uint32_t>(h->b);
  {
    ProfScope prof_scope("k_thresh_count", s);
    k_thresh_count<<<grid, 256, 0, s>>>(c, h->d_hs, h->n, b, h->d, n1, n3, tau, skip_diagonal, rowcnt);
  }
  {
    ProfScope prof_scope("k_thresh_scan", s);
    k_thresh_scan<<<1, 1024, 0, s>>>(rowcnt, n1, count);
  }
  {
    ProfScope prof_scope("k_thresh_write", s);
    k_thresh_write<<<grid, 256, 0, s>>>(c, h->d_hs, h->n, b, h->d, n1, n3, tau, skip_diagonal, rowcnt,
                                        capacity, ij, val);
  }
  return cudaGetLastError();
}

cudaError_t launch_merge(const float* const* parts, int count, int64_t len, float* out,
                         cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((len + 255) / 256, 4096));
  if (count == 0) return cudaMemsetAsync(out, 0, static_cast<size_t>(len) * sizeof(float), s);
  for (int base = 0; base < count; base += 32) {
    PartPtrs pp{};
    const int m = std::min(32, count - base);
    for (int q = 0; q < m; ++q) pp.p[q] = parts[base + q];
    {
      ProfScope prof_scope("k_merge", s);
      k_merge<<<blocks, 256, 0, s>>>(pp, m, len, base > 0 ? 1 : 0, out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cms
