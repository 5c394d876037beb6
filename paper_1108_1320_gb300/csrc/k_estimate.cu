// k_estimate.cu - Sec. 5.2: an upper bound on ||AB||_F from AMS sketches of
// AB.  The AMS sketch of AB with sign functions s1, s2 is
//   X = sum_ij s1(i) s2(j) (AB)_ij = sum_k (sum_i s1(i) A_ik)(sum_j B_kj s2(j)),
// the sum of the AMS sketches of the outer products (Sec. 2.1); with 4-wise
// independent s1, s2 the square X^2 is an unbiased estimate of ||AB||_F^2
// with variance at most 8 E[X^2]^2, and 32 times the median of d squares
// bounds ||AB||_F^2 from above with high probability.
//
// Signs: s(x) = 1 - 2 (((a3 x^3 + a2 x^2 + a1 x + a0) mod p) mod 2),
// p = 2^31 - 1, coefficients r mod p drawn with splitmix64 from the seed in
// the order (t, s1 then s2, a0..a3).  Tables of the signs are built once
// (d (n1 + n3) bytes), then one block per inner index k forms
// u_t = sum_i s1_t(i) A_ik and v_t = sum_j s2_t(j) B_kj in FP64 and stores
// u_t v_t; a fixed-order sum over k gives X_t.
#include <algorithm>

#include "cms_internal.h"

namespace cms {
namespace {

struct Sign4Coeffs {
  uint32_t v[kMaxD][8];   // [t][s1 a0..a3, s2 a0..a3]
};

uint64_t sm64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_sign4_tables(Sign4Coeffs co, int d, int64_t n1, int64_t n3, int8_t* __restrict__ s1,
                               int8_t* __restrict__ s2) {
  const int t = blockIdx.y;
  const int side = blockIdx.z;
  const int64_t ns = side ? n3 : n1;
  int8_t* out = (side ? s2 : s1) + static_cast<size_t>(t) * ns;
  const uint32_t* a = co.v[t] + 4 * side;
  for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < ns;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint64_t xv = static_cast<uint64_t>(x);
    uint32_t v = a[3];
    v = mod_p31(static_cast<uint64_t>(v) * xv + a[2]);
    v = mod_p31(static_cast<uint64_t>(v) * xv + a[1]);
    v = mod_p31(static_cast<uint64_t>(v) * xv + a[0]);
    out[x] = (v & 1u) ? static_cast<int8_t>(-1) : static_cast<int8_t>(1);
  }
}

template <typename T> __device__ __forceinline__ double to_f64e(T v) { return static_cast<double>(v); }
template <> __device__ __forceinline__ double to_f64e<__nv_bfloat16>(__nv_bfloat16 v) {
  return static_cast<double>(__bfloat162float(v));
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;   // valid in thread 0
}

// one block per inner index k: P[t][k] = (sum_i s1_t(i) A_ik)(sum_j s2_t(j) B_kj)
template <typename T>
__global__ void __launch_bounds__(256)
k_ams_rows(const T* __restrict__ A, int64_t lda, const T* __restrict__ B, int64_t ldb, int64_t n1, int64_t n2,
           int64_t n3, int d, const int8_t* __restrict__ s1, const int8_t* __restrict__ s2,
           double* __restrict__ P) {
  __shared__ double red[8];
  for (int64_t k = blockIdx.x; k < n2; k += gridDim.x) {
    const T* a = A + k * lda;   // A_ik at a[i]
    const T* b = B + k * ldb;   // B_kj at b[j]
    for (int t = 0; t < d; ++t) {
      double u = 0.0, v = 0.0;
      const int8_t* sa = s1 + static_cast<size_t>(t) * n1;
      const int8_t* sb = s2 + static_cast<size_t>(t) * n3;
      for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) u += sa[i] * to_f64e(a[i]);
      for (int64_t j = threadIdx.x; j < n3; j += blockDim.x) v += sb[j] * to_f64e(b[j]);
      u = block_sum(u, red);
      v = block_sum(v, red);
      if (threadIdx.x == 0) P[static_cast<size_t>(t) * n2 + k] = u * v;
    }
  }
}

// X_t = sum_k P[t][k] (fixed order: strided partial sums, then a tree)
__global__ void __launch_bounds__(256) k_ams_reduce(const double* __restrict__ P, int64_t n2,
                                                    double* __restrict__ est) {
  __shared__ double red[8];
  const int t = blockIdx.x;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n2; k += blockDim.x) s += P[static_cast<size_t>(t) * n2 + k];
  s = block_sum(s, red);
  if (threadIdx.x == 0) est[t] = s;
}

// bound = 32 median_t X_t^2 (even d: mean of the two middle squares)
__global__ void k_ams_bound(const double* __restrict__ est, int d, double* __restrict__ bound) {
  double sq[kMaxD];
  for (int t = 0; t < d; ++t) sq[t] = est[t] * est[t];
  for (int a = 1; a < d; ++a) {
    const double v = sq[a];
    int q = a - 1;
    while (q >= 0 && sq[q] > v) { sq[q + 1] = sq[q]; --q; }
    sq[q + 1] = v;
  }
  const int mid = d >> 1;
  *bound = 32.0 * ((d & 1) ? sq[mid] : 0.5 * (sq[mid - 1] + sq[mid]));
}

size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// ---------------------------------------------------------------------------
// Sec. 5.1: one step of the doubling search for the number of nonzeros of AB.
// The sketch of (D1 A)(B D2) with random diagonal scalings D1, D2 (values in
// [1, 2) from two splitmix64 streams indexed by i and j), so that a bucket
// sum vanishes (whp, Schwartz-Zippel) only when every entry of AB hashed to
// it is zero.  Every term s1(i) s2(j) D1_i D2_j A_ik B_kj of every nonempty
// inner index is added to its bucket in FP64, its magnitude to a second
// accumulator; a bucket counts as zero when |sum| <= 1e-9 (sum of |terms|)
// (exact cancellation inside an entry of AB leaves only FP64 rounding).
// Splitting and sign functions: those of Fig. 1 drawn from the seed, with
// range b.
__device__ __forceinline__ double unit_scale(uint64_t stream, uint64_t idx) {
  uint64_t z = stream + (idx + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return 1.0 + static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_nnz_scatter(const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const T* __restrict__ a_val,
              const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_idx, const T* __restrict__ b_val,
              int n1, int n3, int64_t n2, Coeffs co, int d, uint32_t b, uint64_t seed, double* __restrict__ cd,
              double* __restrict__ ca) {
  for (int64_t k = blockIdx.x; k < n2; k += gridDim.x) {
    const int64_t a0 = a_ptr[k], na = a_ptr[k + 1] - a0;
    const int64_t b0 = b_ptr[k], nb = b_ptr[k + 1] - b0;
    if (na <= 0 || nb <= 0) continue;
    for (int64_t pr = threadIdx.x; pr < na * nb; pr += blockDim.x) {
      const int64_t ia = a0 + pr / nb, jb = b0 + pr % nb;
      const int i = a_idx[ia], j = b_idx[jb];
      if (i < 0 || i >= n1 || j < 0 || j >= n3) continue;
      const double v = unit_scale(seed ^ 0xA5A5A5A5A5A5A5A5ULL, static_cast<uint64_t>(i)) *
                       unit_scale(seed ^ 0x5A5A5A5A5A5A5A5AULL, static_cast<uint64_t>(j)) *
                       to_f64e(a_val[ia]) * to_f64e(b_val[jb]);
      for (int t = 0; t < d; ++t) {
        const uint32_t* c = co.v[t];
        const uint32_t h1 = poly_p31(c[0], c[1], static_cast<uint32_t>(i)) % b;
        const uint32_t g1 = poly_p31(c[2], c[3], static_cast<uint32_t>(i)) & 1u;
        const uint32_t h2 = poly_p31(c[4], c[5], static_cast<uint32_t>(j)) % b;
        const uint32_t g2 = poly_p31(c[6], c[7], static_cast<uint32_t>(j)) & 1u;
        uint32_t z = h1 + h2;
        if (z >= b) z -= b;
        atomicAdd(&cd[static_cast<size_t>(t) * b + z], (g1 ^ g2) ? -v : v);
        atomicAdd(&ca[static_cast<size_t>(t) * b + z], fabs(v));
      }
    }
  }
}

__global__ void __launch_bounds__(256)
k_nnz_count(const double* __restrict__ cd, const double* __restrict__ ca, uint32_t b,
            unsigned long long* __restrict__ cnt) {
  __shared__ unsigned int part[8];
  const int t = blockIdx.y;
  unsigned int c = 0;
  for (uint32_t z = blockIdx.x * blockDim.x + threadIdx.x; z < b; z += gridDim.x * blockDim.x) {
    const double s = cd[static_cast<size_t>(t) * b + z], m = ca[static_cast<size_t>(t) * b + z];
    c += (m > 0.0 && fabs(s) > 1e-9 * m) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int w = 0; w < 8; ++w) sum += part[w];
    atomicAdd(&cnt[t], sum);
  }
}

}  // namespace

size_t frobenius_ws_bytes(int64_t n1, int64_t n2, int64_t n3, int d) {
  return al256(static_cast<size_t>(d) * n1) + al256(static_cast<size_t>(d) * n3) +
         al256(static_cast<size_t>(d) * std::max<int64_t>(n2, 1) * 8);
}

cudaError_t launch_frobenius(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                             int64_t n3, int dt, uint64_t seed, int d, double* est, double* bound, char* ws,
                             cudaStream_t s) {
  Sign4Coeffs co{};
  uint64_t st = seed;
  for (int t = 0; t < d; ++t)
    for (int q = 0; q < 8; ++q) co.v[t][q] = static_cast<uint32_t>(sm64_next(&st) % kP31);
  int8_t* s1 = reinterpret_cast<int8_t*>(ws);
  int8_t* s2 = reinterpret_cast<int8_t*>(ws + al256(static_cast<size_t>(d) * n1));
  double* P = reinterpret_cast<double*>(ws + al256(static_cast<size_t>(d) * n1) + al256(static_cast<size_t>(d) * n3));
  const int64_t nmax = std::max<int64_t>(std::max(n1, n3), 1);
  {
    ProfScope prof_scope("k_sign4_tables", s);
    dim3 g(static_cast<unsigned>(std::min<int64_t>((nmax + 255) / 256, 1024)), d, 2);
    k_sign4_tables<<<g, 256, 0, s>>>(co, d, n1, n3, s1, s2);
  }
  if (n2 > 0) {
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(n2, 65535));
    ProfScope prof_scope("k_ams_rows", s);
    switch (dt) {
      case CMS_F32:
        k_ams_rows<float><<<grid, 256, 0, s>>>(static_cast<const float*>(A), lda, static_cast<const float*>(B), ldb,
                                               n1, n2, n3, d, s1, s2, P);
        break;
      case CMS_BF16:
        k_ams_rows<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(A), lda,
                                                       static_cast<const __nv_bfloat16*>(B), ldb, n1, n2, n3, d, s1,
                                                       s2, P);
        break;
      default:
        k_ams_rows<double><<<grid, 256, 0, s>>>(static_cast<const double*>(A), lda, static_cast<const double*>(B), ldb,
                                                n1, n2, n3, d, s1, s2, P);
        break;
    }
  }
  {
    ProfScope prof_scope("k_ams_reduce", s);
    k_ams_reduce<<<d, 256, 0, s>>>(P, n2, est);
  }
  {
    ProfScope prof_scope("k_ams_bound", s);
    k_ams_bound<<<1, 1, 0, s>>>(est, d, bound);
  }
  return cudaGetLastError();
}

size_t nnz_ws_bytes(int d, int64_t b_max) {
  return 2 * al256(static_cast<size_t>(d) * b_max * 8) + 256;
}

cudaError_t run_nnz_doubling(const SparseArgsHost& in, int dt, int64_t n2, const Coeffs& co, uint64_t seed, int d,
                             int64_t b_max, char* ws, int64_t* b_out, int64_t* worst_out, cudaStream_t s) {
  double* cd = reinterpret_cast<double*>(ws);
  double* ca = reinterpret_cast<double*>(ws + al256(static_cast<size_t>(d) * b_max * 8));
  unsigned long long* cnt =
      reinterpret_cast<unsigned long long*>(ws + 2 * al256(static_cast<size_t>(d) * b_max * 8));
  *b_out = -1;
  *worst_out = 0;
  unsigned long long host[kMaxD];
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(n2, 65535)));
  for (int64_t b = 2; b <= b_max; b *= 2) {
    const size_t bytes = static_cast<size_t>(d) * b * 8;
    cudaError_t e = cudaMemsetAsync(cd, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ca, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, static_cast<size_t>(d) * 8, s);
    if (e != cudaSuccess) return e;
    if (n2 > 0) {
      ProfScope prof_scope("k_nnz_scatter", s);
      const uint32_t bb = static_cast<uint32_t>(b);
      switch (dt) {
        case CMS_F32:
          k_nnz_scatter<float><<<grid, 256, 0, s>>>(in.a_ptr, in.a_idx, static_cast<const float*>(in.a_val), in.b_ptr,
                                                    in.b_idx, static_cast<const float*>(in.b_val), in.n1, in.n3, n2,
                                                    co, d, bb, seed, cd, ca);
          break;
        case CMS_BF16:
          k_nnz_scatter<__nv_bfloat16><<<grid, 256, 0, s>>>(
              in.a_ptr, in.a_idx, static_cast<const __nv_bfloat16*>(in.a_val), in.b_ptr, in.b_idx,
              static_cast<const __nv_bfloat16*>(in.b_val), in.n1, in.n3, n2, co, d, bb, seed, cd, ca);
          break;
        default:
          k_nnz_scatter<double><<<grid, 256, 0, s>>>(in.a_ptr, in.a_idx, static_cast<const double*>(in.a_val),
                                                     in.b_ptr, in.b_idx, static_cast<const double*>(in.b_val), in.n1,
                                                     in.n3, n2, co, d, bb, seed, cd, ca);
          break;
      }
    }
    {
      ProfScope prof_scope("k_nnz_count", s);
      dim3 g(static_cast<unsigned>(std::min<int64_t>((b + 255) / 256, 1024)), d);
      k_nnz_count<<<g, 256, 0, s>>>(cd, ca, static_cast<uint32_t>(b), cnt);
    }
    e = cudaMemcpyAsync(host, cnt, static_cast<size_t>(d) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    int64_t worst = 0;
    for (int t = 0; t < d; ++t) worst = std::max<int64_t>(worst, static_cast<int64_t>(host[t]));
    if (5 * worst <= b) {
      *b_out = b;
      *worst_out = worst;
      return cudaSuccess;
    }
  }
  return cudaSuccess;
}

}  // namespace cms
