// k_post.cu - covariance post-step of Sec. 3.2: the sketch of Q~, the
// product with its diagonal set to zero, from the sketch of the product.
// Entry (i, i) of AB enters the sketch of repetition t at bucket
// (h1_t(i) + h2_t(i)) mod b with sign s1_t(i) s2_t(i) (the decomposed
// splitting and sign functions of Sec. 2.2), so removing it is one
// subtraction per (i, t).  (AB)_ii = sum_k A_ik B_ki is formed in FP64: a
// block owns 32 consecutive i and its 32 warps take the inner indices
// k = w, w + 32, ... (A read down its columns, A_ik at A[k lda + i], and B
// along its rows, B_ki at B[k ldb + i]: 32 consecutive i per warp load), then
// the 32 partial sums of each i are added in warp order.
#include <algorithm>

#include "cms_internal.h"
#include "sketch_generic.cuh"

namespace cms {
namespace {

template <typename T> __device__ __forceinline__ double to_f64(T v) { return static_cast<double>(v); }
template <> __device__ __forceinline__ double to_f64<__nv_bfloat16>(__nv_bfloat16 v) {
  return static_cast<double>(__bfloat162float(v));
}

template <typename T>
__global__ void __launch_bounds__(1024)
k_remove_diagonal(const T* __restrict__ A, int64_t lda, const T* __restrict__ B, int64_t ldb, int64_t m,
                  int64_t n2, const uint32_t* __restrict__ hs, int64_t n, int d, int64_t b,
                  float* __restrict__ c) {
  __shared__ double part[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * 32 + lane;
  double s = 0.0;
  if (i < m) {
#pragma unroll 4
    for (int64_t k = w; k < n2; k += 32) s = fma(to_f64(A[k * lda + i]), to_f64(B[k * ldb + i]), s);
  }
  part[w][lane] = s;
  __syncthreads();
  if (w != 0 || i >= m) return;
  double diag = 0.0;
  for (int q = 0; q < 32; ++q) diag += part[q][lane];
  for (int t = 0; t < d; ++t) {
    const uint32_t w1 = hs[(static_cast<size_t>(t) * 2 + 0) * n + i];
    const uint32_t w2 = hs[(static_cast<size_t>(t) * 2 + 1) * n + i];
    uint64_t z = static_cast<uint64_t>(w1 & kBucketMask) + (w2 & kBucketMask);
    if (z >= static_cast<uint64_t>(b)) z -= static_cast<uint64_t>(b);
    const double sv = ((w1 ^ w2) >> 31) ? -diag : diag;
    atomicAdd(&c[static_cast<size_t>(t) * b + z], static_cast<float>(-sv));
  }
}

}  // namespace

cudaError_t launch_remove_diagonal(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                                   int64_t n3, int dt, const cms_hashes* h, float* c, cudaStream_t s) {
  const int64_t m = std::min(n1, n3);
  if (m == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((m + 31) / 32);
  ProfScope prof_scope("k_remove_diagonal", s);
  switch (dt) {
    case CMS_F32:
      k_remove_diagonal<float><<<grid, 1024, 0, s>>>(static_cast<const float*>(A), lda, static_cast<const float*>(B),
                                                    ldb, m, n2, h->d_hs, h->n, h->d, h->b, c);
      break;
    case CMS_BF16:
      k_remove_diagonal<__nv_bfloat16><<<grid, 1024, 0, s>>>(static_cast<const __nv_bfloat16*>(A), lda,
                                                            static_cast<const __nv_bfloat16*>(B), ldb, m, n2,
                                                            h->d_hs, h->n, h->d, h->b, c);
      break;
    default:
      k_remove_diagonal<double><<<grid, 1024, 0, s>>>(static_cast<const double*>(A), lda, static_cast<const double*>(B),
                                                     ldb, m, n2, h->d_hs, h->n, h->d, h->b, c);
      break;
  }
  return cudaGetLastError();
}

}  // namespace cms
