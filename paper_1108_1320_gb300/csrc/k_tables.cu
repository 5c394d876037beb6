// k_tables.cu - device construction of the hash tables (Fig. 1's draws of
// h1, s1, h2, s2, Sec. 2.2 polynomial family) and of the bucket-class lists
// used by the fused sketch kernel's gather front end.
#include "cms_internal.h"

namespace cms {
namespace {

// One thread per (t, side, x): evaluate the splitting and sign polynomials.
__global__ void k_hash_tables(Coeffs co, int d, uint32_t n, uint32_t b,
                              uint32_t* __restrict__ hs) {
  const int ts = blockIdx.y;            // t * 2 + side
  const int t = ts >> 1, side = ts & 1;
  const uint32_t ah = co.v[t][side * 4 + 0], ch = co.v[t][side * 4 + 1];
  const uint32_t as = co.v[t][side * 4 + 2], cs = co.v[t][side * 4 + 3];
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const uint32_t h = poly_p31(ah, ch, x) % b;
    const uint32_t neg = poly_p31(as, cs, x) & 1u;
    hs[static_cast<size_t>(ts) * n + x] = h | (neg << 31);
  }
}

// Stable counting sort of x in {0..n-1} by key (bucket mod C), one block per
// (t, side).  Counts use integer shared atomics (exact); placement walks the
// indices in order, warp by warp, so equal keys keep increasing x: the
// result does not depend on scheduling.
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads)
k_bucket_sort(const uint32_t* __restrict__ hs, uint32_t n, uint32_t C,
              uint32_t* __restrict__ perm, uint32_t* __restrict__ off) {
  extern __shared__ uint32_t sm[];
  uint32_t* cnt = sm;          // C
  const int ts = blockIdx.x;
  const uint32_t* tab = hs + static_cast<size_t>(ts) * n;
  uint32_t* pm = perm + static_cast<size_t>(ts) * n;
  uint32_t* of = off + static_cast<size_t>(ts) * (C + 1);
  for (uint32_t z = threadIdx.x; z < C; z += blockDim.x) cnt[z] = 0;
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < n; x += blockDim.x)
    atomicAdd(&cnt[(tab[x] & kBucketMask) % C], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t z = 0; z < C; ++z) {
      const uint32_t v = cnt[z];
      of[z] = run;
      cnt[z] = run;            // becomes the placement cursor
      run += v;
    }
    of[C] = run;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t x = base + threadIdx.x;
    const bool valid = x < n;
    const uint32_t key = valid ? (tab[x] & kBucketMask) % C : 0xFFFFFFFFu;
    for (int w = 0; w < kSortThreads / 32; ++w) {
      __syncthreads();
      if (warp == w) {
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key);
        if (valid) {
          const uint32_t rank = __popc(grp & lt_mask);
          pm[cnt[key] + rank] = x;
        }
        __syncwarp();
        if (valid && lane == __ffs(grp) - 1) cnt[key] += __popc(grp);
      }
    }
  }
}

}  // namespace

cudaError_t launch_hash_tables(const Coeffs& co, int d, int64_t n, int64_t b,
                               uint32_t* hs, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096)), 2 * d);
  {
    ProfScope prof_scope("k_hash_tables", s);
    k_hash_tables<<<grid, 256, 0, s>>>(co, d, static_cast<uint32_t>(n),
                                       static_cast<uint32_t>(b), hs);
  }
  return cudaGetLastError();
}

cudaError_t launch_bucket_sort(const uint32_t* hs, int d, int64_t n, int64_t C,
                               uint32_t* perm, uint32_t* off, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(C) * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope prof_scope("k_bucket_sort", s);
    k_bucket_sort<<<2 * d, kSortThreads, smem, s>>>(hs, static_cast<uint32_t>(n),
                                                    static_cast<uint32_t>(C), perm, off);
  }
  return cudaGetLastError();
}

}  // namespace cms
