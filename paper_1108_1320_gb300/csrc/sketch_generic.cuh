// sketch_generic.cuh - the generic fused task (any 5-smooth C, any storage
// type and alignment): staging in shared memory, gather front end over the
// bucket-class lists, shared-memory Stockham FFTs, Kahan accumulation.
// Shared by the single-instance kernel (k_sketch.cu) and the batched
// persistent kernel (k_sketch_fast.cu).
#pragma once

#include "cms_internal.h"

namespace cms {
namespace generic {

constexpr int kMaxG = 4;

struct SketchArgs {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  int n1, n2, n3, n;
  int64_t b;
  int R, C, nrows, d;
  int nradC;
  int radC[16];
  int G;
  int kchunk, nkc;
  const uint32_t* perm;
  const uint32_t* off;
  const float2* twfe;
  const float2* twC;
  float2* partial;
  int dt;            // storage type of A and B (batched launches)
};

// Staging type in shared memory: BF16 inputs stay BF16 (half the bytes, so
// larger hash domains fit), other inputs are staged as FP32.
template <typename T> struct Staged { using type = float; };
template <> struct Staged<__nv_bfloat16> { using type = __nv_bfloat16; };
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ float load_val(const T* p);
template <> __device__ __forceinline__ float load_val<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_val<double>(const double* p) {
  return static_cast<float>(__ldg(p));
}
template <> __device__ __forceinline__ float load_val<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// One task (t, f1, k-range) of the generic fused kernel; `smem4` is the
// block's dynamic shared memory (generic_smem_bytes).
template <typename T>
__device__ __forceinline__ void generic_task(const SketchArgs& p, int task, float4* smem4) {
  const int C = p.C, G = p.G, n = p.n;
  float2* twC = reinterpret_cast<float2*>(smem4);              // C
  float4* acc = smem4 + (C + 1) / 2;                            // C (sum re, im, comp re, im)
  float2* P = reinterpret_cast<float2*>(acc + C);               // 2 G C
  float2* Q = P + 2 * G * C;                                    // >= 2 G C, staging aliases it
  using S = typename Staged<T>::type;
  S* val = reinterpret_cast<S*>(Q);                             // [2][G][n]

  const int kc = task % p.nkc;
  const int row = (task / p.nkc) % p.nrows;
  const int t = task / (p.nkc * p.nrows);

  for (int i = threadIdx.x; i < C; i += blockDim.x) {
    twC[i] = p.twC[i];
    acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  const T* A = static_cast<const T*>(p.A);
  const T* B = static_cast<const T*>(p.B);
  const int k_begin = kc * p.kchunk;
  const int k_end = min(p.n2, k_begin + p.kchunk);
  const uint32_t* pmA = p.perm + static_cast<size_t>(t * 2 + 0) * n;
  const uint32_t* pmB = p.perm + static_cast<size_t>(t * 2 + 1) * n;
  const uint32_t* ofA = p.off + static_cast<size_t>(t * 2 + 0) * (C + 1);
  const uint32_t* ofB = p.off + static_cast<size_t>(t * 2 + 1) * (C + 1);
  const float2* twA = p.twfe + ((static_cast<size_t>(t) * p.nrows + row) * 2 + 0) * n;
  const float2* twB = twA + n;

  for (int k0 = k_begin; k0 < k_end; k0 += G) {
    const int gcnt = min(G, k_end - k0);
    __syncthreads();
    // stage a_k (column k of A) and b_k (row k of B), zero-filled to n
    for (int g = 0; g < G; ++g) {
      S* va = val + (0 * G + g) * n;
      S* vb = val + (1 * G + g) * n;
      const bool live = g < gcnt;
      const T* colA = A + static_cast<size_t>(k0 + g) * p.lda;
      const T* rowB = B + static_cast<size_t>(k0 + g) * p.ldb;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if constexpr (sizeof(S) == 2) {
          va[i] = (live && i < p.n1) ? colA[i] : __float2bfloat16(0.f);
          vb[i] = (live && i < p.n3) ? rowB[i] : __float2bfloat16(0.f);
        } else {
          va[i] = (live && i < p.n1) ? load_val<T>(colA + i) : 0.f;
          vb[i] = (live && i < p.n3) ? load_val<T>(rowB + i) : 0.f;
        }
      }
    }
    __syncthreads();
    // gather front end: Y[side][g][z2] = sum over the bucket class z2
    for (int task2 = threadIdx.x; task2 < 2 * C; task2 += blockDim.x) {
      const int side = task2 >= C;
      const int z2 = task2 - side * C;
      const uint32_t* pm = side ? pmB : pmA;
      const uint32_t* of = side ? ofB : ofA;
      const float2* tw = side ? twB : twA;
      const S* v = val + side * G * n;
      float2 s[kMaxG];
#pragma unroll
      for (int g = 0; g < kMaxG; ++g) s[g] = make_float2(0.f, 0.f);
      const uint32_t e1 = of[z2 + 1];
      for (uint32_t e = of[z2]; e < e1; ++e) {
        const uint32_t x = pm[e];
        const float2 w = tw[e];
#pragma unroll
        for (int g = 0; g < kMaxG; ++g) {
          if (g < G) {
            const float a = to_f32(v[g * n + x]);
            s[g].x = fmaf(a, w.x, s[g].x);
            s[g].y = fmaf(a, w.y, s[g].y);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < kMaxG; ++g)
        if (g < G) P[(side * G + g) * C + z2] = s[g];
    }
    __syncthreads();
    float2* X = fft_block<false>(P, Q, C, 2 * G, p.radC, p.nradC, twC);
    // spectral products, summed over the group, Kahan-accumulated over k
    for (int f2 = threadIdx.x; f2 < C; f2 += blockDim.x) {
      float2 prod = make_float2(0.f, 0.f);
      for (int g = 0; g < gcnt; ++g) {
        const float2 a = X[g * C + f2];
        const float2 bb = X[(G + g) * C + f2];
        prod.x = fmaf(a.x, bb.x, prod.x);
        prod.x = fmaf(-a.y, bb.y, prod.x);
        prod.y = fmaf(a.x, bb.y, prod.y);
        prod.y = fmaf(a.y, bb.x, prod.y);
      }
      float4 ac = acc[f2];
      kahan_add(ac.x, ac.z, prod.x);
      kahan_add(ac.y, ac.w, prod.y);
      acc[f2] = ac;
    }
  }
  __syncthreads();
  float2* out = p.partial + static_cast<size_t>(task) * C;
  for (int f2 = threadIdx.x; f2 < C; f2 += blockDim.x) {
    const float4 ac = acc[f2];
    out[f2] = make_float2(ac.x - ac.z, ac.y - ac.w);
  }
}


}  // namespace generic
}  // namespace cms
