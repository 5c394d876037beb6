// cms_common.cuh - device helpers shared by the library's kernels:
// polynomial hash arithmetic, complex arithmetic, small DFT codelets and a
// block-cooperative mixed-radix Stockham FFT pass.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/cms.h"

namespace cms {

constexpr uint32_t kP31 = 0x7FFFFFFFu;   // p = 2^31 - 1 (Sec. 2.2 / ref. [13])
constexpr int kMaxD = 64;                // repetitions supported
constexpr uint32_t kBucketMask = 0x7FFFFFFFu;

// Packed hash-table entry: bits 0..30 bucket h(x) < b, bit 31 set when the
// sign s(x) is -1.  Tables are laid out [t][side][x], side 0 = (h1, s1) over
// rows of A, side 1 = (h2, s2) over columns of B.
struct Coeffs {
  uint32_t v[kMaxD][8];   // h1.a h1.c s1.a s1.c h2.a h2.c s2.a s2.c
};

// (y mod p) for y < 2^63 by folding the Mersenne modulus twice.
__host__ __device__ __forceinline__ uint32_t mod_p31(uint64_t y) {
  uint64_t v = (y & kP31) + (y >> 31);
  v = (v & kP31) + (v >> 31);
  if (v >= kP31) v -= kP31;
  return static_cast<uint32_t>(v);
}

// Degree-1 polynomial value (a x + c) mod p; a, c < p, x < 2^32.
__host__ __device__ __forceinline__ uint32_t poly_p31(uint32_t a, uint32_t c, uint32_t x) {
  return mod_p31(static_cast<uint64_t>(a) * x + c);
}

// ------------------------------------------------------------ complex ops --
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __host__ __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
template <bool INV> __host__ __device__ __forceinline__ double2 mul_mi(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

template <typename V> struct scalar_of;
template <> struct scalar_of<float2> { using type = float; };
template <> struct scalar_of<double2> { using type = double; };

template <typename V> __host__ __device__ __forceinline__ V cmake(double re, double im);
template <> __host__ __device__ __forceinline__ float2 cmake<float2>(double re, double im) {
  return make_float2(static_cast<float>(re), static_cast<float>(im));
}
template <> __host__ __device__ __forceinline__ double2 cmake<double2>(double re, double im) {
  return make_double2(re, im);
}

// ---------------------------------------------------------- DFT codelets --
// In-register DFT of length RAD: v_s = sum_q u_q w^{qs}, w = exp(-2 pi i/RAD)
// (forward) or exp(+2 pi i/RAD) (inverse, unscaled).
template <int RAD, bool INV, typename V> struct Dft;

template <bool INV, typename V> struct Dft<2, INV, V> {
  __device__ __forceinline__ static void run(V* u) {
    V a = u[0], b = u[1];
    u[0] = cadd(a, b);
    u[1] = csub(a, b);
  }
};

template <bool INV, typename V> struct Dft<4, INV, V> {
  __device__ __forceinline__ static void run(V* u) {
    V s02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
    V s13 = cadd(u[1], u[3]), d13 = mul_mi<INV>(csub(u[1], u[3]));
    u[0] = cadd(s02, s13);
    u[2] = csub(s02, s13);
    u[1] = cadd(d02, d13);
    u[3] = csub(d02, d13);
  }
};

template <bool INV, typename V> struct Dft<8, INV, V> {
  __device__ __forceinline__ static void run(V* u) {
    using S = typename scalar_of<V>::type;
    const S r = S(0.70710678118654752440);
    V e[4] = {u[0], u[2], u[4], u[6]};
    V o[4] = {u[1], u[3], u[5], u[7]};
    Dft<4, INV, V>::run(e);
    Dft<4, INV, V>::run(o);
    // w8^s for s = 1, 2, 3 (forward: (1-i)/sqrt2, -i, (-1-i)/sqrt2)
    V o1 = o[1], o3 = o[3];
    V t1;
    if (INV) {
      t1.x = (o1.x - o1.y) * r; t1.y = (o1.x + o1.y) * r;   // (1+i)/sqrt2
    } else {
      t1.x = (o1.x + o1.y) * r; t1.y = (o1.y - o1.x) * r;   // (1-i)/sqrt2
    }
    V t2 = mul_mi<INV>(o[2]);
    V t3;
    if (INV) {
      t3.x = -(o3.x + o3.y) * r; t3.y = (o3.x - o3.y) * r;  // (-1+i)/sqrt2
    } else {
      t3.x = (o3.y - o3.x) * r; t3.y = -(o3.x + o3.y) * r;  // (-1-i)/sqrt2
    }
    u[0] = cadd(e[0], o[0]); u[4] = csub(e[0], o[0]);
    u[1] = cadd(e[1], t1);   u[5] = csub(e[1], t1);
    u[2] = cadd(e[2], t2);   u[6] = csub(e[2], t2);
    u[3] = cadd(e[3], t3);   u[7] = csub(e[3], t3);
  }
};

template <bool INV, typename V> struct Dft<3, INV, V> {
  __device__ __forceinline__ static void run(V* u) {
    using S = typename scalar_of<V>::type;
    const S h = S(0.86602540378443864676);  // sqrt(3)/2
    V t1 = cadd(u[1], u[2]);
    V t2 = csub(u[1], u[2]);
    V m = make_sub_half(u[0], t1);
    // forward: v1 = m - i h t2, v2 = m + i h t2
    V it2;  // (-i) * h * t2 for forward
    it2.x = (INV ? -t2.y : t2.y) * h;
    it2.y = (INV ? t2.x : -t2.x) * h;
    u[0] = cadd(u[0], t1);
    u[1] = cadd(m, it2);
    u[2] = csub(m, it2);
  }
  __device__ __forceinline__ static V make_sub_half(V a, V t) {
    using S = typename scalar_of<V>::type;
    V r; r.x = a.x - S(0.5) * t.x; r.y = a.y - S(0.5) * t.y; return r;
  }
};

template <bool INV, typename V> struct Dft<5, INV, V> {
  __device__ __forceinline__ static void run(V* u) {
    using S = typename scalar_of<V>::type;
    const S c1 = S(0.30901699437494742410);   // cos(2 pi/5)
    const S c2 = S(-0.80901699437494742410);  // cos(4 pi/5)
    const S s1 = S(0.95105651629515357212);   // sin(2 pi/5)
    const S s2 = S(0.58778525229247312917);   // sin(4 pi/5)
    V a1 = cadd(u[1], u[4]), b1 = csub(u[1], u[4]);
    V a2 = cadd(u[2], u[3]), b2 = csub(u[2], u[3]);
    V r1, r2, q1, q2;
    r1.x = u[0].x + c1 * a1.x + c2 * a2.x; r1.y = u[0].y + c1 * a1.y + c2 * a2.y;
    r2.x = u[0].x + c2 * a1.x + c1 * a2.x; r2.y = u[0].y + c2 * a1.y + c1 * a2.y;
    // q1 = s1 b1 + s2 b2 ; q2 = s2 b1 - s1 b2
    q1.x = s1 * b1.x + s2 * b2.x; q1.y = s1 * b1.y + s2 * b2.y;
    q2.x = s2 * b1.x - s1 * b2.x; q2.y = s2 * b1.y - s1 * b2.y;
    // forward: v1 = r1 - i q1, v4 = r1 + i q1, v2 = r2 - i q2, v3 = r2 + i q2
    V iq1 = mul_mi<INV>(q1), iq2 = mul_mi<INV>(q2);
    u[0] = cadd(u[0], cadd(a1, a2));
    u[1] = cadd(r1, iq1);
    u[4] = csub(r1, iq1);
    u[2] = cadd(r2, iq2);
    u[3] = csub(r2, iq2);
  }
};

// ------------------------------------------------- Stockham radix pass ----
// One pass of a mixed-radix Stockham autosort FFT of length N on `nvec`
// vectors stored back to back (vector v at src + v*N).  Sub-transforms of
// length L are combined RAD at a time into length L*RAD; with K' = N/(L RAD),
// butterfly beta = rho' + K' f' reads src[rho' + K'(q + RAD f')], twiddles
// input q by w_N^{q f' K'}, and writes dst[beta + (N/RAD) s].  `tw` holds
// w_N^m = exp(-2 pi i m / N), m < N.  Input natural order, output natural
// order after the last pass.
template <int RAD, bool INV, typename V>
__device__ __forceinline__ void stockham_pass_block(const V* __restrict__ src, V* __restrict__ dst,
                                                    int N, int L, int nvec, const V* __restrict__ tw) {
  const int Kp = N / (L * RAD);
  const int nb = N / RAD;
  const int total = nvec * nb;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int v = idx / nb;
    const int beta = idx - v * nb;
    const int fp = beta / Kp;
    const int rho = beta - fp * Kp;
    const V* s = src + static_cast<size_t>(v) * N + rho + Kp * RAD * fp;
    V u[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) u[q] = s[Kp * q];
    if (L > 1) {
#pragma unroll
      for (int q = 1; q < RAD; ++q) {
        V w = tw[q * fp * Kp];
        if (INV) w.y = -w.y;
        u[q] = cmul(u[q], w);
      }
    }
    Dft<RAD, INV, V>::run(u);
    V* d = dst + static_cast<size_t>(v) * N + beta;
#pragma unroll
    for (int s2 = 0; s2 < RAD; ++s2) d[nb * s2] = u[s2];
  }
}

// Run the passes listed in rad[0..nrad) over `nvec` vectors of length N held
// in buffer a; b is the ping-pong buffer.  Returns the buffer holding the
// result.  Includes the block barriers between passes.
template <bool INV, typename V>
__device__ V* fft_block(V* a, V* b, int N, int nvec, const int* rad, int nrad, const V* tw) {
  int L = 1;
  V* src = a;
  V* dst = b;
  for (int p = 0; p < nrad; ++p) {
    const int r = rad[p];
    switch (r) {
      case 2: stockham_pass_block<2, INV>(src, dst, N, L, nvec, tw); break;
      case 3: stockham_pass_block<3, INV>(src, dst, N, L, nvec, tw); break;
      case 4: stockham_pass_block<4, INV>(src, dst, N, L, nvec, tw); break;
      case 5: stockham_pass_block<5, INV>(src, dst, N, L, nvec, tw); break;
      default: stockham_pass_block<8, INV>(src, dst, N, L, nvec, tw); break;
    }
    __syncthreads();
    L *= r;
    V* tmp = src; src = dst; dst = tmp;
  }
  return src;
}

// Radix list for a 5-smooth length N: 8s first, then 4, 2, 5, 3.  Returns the
// count, or -1 when N has another prime factor or needs more than maxr passes.
__host__ __device__ inline int factor_radices(int64_t N, int* rad, int maxr) {
  int n = 0;
  while (N % 8 == 0 && N > 1) { if (n >= maxr) return -1; rad[n++] = 8; N /= 8; }
  while (N % 4 == 0 && N > 1) { if (n >= maxr) return -1; rad[n++] = 4; N /= 4; }
  while (N % 2 == 0 && N > 1) { if (n >= maxr) return -1; rad[n++] = 2; N /= 2; }
  while (N % 5 == 0 && N > 1) { if (n >= maxr) return -1; rad[n++] = 5; N /= 5; }
  while (N % 3 == 0 && N > 1) { if (n >= maxr) return -1; rad[n++] = 3; N /= 3; }
  return N == 1 ? n : -1;
}

}  // namespace cms
