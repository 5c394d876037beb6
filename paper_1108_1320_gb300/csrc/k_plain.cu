// k_plain.cu - the plain form of COMPRESSEDPRODUCT (Fig. 1) in FP64: one
// instance per call and one kernel per step, every intermediate in device
// memory.  Per repetition t and batch of inner indices k:
//   scatter  Z_k = pa_k + i pb_k (both count sketches packed in one complex
//            vector; FP64 atomics in global memory),
//   FFT      Z_k -> DFT_b(Z_k), one launch per mixed-radix Stockham pass,
//   product  S[f] += PA_k[f] PB_k[f] with PA = (Z[f] + conj Z[-f]) / 2,
//            PB = (Z[f] - conj Z[-f]) / (2i),
// then one inverse FFT of S and c_t = Re(.) / b.
#include <algorithm>

#include "cms_internal.h"

namespace cms {
namespace {

__global__ void k_plain_twiddles(double2* __restrict__ tw, int64_t b) {
  for (int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; m < b;
       m += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double s, c;
    sincospi(2.0 * static_cast<double>(m) / static_cast<double>(b), &s, &c);
    tw[m] = make_double2(c, -s);
  }
}

__global__ void k_plain_scatter(const double* __restrict__ A, int64_t lda,
                                const double* __restrict__ B, int64_t ldb, int64_t n1,
                                int64_t n3, int64_t k0, const uint32_t* __restrict__ hsA,
                                const uint32_t* __restrict__ hsB, int64_t b,
                                double2* __restrict__ Z) {
  const int64_t kk = blockIdx.y;
  const int64_t k = k0 + kk;
  double2* z = Z + kk * b;
  const int64_t nmax = n1 > n3 ? n1 : n3;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nmax;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (i < n1) {
      const uint32_t w = hsA[i];
      double v = A[i + k * lda];
      if (w >> 31) v = -v;
      atomicAdd(&z[w & kBucketMask].x, v);
    }
    if (i < n3) {
      const uint32_t w = hsB[i];
      double v = B[k * ldb + i];
      if (w >> 31) v = -v;
      atomicAdd(&z[w & kBucketMask].y, v);
    }
  }
}

template <int RAD, bool INV>
__global__ void k_plain_pass(const double2* __restrict__ src, double2* __restrict__ dst,
                             int64_t N, int64_t L, int64_t nvec, const double2* __restrict__ tw) {
  const int64_t Kp = N / (L * RAD);
  const int64_t nb = N / RAD;
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nvec * nb) return;
  const int64_t v = idx / nb;
  const int64_t beta = idx - v * nb;
  const int64_t fp = beta / Kp;
  const int64_t rho = beta - fp * Kp;
  const double2* s = src + v * N + rho + Kp * RAD * fp;
  double2 u[RAD];
#pragma unroll
  for (int q = 0; q < RAD; ++q) u[q] = s[Kp * q];
  if (L > 1) {
#pragma unroll
    for (int q = 1; q < RAD; ++q) {
      double2 w = tw[q * fp * Kp];
      if (INV) w.y = -w.y;
      u[q] = cmul(u[q], w);
    }
  }
  Dft<RAD, INV, double2>::run(u);
  double2* d = dst + v * N + beta;
#pragma unroll
  for (int s2 = 0; s2 < RAD; ++s2) d[nb * s2] = u[s2];
}

__global__ void k_plain_product(const double2* __restrict__ Zf, int64_t nk, int64_t b,
                                double2* __restrict__ S) {
  for (int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; f < b;
       f += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t fm = f == 0 ? 0 : b - f;
    double2 acc = S[f];
    for (int64_t kk = 0; kk < nk; ++kk) {
      const double2 z = Zf[kk * b + f];
      const double2 zc = cconj(Zf[kk * b + fm]);
      const double2 pa = cscale(cadd(z, zc), 0.5);
      const double2 dm = cscale(csub(z, zc), 0.5);
      const double2 pb = make_double2(dm.y, -dm.x);   // dm / i
      acc = cadd(acc, cmul(pa, pb));
    }
    S[f] = acc;
  }
}

__global__ void k_plain_finish(const double2* __restrict__ X, int64_t b, double* __restrict__ c) {
  for (int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; f < b;
       f += static_cast<int64_t>(gridDim.x) * blockDim.x)
    c[f] = X[f].x / static_cast<double>(b);
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

unsigned grid_for(int64_t work) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 1 << 20)));
}

template <bool INV>
cudaError_t run_fft(const PlainPlan& p, double2* a, double2* bbuf, int64_t nvec,
                    const double2* tw, double2** result, cudaStream_t s) {
  double2* src = a;
  double2* dst = bbuf;
  int64_t L = 1;
  const int64_t N = p.b;
  for (int q = 0; q < p.nrad; ++q) {
    const int r = p.rad[q];
    const int64_t work = nvec * (N / r);
    const unsigned g = static_cast<unsigned>((work + 255) / 256);
    ProfScope prof_scope("k_plain_pass", s);
    switch (r) {
      case 2: k_plain_pass<2, INV><<<g, 256, 0, s>>>(src, dst, N, L, nvec, tw); break;
      case 3: k_plain_pass<3, INV><<<g, 256, 0, s>>>(src, dst, N, L, nvec, tw); break;
      case 4: k_plain_pass<4, INV><<<g, 256, 0, s>>>(src, dst, N, L, nvec, tw); break;
      case 5: k_plain_pass<5, INV><<<g, 256, 0, s>>>(src, dst, N, L, nvec, tw); break;
      default: k_plain_pass<8, INV><<<g, 256, 0, s>>>(src, dst, N, L, nvec, tw); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    L *= r;
    std::swap(src, dst);
  }
  *result = src;
  return cudaSuccess;
}

}  // namespace

int make_plain_plan(const cms_hashes* h, int64_t n2, PlainPlan* plan, std::string* why) {
  PlainPlan p;
  p.b = h->b;
  p.nrad = factor_radices(h->b, p.rad, 24);
  if (p.nrad < 0) { *why = "b is not 5-smooth (2^x 3^y 5^z)"; return CMS_ERR_UNSUPPORTED; }
  // batch of inner indices: about 64 MiB per spectrum buffer
  const int64_t per_k = h->b * 16;
  p.kc = std::max<int64_t>(1, std::min<int64_t>({std::max<int64_t>(n2, 1), (64LL << 20) / per_k, 65535}));
  size_t off = 0;
  p.off_Z = off;  off = align256(off + static_cast<size_t>(p.kc) * per_k);
  p.off_Z2 = off; off = align256(off + static_cast<size_t>(p.kc) * per_k);
  p.off_S = off;  off = align256(off + static_cast<size_t>(per_k));
  p.off_tw = off; off = align256(off + static_cast<size_t>(per_k));
  p.ws_bytes = off;
  *plan = p;
  return CMS_OK;
}

cudaError_t launch_plain(const PlainPlan& p, const cms_hashes* h, const double* A, int64_t lda,
                         const double* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3,
                         double* c, char* ws, cudaStream_t s) {
  double2* Z = reinterpret_cast<double2*>(ws + p.off_Z);
  double2* Z2 = reinterpret_cast<double2*>(ws + p.off_Z2);
  double2* S = reinterpret_cast<double2*>(ws + p.off_S);
  double2* tw = reinterpret_cast<double2*>(ws + p.off_tw);
  const int64_t b = p.b;
  {
    ProfScope prof_scope("k_plain_twiddles", s);
    k_plain_twiddles<<<grid_for(b), 256, 0, s>>>(tw, b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nmax = std::max<int64_t>(std::max<int64_t>(n1, n3), 1);
  for (int t = 0; t < h->d; ++t) {
    const uint32_t* hsA = h->d_hs + static_cast<size_t>(2 * t) * h->n;
    const uint32_t* hsB = h->d_hs + static_cast<size_t>(2 * t + 1) * h->n;
    e = cudaMemsetAsync(S, 0, static_cast<size_t>(b) * 16, s);
    if (e != cudaSuccess) return e;
    for (int64_t k0 = 0; k0 < n2; k0 += p.kc) {
      const int64_t nk = std::min<int64_t>(p.kc, n2 - k0);
      e = cudaMemsetAsync(Z, 0, static_cast<size_t>(nk) * b * 16, s);
      if (e != cudaSuccess) return e;
      dim3 g(static_cast<unsigned>(std::min<int64_t>((nmax + 255) / 256, 1024)),
             static_cast<unsigned>(nk));
      {
        ProfScope prof_scope("k_plain_scatter", s);
        k_plain_scatter<<<g, 256, 0, s>>>(A, lda, B, ldb, n1, n3, k0, hsA, hsB, b, Z);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      double2* F = nullptr;
      e = run_fft<false>(p, Z, Z2, nk, tw, &F, s);
      if (e != cudaSuccess) return e;
      {
        ProfScope prof_scope("k_plain_product", s);
        k_plain_product<<<grid_for(b), 256, 0, s>>>(F, nk, b, S);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    double2* X = nullptr;
    e = run_fft<true>(p, S, Z, 1, tw, &X, s);
    if (e != cudaSuccess) return e;
    {
      ProfScope prof_scope("k_plain_finish", s);
      k_plain_finish<<<grid_for(b), 256, 0, s>>>(X, b, c + static_cast<size_t>(t) * b);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cms
