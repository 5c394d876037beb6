// k_sketch.cu - the fused FP32 path of COMPRESSEDPRODUCT (Fig. 1, Sec. 2.2).
//
// For one repetition t the sketch spectrum is
//   S_t[f] = sum_k PA_k[f] PB_k[f],  PA_k = DFT_b(pa_k), PB_k = DFT_b(pb_k),
// with pa_k[z] = sum_{h1(i)=z} s1(i) A_ik and pb_k likewise from row k of B
// (Fig. 1; Sec. 2.2 "p*_t = p_u(w^t) p_v(w^t)").  The length-b DFT is split
// as b = R * C (Cooley-Tukey four-step, input index z = C z1 + z2, output
// f = f1 + R f2):
//   PA_k[f1 + R f2] = sum_{z2} w_C^{f2 z2} Y_k[f1][z2],
//   Y_k[f1][z2]     = sum_{i : h1(i) mod C = z2} s1(i) A_ik w_b^{f1 h1(i)}.
// The first step is evaluated directly from the <= n nonzeros of the sketch
// (a pruned first stage), so a thread block owning row f1 needs nothing but
// column k of A and row k of B: no length-b vector is ever formed, and rows
// are independent.  Because pa, pb are real, row R - f1 is the conjugate
// mirror of row f1 and only rows f1 = 0..floor(R/2) are computed.
//
// K0  twiddle tables (front-end twiddles per (t, f1, side, entry); w_C; w_R)
// K1  per task (t, f1, k-range): gather front end -> 2G length-C FFTs in
//     shared memory -> spectral products summed over the group -> Kahan
//     compensated accumulation over k -> one partial row written out
// K2a per (t, f1): fixed-order sum of the k-range partials, inverse
//     length-C FFT, twiddle w_b^{-f1 z2}
// K2b per output z = C z1 + z2: real inverse length-R DFT over f1 using the
//     conjugate symmetry, scaled by 1/b (Fig. 1, p[t] := FFT^{-1}(p[t])).
#include <algorithm>
#include <vector>

#include "cms_internal.h"
#include "sketch_generic.cuh"

namespace cms {
namespace {

using namespace generic;



// w_M^m = exp(-2 pi i m / M) in FP32 for 0 <= m < M: the angle is reduced to
// (-pi, pi] with integers first, so 2m/M has at most one rounding (none for
// power-of-two M) before sincospif.
__device__ __forceinline__ float2 w_pow(uint64_t m, int64_t M) {
  const int64_t mm = 2 * static_cast<int64_t>(m) > M ? static_cast<int64_t>(m) - M : static_cast<int64_t>(m);
  float s, c;
  sincospif(2.0f * static_cast<float>(mm) / static_cast<float>(M), &s, &c);
  return make_float2(c, -s);
}

// w_M^m = exp(-2 pi i m / M) for m < M, rounded from double, by the first
// ceil(M / 256) blocks; with hi != nullptr the blocks after them write
// hi[i] = w_b^{i S} for i < nhi (the high half of the warp-specialised
// kernel's split twiddle w_b^m = w_b^{m mod S} w_b^{(m div S) S}).
__global__ void k_twiddle_table(float2* __restrict__ tw, int M, float2* __restrict__ hi, int S, int nhi,
                                int64_t b, float2* __restrict__ tw2, int M2) {
  // blocks [0, nbt): w_M^m; then, when hi is given, nbh blocks of w_b^{i S};
  // then, when tw2 is given, the blocks of w_M2^m (one launch for all three)
  const int nbt = (M + 255) / 256;
  const int nbh = hi != nullptr ? (nhi + 255) / 256 : 0;
  const int blk = static_cast<int>(blockIdx.x);
  if (blk < nbt) {
    const int m = blk * blockDim.x + threadIdx.x;
    if (m < M) {
      double s, c;
      sincospi(2.0 * static_cast<double>(m) / static_cast<double>(M), &s, &c);
      tw[m] = make_float2(static_cast<float>(c), static_cast<float>(-s));
    }
  } else if (blk < nbt + nbh) {
    const int i = (blk - nbt) * blockDim.x + threadIdx.x;
    if (i < nhi) {
      const double a = 2.0 * static_cast<double>(static_cast<int64_t>(i) * S) / static_cast<double>(b);
      double s, c;
      sincospi(a, &s, &c);
      hi[i] = make_float2(static_cast<float>(c), static_cast<float>(-s));
    }
  } else if (tw2 != nullptr) {
    const int m = (blk - nbt - nbh) * blockDim.x + threadIdx.x;
    if (m < M2) {
      double s, c;
      sincospi(2.0 * static_cast<double>(m) / static_cast<double>(M2), &s, &c);
      tw2[m] = make_float2(static_cast<float>(c), static_cast<float>(-s));
    }
  }
}

// Grid of k_twiddle_table for the three tables.
unsigned twiddle_blocks(int M, const float2* hi, int nhi, const float2* tw2, int M2) {
  return static_cast<unsigned>((M + 255) / 256 + (hi != nullptr ? (nhi + 255) / 256 : 0) +
                               (tw2 != nullptr ? (M2 + 255) / 256 : 0));
}

// Front-end twiddle of sorted entry e of table (t, side) for row f1:
// s(x) w_b^{(h(x) f1) mod b}, x = perm[e].
__global__ void k_frontend_twiddles(const uint32_t* __restrict__ hs,
                                    const uint32_t* __restrict__ perm, int n, int64_t b,
                                    int nrows, float2* __restrict__ twfe) {
  const int f1 = blockIdx.y;
  const int ts = blockIdx.z;  // t * 2 + side
  const int t = ts >> 1, side = ts & 1;
  const uint32_t* pm = perm + static_cast<size_t>(ts) * n;
  const uint32_t* tab = hs + static_cast<size_t>(ts) * n;
  float2* out = twfe + ((static_cast<size_t>(t) * nrows + f1) * 2 + side) * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const uint32_t w = tab[pm[e]];
    const uint64_t m = (static_cast<uint64_t>(w & kBucketMask) * static_cast<uint64_t>(f1)) %
                       static_cast<uint64_t>(b);
    float2 v = w_pow(m, b);
    if (w >> 31) { v.x = -v.x; v.y = -v.y; }
    out[e] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sketch_fused(SketchArgs p) {
  extern __shared__ float4 smem4[];
  generic_task<T>(p, blockIdx.x, smem4);
}

struct InvArgs {
  int64_t b;
  int R, C, nrows, d, nkc;
  int nradC;
  int radC[16];
  const float2* partial;
  const float2* twC;
  float2* V;
  const int32_t* skip_if_zero;   // optional: return at once when it holds 0
};

// s + e += x with the rounding error of each add carried in e (Neumaier's
// variant of Kahan summation: the larger magnitude decides which error term
// is exact).
__device__ __forceinline__ void neumaier_add(float& s, float& e, float x) {
  const float t = s + x;
  e += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

// K2a body: block tr = t * nrows + f1 of one product.
__device__ __forceinline__ void rows_inverse_block(const InvArgs& p, int tr, float2* sm2) {
  const int C = p.C;
  float2* twC = sm2;
  float2* P = twC + C;
  float2* Q = P + C;
  const int f1 = tr % p.nrows;
  for (int i = threadIdx.x; i < C; i += blockDim.x) twC[i] = p.twC[i];
  const float2* part = p.partial + static_cast<size_t>(tr) * p.nkc * C;
  for (int f2 = threadIdx.x; f2 < C; f2 += blockDim.x) {
    // the k-chunk partials in chunk order, compensated (Neumaier) in FP32:
    // the error of the plain FP64 sum without its FP64 adds
    float sx = 0.f, ex = 0.f, sy = 0.f, ey = 0.f;
#pragma unroll 4
    for (int kc = 0; kc < p.nkc; ++kc) {
      const float2 v = __ldg(part + static_cast<size_t>(kc) * C + f2);
      neumaier_add(sx, ex, v.x);
      neumaier_add(sy, ey, v.y);
    }
    P[f2] = make_float2(sx + ex, sy + ey);
  }
  __syncthreads();
  float2* X = fft_block<true>(P, Q, C, 1, p.radC, p.nradC, twC);
  float2* out = p.V + static_cast<size_t>(tr) * C;
  for (int z2 = threadIdx.x; z2 < C; z2 += blockDim.x) {
    // f1 <= R / 2 and z2 < C, so f1 z2 < b / 2 needs no reduction mod b
    const uint64_t m = static_cast<uint64_t>(f1) * static_cast<uint64_t>(z2);
    const float2 w = cconj(w_pow(m, p.b));   // w_b^{-m}
    out[z2] = cmul(X[z2], w);
  }
}

// K2a: one block per (t, f1).
__global__ void __launch_bounds__(256) k_rows_inverse(InvArgs p) {
  extern __shared__ float2 sm2[];
  if (p.skip_if_zero && *p.skip_if_zero == 0) return;
  rows_inverse_block(p, blockIdx.x, sm2);
}

// The instance of a batched launch that owns block `blk`: the last i with
// start[i] <= blk (start ascending, start[0] = 0).
__device__ __forceinline__ int batch_instance(const int* __restrict__ start, int count, int blk) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// K2a for a batch: every instance's (t, f1) blocks in one launch.
__global__ void __launch_bounds__(256)
k_rows_inverse_batched(const InvArgs* __restrict__ args, const int* __restrict__ start, int count) {
  extern __shared__ float2 sm2[];
  const int i = batch_instance(start, count, static_cast<int>(blockIdx.x));
  const InvArgs p = args[i];
  rows_inverse_block(p, static_cast<int>(blockIdx.x) - __ldg(start + i), sm2);
}

// K2b: c[t][C z1 + z2] = (1/b) Re sum_{f1=0}^{R-1} V[f1][z2] w_R^{-f1 z1}, rows
// above R/2 taken as conjugates of rows below it.
__device__ __forceinline__ void cols_inverse_point(const float2* __restrict__ V, const float2* __restrict__ twR,
                                                   int64_t b, int R, int C, int nrows, float* __restrict__ c,
                                                   int t, int64_t z) {
  const int z1 = static_cast<int>(z / C);
  const int z2 = static_cast<int>(z - static_cast<int64_t>(z1) * C);
  const float2* Vt = V + static_cast<size_t>(t) * nrows * C + z2;
  float sum = Vt[0].x;
  const bool even = (R % 2) == 0;
  int e = 0;   // f1 z1 mod R, stepped (z1 < R)
  for (int f1 = 1; f1 < nrows; ++f1) {
    e += z1;
    if (e >= R) e -= R;
    const float2 v = Vt[static_cast<size_t>(f1) * C];
    const float2 w = __ldg(twR + e);                             // w_R^{f1 z1}
    const float term = v.x * w.x + v.y * w.y;                    // Re(v conj(w))
    sum += (even && 2 * f1 == R) ? term : 2.f * term;
  }
  c[static_cast<size_t>(t) * b + z] = sum / static_cast<float>(b);
}

__global__ void __launch_bounds__(256)
k_cols_inverse(const float2* __restrict__ V, const float2* __restrict__ twR, int64_t b,
               int R, int C, int nrows, float* __restrict__ c, const int32_t* __restrict__ skip_if_zero) {
  if (skip_if_zero && *skip_if_zero == 0) return;
  const int64_t z = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= b) return;
  cols_inverse_point(V, twR, b, R, C, nrows, c, static_cast<int>(blockIdx.y), z);
}

// K2b for long columns (large R): nv adjacent columns z2 of one repetition
// per block; the full length-R spectrum of each is rebuilt from rows
// 0..R/2 (row R - f1 is the conjugate of row f1) and inverted by the
// shared-memory mixed-radix FFT (O(R log R) per column instead of the
// direct sum's O(R^2)); c[z1 C + z2] = Re(x[z1]) / b.
__global__ void __launch_bounds__(256)
k_cols_inverse_fft(const float2* __restrict__ V, const float2* __restrict__ twR, int64_t b, int R, int C,
                   int nrows, int nv, float* __restrict__ c, const int32_t* __restrict__ skip_if_zero) {
  extern __shared__ __align__(16) float2 csm[];
  if (skip_if_zero && *skip_if_zero == 0) return;
  const int t = static_cast<int>(blockIdx.y);
  const int z0 = static_cast<int>(blockIdx.x) * nv;
  const int nvb = min(nv, C - z0);
  const float2* Vt = V + static_cast<size_t>(t) * nrows * C;
  float2* a = csm;
  float2* bb = csm + static_cast<size_t>(nv) * R;
  for (int i = threadIdx.x; i < R * nv; i += blockDim.x) {
    const int f = i / nv, v = i - (i / nv) * nv;
    float2 x = make_float2(0.f, 0.f);
    if (v < nvb) {
      if (f < nrows) {
        x = Vt[static_cast<size_t>(f) * C + z0 + v];
      } else {
        const float2 y = Vt[static_cast<size_t>(R - f) * C + z0 + v];
        x = make_float2(y.x, -y.y);
      }
    }
    a[static_cast<size_t>(v) * R + f] = x;
  }
  __syncthreads();
  int rad[16];
  const int nrad = factor_radices(R, rad, 16);
  const float2* out = fft_block<true>(a, bb, R, nv, rad, nrad, twR);
  const float inv_b = 1.f / static_cast<float>(b);
  float* ct = c + static_cast<size_t>(t) * b;
  for (int i = threadIdx.x; i < R * nv; i += blockDim.x) {
    const int z1 = i / nv, v = i - (i / nv) * nv;
    if (v < nvb) ct[static_cast<size_t>(z1) * C + z0 + v] = out[static_cast<size_t>(v) * R + z1].x * inv_b;
  }
}

struct ColsArgs {
  const float2* V;
  const float2* twR;
  float* c;
  int64_t b;
  int R, C, nrows;
  int nbx;   // blocks of 256 points per repetition
};

// K2b for a batch: every instance's (repetition, point block) in one launch.
__global__ void __launch_bounds__(256)
k_cols_inverse_batched(const ColsArgs* __restrict__ args, const int* __restrict__ start, int count) {
  const int i = batch_instance(start, count, static_cast<int>(blockIdx.x));
  const ColsArgs a = args[i];
  const int local = static_cast<int>(blockIdx.x) - __ldg(start + i);
  const int t = local / a.nbx;
  const int64_t z = static_cast<int64_t>(local % a.nbx) * blockDim.x + threadIdx.x;
  if (z < a.b) cols_inverse_point(a.V, a.twR, a.b, a.R, a.C, a.nrows, a.c, t, z);
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

size_t fused_smem_bytes(int C, int G, int n, int dt) {
  const size_t tw = static_cast<size_t>((C + 1) / 2) * 16;
  const size_t acc = static_cast<size_t>(C) * 16;
  const size_t Pb = static_cast<size_t>(2 * G) * C * 8;
  const size_t elem = dt == CMS_BF16 ? 2 : 4;    // staging element (BF16 stays BF16)
  const size_t Qb = std::max(static_cast<size_t>(2 * G) * C * 8, static_cast<size_t>(2 * G) * n * elem);
  return tw + acc + Pb + Qb;
}

}  // namespace

// b = R x C.  C = P Q for the register-FFT kernels (P, Q codelet lengths)
// when such a factor divides b (the largest one), else the largest divisor
// of b up to 1024 (the shared-memory kernel takes any 5-smooth C).
bool choose_factorisation(int64_t b, int64_t* R, int64_t* C) {
  int rad[64];
  if (b < 1 || factor_radices(b, rad, 64) < 0) { *R = 0; *C = 0; return false; }
  int64_t best = 1, best_pq = 0;
  for (int64_t c = 1; c <= std::min<int64_t>(b, 1024); ++c) {
    if (b % c != 0) continue;
    best = c;
    if (fe_pq(c, nullptr, nullptr)) best_pq = c;
  }
  if (best_pq > 0) best = best_pq;
  *C = best;
  *R = b / best;
  return true;
}

namespace {

// Inner-index chunks per (t, f1) unit so that the task count fills whole
// waves of `slots` concurrent blocks as evenly as possible.
int64_t choose_chunks(int64_t units, int64_t n2, int G, int64_t slots, int64_t lo, int64_t hi) {
  const int64_t max_chunks = std::max<int64_t>(1, (n2 + G - 1) / G);
  hi = std::min(hi, max_chunks);
  lo = std::min(lo, hi);
  int64_t best = lo;
  double best_eff = -1.0;
  for (int64_t c = lo; c <= hi; ++c) {
    const int64_t tasks = units * c;
    const int64_t waves = (tasks + slots - 1) / slots;
    const double eff = static_cast<double>(tasks) / static_cast<double>(waves * slots);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = c; }
  }
  return best;
}

}  // namespace

int make_sketch_plan(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3, int dt,
                     int num_sms, size_t smem_optin, SketchPlan* plan, std::string* why,
                     const void* A, int64_t lda, const void* B, int64_t ldb, bool allow_fast,
                     int nkc_override, int G_override, bool allow_ws, bool allow_wide) {
  SketchPlan p;
  const bool bf16 = dt == CMS_BF16;
  (void)bf16;
  p.b = h->b;
  p.d = h->d;
  if (h->C <= 0) { *why = "b is not 5-smooth (2^x 3^y 5^z): the fused FFT path needs it"; return CMS_ERR_UNSUPPORTED; }
  p.R = h->R;
  p.C = h->C;
  p.nrows = static_cast<int>(p.R / 2 + 1);
  p.nradC = factor_radices(p.C, p.radC, 16);
  if (p.nradC < 0) { *why = "internal: C not factorable"; return CMS_ERR_UNSUPPORTED; }
  if (p.R > 65536) { *why = "R = b / C too large"; return CMS_ERR_UNSUPPORTED; }
  const int n = static_cast<int>(h->n);
  const int64_t units = static_cast<int64_t>(p.d) * p.nrows;

  // the C = P Q register-FFT kernels: FP32 or BF16 rows that TMA can copy
  // (16-byte aligned rows, or aligned supersets of unaligned ones)
  p.dt = dt;
  const int per16 = dt == CMS_BF16 ? 8 : 4;   // elements per 16 bytes
  // rows not in whole 16-byte units are copied as their aligned supersets
  // (the lock-step kernel only): staged rows then start up to per16 - 1
  // elements in, and padding reads a zero slot past every copy
  const bool aligned = (A == nullptr || reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                       (B == nullptr || reinterpret_cast<uintptr_t>(B) % 16 == 0) &&
                       lda % per16 == 0 && ldb % per16 == 0 && n1 % per16 == 0 && n3 % per16 == 0;
  const size_t esz = dt == CMS_BF16 ? 2 : 4;
  const bool elem_aligned = (A == nullptr || reinterpret_cast<uintptr_t>(A) % esz == 0) &&
                            (B == nullptr || reinterpret_cast<uintptr_t>(B) % esz == 0);
  if (allow_fast && (dt == CMS_F32 || dt == CMS_BF16) && fe_pq(p.C, nullptr, nullptr) &&
      h->fe_ecap > 0 && elem_aligned) {
    p.alias = A != nullptr && A == B && lda == ldb && n1 == n3;
    p.unal = !aligned;
    p.npad = p.unal ? static_cast<int>((h->n + 3 * per16 + per16 - 1) / per16 * per16)
                    : static_cast<int>(((h->n + 1) + per16 - 1) / per16 * per16);
    p.zpos = p.unal ? static_cast<int>(h->n + 2 * per16) : 0;
    int sh = 0;
    while ((static_cast<int64_t>(1) << (2 * sh)) < p.b) ++sh;
    p.tw_shift = sh;
    p.nhi = static_cast<int>((p.b + (static_cast<int64_t>(1) << sh) - 1) >> sh);
    const size_t sm = fast_smem_bytes(p.npad, h->fe_ecap, p.alias ? 1 : 0, p.tw_shift, p.nhi, dt == CMS_BF16 ? 2 : 4, 0);
    // large hash domains: the records of two rows (16 bytes per entry) may
    // not fit beside the staging rows; the lock-step kernel then keeps them
    // in tensor memory (and asks for a whole SM)
    const size_t sm_tm = std::max(kSmemOneBlockPerSm,
                                  fast_smem_bytes(p.npad, h->fe_ecap, p.alias ? 1 : 0, p.tw_shift, p.nhi,
                                                  dt == CMS_BF16 ? 2 : 4, 1));
    // the warp-specialised kernel caches up to 1024 overflow twiddles in the
    // shared memory left over (at least 64 entries, or it is not used)
    const size_t ws_base = ws_smem_bytes(p.npad, h->fe_ecap, p.alias ? 1 : 0, p.tw_shift, p.nhi, 0);
    // (1 KB is left for the kernel's static shared variables)
    const int ovcap = ws_base + 64 * 18 + 1024 <= smem_optin
                          ? static_cast<int>(std::min<size_t>(1024, (smem_optin - ws_base - 1024) / 18))
                          : 0;
    const size_t sm_ws = ws_smem_bytes(p.npad, h->fe_ecap, p.alias ? 1 : 0, p.tw_shift, p.nhi, ovcap);
    const bool ws_ok = allow_ws && dt == CMS_F32 && !p.unal && p.C == kFeC && ovcap >= 64 &&
                       sm_ws <= smem_optin && ws_kernel_usable();
    // the front-end records hold staging indices (< 3 npad) in 16 bits
    if ((sm <= smem_optin || ws_ok || sm_tm <= smem_optin) && 3 * static_cast<int64_t>(p.npad) <= 65535) {
      p.fast = true;
      p.ws = ws_ok;
      p.tmem_rec = !ws_ok && sm > smem_optin;
      p.ovcap = ws_ok ? ovcap : 0;
      p.G = 2;
      p.threads = ws_ok ? 512 : 256;
      p.smem = ws_ok ? sm_ws : (p.tmem_rec ? sm_tm : sm);
    }
  }
  // long sketches (b a multiple of 2^16): the cluster kernel, one row of
  // C = 2^16 bins per 8-CTA cluster, when a_k (and b_k) fit its 64 KB
  // staging buffer as whole 16-byte units; preferred over the register-FFT
  // kernels from R = b / 2^16 >= 4 on (few rows, each entry visited by few)
  if (allow_wide && (dt == CMS_F32 || dt == CMS_BF16) && p.b % kWideC == 0 && aligned) {
    const bool al = A != nullptr && A == B && lda == ldb && n1 == n3;
    const int64_t n1s = al ? 0 : (n1 + per16 - 1) / per16 * per16;
    const int64_t stage = al ? n1 * static_cast<int64_t>(esz) : (n1s + n3) * static_cast<int64_t>(esz);
    const int64_t Rw = p.b / kWideC;
    if (stage <= 65536 && h->n <= 65535 && (!p.fast || Rw >= 4) && wide_max_clusters(dt) > 0 &&
        wide_smem_bytes() <= smem_optin) {
      p.wide = true;
      p.fast = false;
      p.ws = false;
      p.alias = al;
      p.unal = false;
      p.C = kWideC;
      p.R = Rw;
      p.nrows = static_cast<int>(Rw / 2 + 1);
      p.nradC = 0;
      p.G = 1;
      p.threads = 256;
      p.smem = wide_smem_bytes();
    }
  }
  if (p.wide) {
    const int64_t wunits = static_cast<int64_t>(p.d) * p.nrows;
    const int64_t slots = std::max(1, wide_max_clusters(dt));
    const int64_t lo = std::max<int64_t>(1, (slots + wunits - 1) / wunits);
    int64_t nkc = choose_chunks(wunits, n2, 1, slots, lo, std::max<int64_t>(lo, 4 * lo));
    if (nkc_override > 0) nkc = std::min<int64_t>(nkc_override, std::max<int64_t>(1, n2));
    int64_t kchunk = n2 > 0 ? (n2 + nkc - 1) / nkc : 1;
    nkc = n2 > 0 ? (n2 + kchunk - 1) / kchunk : 1;
    p.kchunk = kchunk;
    p.nkc = static_cast<int>(nkc);
    size_t off = 0;
    p.off_partial = off; off = align256(off + static_cast<size_t>(wunits) * p.nkc * kWideC * 8);
    p.off_V = off;       off = align256(off + static_cast<size_t>(wunits) * kWideC * 8);
    p.off_T = off;       off = align256(off + static_cast<size_t>(wunits) * kWideC * 8);
    p.off_twfe = off;
    p.off_twC = off;     off = align256(off + 256 * 8);
    p.off_twR = off;     off = align256(off + static_cast<size_t>(p.R) * 8);
    p.off_wtab = off;    off = wide_tables_layout(p.d, h->n, off).end;
    p.ws_bytes = off;
    *plan = p;
    return CMS_OK;
  }
  if (!p.fast) {
    int G = 0;
    for (int g = kMaxG; g >= 1; --g) {
      if (fused_smem_bytes(static_cast<int>(p.C), g, n, dt) <= 112 * 1024) { G = g; break; }
    }
    if (G == 0) {
      for (int g = kMaxG; g >= 1; --g)
        if (fused_smem_bytes(static_cast<int>(p.C), g, n, dt) <= smem_optin) { G = g; break; }
    }
    if (G == 0) {
      *why = "hash domain n too large for the shared-memory staging of the fused kernel";
      return CMS_ERR_UNSUPPORTED;
    }
    if (G_override > 0 && G_override <= kMaxG &&
        fused_smem_bytes(static_cast<int>(p.C), G_override, n, dt) <= smem_optin)
      G = G_override;
    p.G = G;
    p.smem = fused_smem_bytes(static_cast<int>(p.C), G, n, dt);
  }
  const int G = p.G;
  const int per_sm = p.fast ? 1 : std::max<int>(1, static_cast<int>(std::min<size_t>(4, (228 * 1024) / (p.smem + 1024))));
  const int64_t slots = static_cast<int64_t>(num_sms) * per_sm;
  // the fast kernel's blocks own two rows each
  const int64_t blocks_per_chunk = p.fast ? static_cast<int64_t>(p.d) * ((p.nrows + 1) / 2) : units;
  const int64_t lo = std::max<int64_t>(1, (2 * slots + blocks_per_chunk - 1) / blocks_per_chunk);
  int64_t nkc = choose_chunks(blocks_per_chunk, n2, G, slots, lo, std::max<int64_t>(lo, 4 * lo));
  if (nkc_override > 0) nkc = std::min<int64_t>(nkc_override, std::max<int64_t>(1, (n2 + G - 1) / G));
  int64_t kchunk = n2 > 0 ? (n2 + nkc - 1) / nkc : G;
  kchunk = ((kchunk + G - 1) / G) * G;
  nkc = n2 > 0 ? (n2 + kchunk - 1) / kchunk : 1;
  p.kchunk = kchunk;
  p.nkc = static_cast<int>(nkc);
  size_t off = 0;
  p.off_partial = off; off = align256(off + static_cast<size_t>(units) * p.nkc * p.C * 8);
  p.off_V = off;       off = align256(off + static_cast<size_t>(units) * p.C * 8);
  p.off_twfe = off;    off = align256(off + static_cast<size_t>(units) * 2 * h->n * 8);  // both kernels: same size
  p.off_twC = off;     off = align256(off + static_cast<size_t>(p.C) * 8);
  p.off_twR = off;     off = align256(off + static_cast<size_t>(p.R) * 8);
  p.off_thi = off;     off = align256(off + (p.ws ? static_cast<size_t>(p.nhi) * 8 : 0));
  p.ws_bytes = off;
  *plan = p;
  return CMS_OK;
}

cudaError_t launch_sketch(const SketchPlan& plan, const cms_hashes* h, const void* A,
                          int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                          int64_t n3, int dt, float* c, char* ws, cudaStream_t s) {
  float2* partial = reinterpret_cast<float2*>(ws + plan.off_partial);
  float2* V = reinterpret_cast<float2*>(ws + plan.off_V);
  float2* twfe = reinterpret_cast<float2*>(ws + plan.off_twfe);
  float2* twC = reinterpret_cast<float2*>(ws + plan.off_twC);
  float2* twR = reinterpret_cast<float2*>(ws + plan.off_twR);
  const int n = static_cast<int>(h->n);

  if (plan.wide) {
    cudaError_t e = launch_twiddle_tables(twC, 256, twR, static_cast<int>(plan.R), s);
    if (e == cudaSuccess) e = launch_sketch_wide(plan, h, A, lda, B, ldb, n1, n2, n3, ws, partial, s);
    if (e != cudaSuccess) return e;
    return launch_inverse_wide(plan, partial, V, reinterpret_cast<float2*>(ws + plan.off_T), twC, twR, c, s);
  }
  {
    ProfScope prof_scope("k_twiddle_table", s);
    // with the warp-specialised kernel's high twiddles and the length-R
    // table in extra blocks
    float2* hi = plan.ws ? reinterpret_cast<float2*>(ws + plan.off_thi) : nullptr;
    const int R = static_cast<int>(plan.R);
    k_twiddle_table<<<twiddle_blocks(static_cast<int>(plan.C), hi, plan.nhi, twR, R), 256, 0, s>>>(
        twC, static_cast<int>(plan.C), hi, 1 << plan.tw_shift, plan.nhi, plan.b, twR, R);
  }
  if (!plan.fast) {
    dim3 grid(static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 64)), plan.nrows, 2 * plan.d);
    {
      ProfScope prof_scope("k_frontend_twiddles", s);
      k_frontend_twiddles<<<grid, 256, 0, s>>>(h->d_hs, h->d_perm, n, plan.b, plan.nrows, twfe);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  if (plan.fast) {
    e = plan.ws ? launch_sketch_ws(plan, h, A, lda, B, ldb, n1, n2, n3, partial,
                                   reinterpret_cast<float2*>(ws + plan.off_thi), s)
                : launch_sketch_fast(plan, h, A, lda, B, ldb, n1, n2, n3, partial, s);
    if (e != cudaSuccess) return e;
  } else {
  SketchArgs a{};
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
  a.n1 = static_cast<int>(n1); a.n2 = static_cast<int>(n2); a.n3 = static_cast<int>(n3); a.n = n;
  a.b = plan.b; a.R = static_cast<int>(plan.R); a.C = static_cast<int>(plan.C);
  a.nrows = plan.nrows; a.d = plan.d;
  a.nradC = plan.nradC;
  for (int i = 0; i < 16; ++i) a.radC[i] = plan.radC[i];
  a.G = plan.G; a.kchunk = static_cast<int>(plan.kchunk); a.nkc = plan.nkc;
  a.perm = h->d_perm; a.off = h->d_off; a.twfe = twfe; a.twC = twC; a.partial = partial;
  const unsigned ntask = static_cast<unsigned>(static_cast<int64_t>(plan.d) * plan.nrows * plan.nkc);
  const int smem = static_cast<int>(plan.smem);
  switch (dt) {
    case CMS_F32:
      e = cudaFuncSetAttribute(k_sketch_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) {
        ProfScope prof_scope("k_sketch_fused", s);
        k_sketch_fused<float><<<ntask, plan.threads, smem, s>>>(a);
      }
      break;
    case CMS_BF16:
      e = cudaFuncSetAttribute(k_sketch_fused<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) {
        ProfScope prof_scope("k_sketch_fused", s);
        k_sketch_fused<__nv_bfloat16><<<ntask, plan.threads, smem, s>>>(a);
      }
      break;
    default:
      e = cudaFuncSetAttribute(k_sketch_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) {
        ProfScope prof_scope("k_sketch_fused", s);
        k_sketch_fused<double><<<ntask, plan.threads, smem, s>>>(a);
      }
      break;
  }
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  }

  return launch_inverse(plan, partial, V, twC, twR, c, s);
}

cudaError_t launch_frontend_twiddles(const SketchPlan& plan, const cms_hashes* h, char* ws, cudaStream_t s) {
  const int n = static_cast<int>(h->n);
  float2* twfe = reinterpret_cast<float2*>(ws + plan.off_twfe);
  dim3 grid(static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 64)), plan.nrows, 2 * plan.d);
  {
    ProfScope prof_scope("k_frontend_twiddles", s);
    k_frontend_twiddles<<<grid, 256, 0, s>>>(h->d_hs, h->d_perm, n, plan.b, plan.nrows, twfe);
  }
  return cudaGetLastError();
}

cudaError_t launch_twiddle_tables(float2* twC, int C, float2* twR, int R, cudaStream_t s) {
  {
    ProfScope prof_scope("k_twiddle_table", s);
    k_twiddle_table<<<twiddle_blocks(C, nullptr, 0, twR, R), 256, 0, s>>>(twC, C, nullptr, 1, 0, 1, twR, R);
  }
  return cudaGetLastError();
}

cudaError_t launch_inverse(const SketchPlan& plan, const float2* partial, float2* V, const float2* twC,
                           const float2* twR, float* c, cudaStream_t s, const int32_t* skip_if_zero) {
  cudaError_t e = cudaSuccess;
  InvArgs ia{};
  ia.b = plan.b; ia.R = static_cast<int>(plan.R); ia.C = static_cast<int>(plan.C);
  ia.nrows = plan.nrows; ia.d = plan.d; ia.nkc = plan.nkc;
  ia.nradC = plan.nradC;
  for (int i = 0; i < 16; ++i) ia.radC[i] = plan.radC[i];
  ia.partial = partial; ia.twC = twC; ia.V = V; ia.skip_if_zero = skip_if_zero;
  const int smem2 = static_cast<int>(3 * plan.C * 8);
  if (smem2 > 48 * 1024) {
    e = cudaFuncSetAttribute(k_rows_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2);
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope prof_scope("k_rows_inverse", s);
    k_rows_inverse<<<static_cast<unsigned>(plan.d * plan.nrows), 256, smem2, s>>>(ia);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_cols_inverse(plan, V, twR, c, s, skip_if_zero);
}

size_t inverse_batch_bytes(int count) {
  const size_t n = static_cast<size_t>(std::max(count, 1));
  return align256(n * sizeof(InvArgs)) + align256(n * sizeof(ColsArgs)) + 2 * align256((n + 1) * sizeof(int));
}

cudaError_t build_inverse_batch(const std::vector<InverseSpec>& specs, void* d_buf, InverseBatch* out,
                                cudaStream_t s) {
  const int count = static_cast<int>(specs.size());
  std::vector<InvArgs> rows(count);
  std::vector<ColsArgs> cols(count);
  std::vector<int> rstart(count + 1), cstart(count + 1);
  int tr = 0, tc = 0;
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    const SketchPlan& plan = *specs[i].plan;
    InvArgs ia{};
    ia.b = plan.b; ia.R = static_cast<int>(plan.R); ia.C = static_cast<int>(plan.C);
    ia.nrows = plan.nrows; ia.d = plan.d; ia.nkc = plan.nkc;
    ia.nradC = plan.nradC;
    for (int r = 0; r < 16; ++r) ia.radC[r] = plan.radC[r];
    ia.partial = specs[i].partial; ia.twC = specs[i].twC; ia.V = specs[i].V; ia.skip_if_zero = nullptr;
    rows[i] = ia;
    rstart[i] = tr;
    tr += plan.d * plan.nrows;
    smem = std::max(smem, static_cast<size_t>(3 * plan.C * 8));
    ColsArgs ca{};
    ca.V = specs[i].V; ca.twR = specs[i].twR; ca.c = specs[i].c; ca.b = plan.b;
    ca.R = static_cast<int>(plan.R); ca.C = static_cast<int>(plan.C); ca.nrows = plan.nrows;
    ca.nbx = static_cast<int>((plan.b + 255) / 256);
    cols[i] = ca;
    cstart[i] = tc;
    tc += ca.nbx * plan.d;
  }
  rstart[count] = tr;
  cstart[count] = tc;
  char* base = static_cast<char*>(d_buf);
  const size_t o_rows = 0;
  const size_t o_cols = o_rows + align256(static_cast<size_t>(std::max(count, 1)) * sizeof(InvArgs));
  const size_t o_rs = o_cols + align256(static_cast<size_t>(std::max(count, 1)) * sizeof(ColsArgs));
  const size_t o_cs = o_rs + align256(static_cast<size_t>(count + 1) * sizeof(int));
  cudaError_t e = cudaMemcpyAsync(base + o_rows, rows.data(), count * sizeof(InvArgs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_cols, cols.data(), count * sizeof(ColsArgs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_rs, rstart.data(), (count + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_cs, cstart.data(), (count + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
  out->buf = d_buf;
  out->count = count;
  out->row_blocks = tr;
  out->col_blocks = tc;
  out->smem = smem;
  out->o_rows = o_rows; out->o_cols = o_cols; out->o_rs = o_rs; out->o_cs = o_cs;
  return e;
}

cudaError_t launch_inverse_batched(const InverseBatch& ib, cudaStream_t s) {
  if (ib.count == 0) return cudaSuccess;
  const char* base = static_cast<const char*>(ib.buf);
  cudaError_t e = cudaSuccess;
  if (ib.smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_rows_inverse_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(ib.smem));
    if (e != cudaSuccess) return e;
  }
  if (ib.row_blocks > 0) {
    ProfScope prof_scope("k_rows_inverse_batched", s);
    k_rows_inverse_batched<<<static_cast<unsigned>(ib.row_blocks), 256, ib.smem, s>>>(
        reinterpret_cast<const InvArgs*>(base + ib.o_rows), reinterpret_cast<const int*>(base + ib.o_rs), ib.count);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ib.col_blocks > 0) {
    ProfScope prof_scope("k_cols_inverse_batched", s);
    k_cols_inverse_batched<<<static_cast<unsigned>(ib.col_blocks), 256, 0, s>>>(
        reinterpret_cast<const ColsArgs*>(base + ib.o_cols), reinterpret_cast<const int*>(base + ib.o_cs), ib.count);
  }
  return cudaGetLastError();
}

cudaError_t launch_cols_inverse(const SketchPlan& plan, const float2* V, const float2* twR, float* c,
                                cudaStream_t s, const int32_t* skip_if_zero) {
  const int R = static_cast<int>(plan.R), C = static_cast<int>(plan.C);
  int rad[16];
  // long columns: an FFT per column (nv columns per block, 128 KB of shared
  // memory at most) instead of the direct sum over the R/2 + 1 rows
  if (R >= 256 && R <= 8192 && factor_radices(R, rad, 16) >= 0) {
    const int nv = std::max(1, 8192 / R);
    const int smem = 2 * nv * R * static_cast<int>(sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(k_cols_inverse_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 g(static_cast<unsigned>((C + nv - 1) / nv), plan.d);
    {
      ProfScope prof_scope("k_cols_inverse", s);
      k_cols_inverse_fft<<<g, 256, smem, s>>>(V, twR, plan.b, R, C, plan.nrows, nv, c, skip_if_zero);
    }
    return cudaGetLastError();
  }
  dim3 g2(static_cast<unsigned>((plan.b + 255) / 256), plan.d);
  {
    ProfScope prof_scope("k_cols_inverse", s);
    k_cols_inverse<<<g2, 256, 0, s>>>(V, twR, plan.b, static_cast<int>(plan.R), static_cast<int>(plan.C),
                                      plan.nrows, c, skip_if_zero);
  }
  return cudaGetLastError();
}

}  // namespace cms
