// k_sketch_ws.cu - warp-specialised form of the C = 1024 fused sketch kernel
// (the computation of k_sketch_fast, see there and k_sketch.cu for the
// four-step split of the length-b DFT and the pruned first stage).
//
// In the lock-step kernel all warps gather (front end) and then all warps
// run FFTs, so the gather, bound by shared-memory latency and bank traffic,
// never overlaps the FP32-bound FFTs.  Here the two run in different warps
// of a 512-thread block (one block per SM):
//
//  * warps 8-15 (front end, 64 registers after setmaxnreg.dec): gather
//    Y[f1][z2] = sum s(x) A_xk w_b^{f1 h(x)} for two rows f1 and a group of
//    G = 2 inner indices into one of two Y buffers.  Their per-entry
//    twiddles live in tensor memory (TMEM), 32 columns per (side, bucket
//    group) item; an item's count selects a fully unrolled body whose index
//    loads, gathers and TMEM load are all in flight together;
//  * warps 0-7 (FFT, 192 registers after setmaxnreg.inc): one length-1024
//    FFT per warp and group (row, side, inner index) from the other Y
//    buffer, the spectral products in registers and the Kahan folds into
//    shared memory;
//  * the TMA bulk copies of the staging rows (two buffers) are issued by
//    the first front-end thread for the first two groups, then by the first
//    FFT thread as soon as the front end has released a buffer.
// The FFT warps, the critical path, have the lower warp indices: with the
// front end on warps 8-15 the kernel runs 0.6% faster than the other way
// round (the schedulers appear to favour lower warps among ready ones).
//
// Hand-offs: staging full is an mbarrier (TMA transaction count) with a
// bounded wait; Y full and Y free are named barriers (bar.arrive by the
// producing warps, bar.sync by the consuming ones), on which waiting warps
// take no issue slots.  After a timed-out copy the block records the error
// and stops waiting for copies (the results are then garbage and reported
// as such) but still passes every named barrier, so no warp is left behind.
#include <algorithm>
#include <cstdlib>
#include <atomic>

#include "cms_internal.h"
#include "warp_fft.cuh"

namespace cms {
namespace {

using namespace wfft;

constexpr int kC = kFeC;                 // 1024
constexpr int kG = 2;                    // inner indices per group
constexpr int kRows = 2;                 // rows f1 per block
constexpr int kFeWarps = 8;
constexpr int kFftWarps = kRows * 2 * kG;   // 8
constexpr int kThreadsWs = 32 * (kFeWarps + kFftWarps);   // 512
constexpr int kFeThreads = 32 * kFeWarps;
constexpr int kFftThreads = 32 * kFftWarps;
constexpr int kFlush = 32;               // groups between Kahan folds
constexpr int kPitch = 33;
constexpr int kRegion = 32 * kPitch;     // float2 per FFT region (>= kC)
constexpr int kItems = 2 * (kC / 32);    // (side, bucket group) items: 64
constexpr int kItemsFe = kItems / kFeWarps;   // 8 per front-end warp
// registers per thread after setmaxnreg (launch: 65536 / 512 = 128 each)
constexpr int kRegsFe = 64;
constexpr int kRegsFft = 192;
static_assert(kFeThreads * kRegsFe + kFftThreads * kRegsFft <= 65536, "register split exceeds the launch pool");
// named barriers (0 is __syncthreads)
constexpr int kBarPair = 2;              // 2..5: FFT warp pairs, 64 threads
constexpr int kBarFft = 6;               // FFT warps, 256 threads
constexpr int kBarYFull = 7;             // 7, 8: Y buffer b written (front end arrives, FFT syncs)
constexpr int kBarYFree = 9;             // 9, 10: Y buffer b consumed (FFT arrives, front end syncs)
constexpr int kBarFeOvf = 11;            // front-end warps: overflow cache written
// tensor-memory columns of a lane quarter: front-end records of the two
// front-end warps sharing it (kFeColCap each), then two 64-column buffers
// through which the partner FFT warps of that quarter swap half spectra
constexpr uint32_t kFeColCap = 192;
constexpr uint32_t kXCol = 2 * kFeColCap;   // 384

__device__ uint32_t g_ws_error = 0;      // 1: a wait gave up

struct WsArgs {
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb;
  int n1, n2, n3, n, npad;
  int64_t b;
  int nrows, nunits;
  int kchunk, nkc;
  int alias;
  uint32_t ecap;
  int tw_shift, nhi;
  const uint32_t* rec_x;
  const uint32_t* rec_hs;
  const uint32_t* grp;
  const uint16_t* dest;
  const uint32_t* ovf_off;
  const uint32_t* ovf_x;
  const uint32_t* ovf_hs;  // packed hash of each overflow entry
  const uint8_t* assign;   // [t][side][32]: bucket group of (front-end warp, slot)
  float2* partial;
  const float2* thi_g;  // w_b^{i 2^tw_shift}, i < nhi (k_twiddle_table, FP64)
  int ovcap;          // overflow entries whose twiddles the prologue caches
  int force_xsmem;    // debug: swap half spectra through shared memory
};

struct WsLayout {
  size_t stage, rec_x, ybuf, acc, tlo, thi, wmeta, wdst, ibase, istart, wcls, wcol, wext, ovf, wovf, ovtw, ovx, bars, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

// Staging: [buffer][side][k slot][npad] (one side when A and B alias).
__host__ __device__ inline size_t stage_floats(int npad, int alias) {
  return static_cast<size_t>(alias ? 1 : 2) * kG * npad;
}

__host__ __device__ inline WsLayout ws_layout(int npad, uint32_t ecap, int alias, int tw_shift, int nhi,
                                              int ovcap) {
  WsLayout L{};
  size_t o = 0;
  L.stage = o;  o = al16(o + 2 * stage_floats(npad, alias) * 4);
  L.rec_x = o;  o = al16(o + static_cast<size_t>(2) * ecap * 2);
  L.ybuf = o;   o = al16(o + static_cast<size_t>(2) * kFftWarps * kRegion * 8);
  L.acc = o;    o = al16(o + static_cast<size_t>(kRows) * kC * 16);
  L.tlo = o;    o = al16(o + (static_cast<size_t>(1) << tw_shift) * 8);
  L.thi = o;    o = al16(o + static_cast<size_t>(nhi) * 8);
  L.wmeta = o;  o = al16(o + static_cast<size_t>(kItems) * 4);
  L.wdst = o;   o = al16(o + static_cast<size_t>(kFeWarps) * 32 * kItemsFe * 2);
  L.ibase = o;  o = al16(o + static_cast<size_t>(kItems) * 4);
  L.istart = o; o = al16(o + static_cast<size_t>(kItems + 1) * 4);
  L.wcls = o;   o = al16(o + static_cast<size_t>(kFeWarps) * 16);
  L.wcol = o;   o = al16(o + static_cast<size_t>(kItems) * 2);
  L.wext = o;   o = al16(o + static_cast<size_t>(kItems + kFeWarps) * 2);
  L.ovf = o;    o = al16(o + static_cast<size_t>(2) * (kC + 1) * 2);
  L.wovf = o;   o = al16(o + static_cast<size_t>(kFeWarps) * 4);
  L.ovtw = o;   o = al16(o + static_cast<size_t>(ovcap) * 16);
  L.ovx = o;    o = al16(o + static_cast<size_t>(ovcap) * 2);
  L.bars = o;   o = al16(o + 2 * 8);
  L.total = o;
  return L;
}

__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Producer side of a named barrier: signals arrival without waiting (the
// hardware orders this thread's prior shared-memory accesses before it).
__device__ __forceinline__ void named_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Item j (0..7) of front-end warp w: side j div 4, and the bucket group that
// the table builder dealt to slot 4 w + (j mod 4) of that side (groups
// balanced over the warps by padded count plus longest overflow list).
__device__ __forceinline__ int fe_group(const WsArgs& p, int t, int w, int j) {
  return p.assign[(static_cast<size_t>(t) * 2 + (j >> 2)) * (kC / 32) + w * 4 + (j & 3)];
}

// Tensor-memory loads of N consecutive columns of this thread's row into
// r[0..N-1], without waiting (N = 4, 8, 16; the column is a multiple of N).
template <int N>
__device__ __forceinline__ void tmem_ld_part(uint32_t taddr, uint32_t* r) {
  if constexpr (N == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
  } else if constexpr (N == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
  } else {
    static_assert(N == 16, "4, 8 or 16 columns");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
  }
}

// Wait for this thread's tensor-memory loads into a[0..15] and b[0..3].
__device__ __forceinline__ void tmem_wait_ld16_4(uint32_t (&a)[32], uint32_t (&b)[4]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]),
                 "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]),
                 "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3])
               :
               : "memory");
}

// The records of a chunk: NCOL = 4, 8, 12 or 16 columns from a column that
// is a multiple of 16 (or of NCOL below 16), 20, 24, 28 or 32 columns from a
// multiple of 32; each load starts on a multiple of its own size.
template <int NCOL>
__device__ __forceinline__ void tmem_ld_chunk(uint32_t taddr, uint32_t (&r)[32]) {
  if constexpr (NCOL == 32) {
    tmem_ld32_nowait(taddr, r);
  } else {
    constexpr int A16 = NCOL & 16, A8 = NCOL & 8, A4 = NCOL & 4;
    if constexpr (A16 != 0) tmem_ld_part<16>(taddr, r);
    if constexpr (A8 != 0) tmem_ld_part<8>(taddr + A16, r + A16);
    if constexpr (A4 != 0) tmem_ld_part<4>(taddr + A16 + A8, r + A16 + A8);
  }
}

// Tensor-memory footprint of a chunk of K items of count C: 32 columns for
// C >= 5, 16 columns otherwise (C = 1 chunks hold 4 items, C = 2 chunks 2);
// a lone item of count 1 takes 4 columns of its block.
template <int C, int K>
__device__ __forceinline__ constexpr int fe_chunk_cols() {
  return C >= 5 ? 32 : (C == 1 && K == 1 ? 4 : 16);
}

// K consecutive items of count C (C padded entries per lane each): every
// index load, gather and the tensor-memory load of the chunk are in flight
// together, then each item's 2 x 2 sums (rows x inner indices) go to its Y
// slot.  The first entry of a sum is a product, the rest are FMAs.
template <int C, int K>
__device__ __forceinline__ void fe_chunk(const uint16_t*& xp, uint32_t& tc, int& pos, const uint16_t* wd,
                                         float2* work, const float* st0, const float* st1) {
  constexpr int S = C * K;
  uint32_t tw[32];
  tmem_ld_chunk<4 * S>(tc, tw);
  int x[S];
#pragma unroll
  for (int e = 0; e < S; ++e) x[e] = xp[32 * e];
  float v0[S], v1[S];
#pragma unroll
  for (int e = 0; e < S; ++e) {
    v0[e] = st0[x[e]];
    v1[e] = st1[x[e]];
  }
  if constexpr (4 * S <= 16) tmem_wait_ld16(tw);
  else tmem_wait_ld32(tw);
#pragma unroll
  for (int it = 0; it < K; ++it) {
    float2 a00, a01, a10, a11;   // [row][k]
#pragma unroll
    for (int e = 0; e < C; ++e) {
      const int q = it * C + e;
      const float w0 = __uint_as_float(tw[4 * q]), w1 = __uint_as_float(tw[4 * q + 1]);
      const float w2 = __uint_as_float(tw[4 * q + 2]), w3 = __uint_as_float(tw[4 * q + 3]);
      if (e == 0) {
        a00 = make_float2(v0[q] * w0, v0[q] * w1);
        a01 = make_float2(v1[q] * w0, v1[q] * w1);
        a10 = make_float2(v0[q] * w2, v0[q] * w3);
        a11 = make_float2(v1[q] * w2, v1[q] * w3);
      } else {
        a00.x = fmaf(v0[q], w0, a00.x); a00.y = fmaf(v0[q], w1, a00.y);
        a01.x = fmaf(v1[q], w0, a01.x); a01.y = fmaf(v1[q], w1, a01.y);
        a10.x = fmaf(v0[q], w2, a10.x); a10.y = fmaf(v0[q], w3, a10.y);
        a11.x = fmaf(v1[q], w2, a11.x); a11.y = fmaf(v1[q], w3, a11.y);
      }
    }
    float2* dp = work + wd[32 * (pos + it)];
    dp[0] = a00;
    dp[kRegion] = a01;
    dp[2 * kG * kRegion] = a10;
    dp[2 * kG * kRegion + kRegion] = a11;
  }
  pos += K;
  xp += 32 * S;
  tc += fe_chunk_cols<C, K>();
}

// The n items of count C of a front-end warp, in chunks of 4 (C = 1) or 2
// (C = 2) items where whole chunks remain, then one item at a time (a lone
// item of count 2 keeps a 16-column block to itself, one of count 1 takes 4
// columns of the last block).
template <int C>
__device__ __forceinline__ void fe_class(int n, const uint16_t*& xp, uint32_t& tc, int& pos, const uint16_t* wd,
                                         float2* work, const float* st0, const float* st1) {
  constexpr int K = C == 1 ? 4 : (C == 2 ? 2 : 1);
  int i = 0;
  if constexpr (K > 1) {
#pragma unroll 1
    for (; i + K <= n; i += K) fe_chunk<C, K>(xp, tc, pos, wd, work, st0, st1);
  }
#pragma unroll 1
  for (; i < n; ++i) fe_chunk<C, 1>(xp, tc, pos, wd, work, st0, st1);
}

__global__ void __launch_bounds__(kThreadsWs, 1) k_sketch_ws(WsArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_err;
  __shared__ int s_xsmem;   // 1: some front-end warp needs more than kFeColCap columns

  const WsLayout L = ws_layout(p.npad, p.ecap, p.alias, p.tw_shift, p.nhi, p.ovcap);
  float* stage = reinterpret_cast<float*>(sm + L.stage);
  uint16_t* rec_x = reinterpret_cast<uint16_t*>(sm + L.rec_x);     // [stream slot][lane]
  float2* ybuf = reinterpret_cast<float2*>(sm + L.ybuf);           // [buffer][FFT warp][kRegion]
  float4* acc = reinterpret_cast<float4*>(sm + L.acc);
  float2* tlo = reinterpret_cast<float2*>(sm + L.tlo);
  float2* thi = reinterpret_cast<float2*>(sm + L.thi);
  uint32_t* wmeta = reinterpret_cast<uint32_t*>(sm + L.wmeta);     // [fe warp][item]: cnt | side << 8 | longest overflow list << 9 | ovf << 31
  uint16_t* wdst = reinterpret_cast<uint16_t*>(sm + L.wdst);       // [fe warp][item][lane]: Y slot (row 0, k 0)
  uint32_t* ibase = reinterpret_cast<uint32_t*>(sm + L.ibase);     // [fe warp][item]: side * ecap + first record
  uint32_t* istart = reinterpret_cast<uint32_t*>(sm + L.istart);   // [fe warp][item]: first stream slot
  uint8_t* wcls = reinterpret_cast<uint8_t*>(sm + L.wcls);         // [fe warp][count]: items of that count
  uint16_t* wcol = reinterpret_cast<uint16_t*>(sm + L.wcol);       // [fe warp][item]: first TMEM column
  // [fe warp][item]: first TMEM column of the item's overflow records (none:
  // 0xFFFF); then [fe warp]: end of the warp's item records
  uint16_t* wext = reinterpret_cast<uint16_t*>(sm + L.wext);
  uint16_t* ovf = reinterpret_cast<uint16_t*>(sm + L.ovf);
  uint32_t* wovf = reinterpret_cast<uint32_t*>(sm + L.wovf);
  float4* ovtw = reinterpret_cast<float4*>(sm + L.ovtw);         // cached overflow twiddles (both rows)
  uint16_t* ovx = reinterpret_cast<uint16_t*>(sm + L.ovx);       // their staging indices
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* full_stage = bars;       // [2] TMA transactions of a staging buffer

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int task = blockIdx.x;
  const int kc = task % p.nkc;
  const int unit = (task / p.nkc) % p.nunits;
  const int t = task / (p.nkc * p.nunits);
  uint32_t f1r[kRows];
  f1r[0] = static_cast<uint32_t>(2 * unit);
  f1r[1] = static_cast<uint32_t>(min(2 * unit + 1, p.nrows - 1));
  const bool row1_live = 2 * unit + 1 < p.nrows;
  const int n = p.n;
  const int S = 1 << p.tw_shift;
  const ModB modb = make_modb(p.b);
  const int nside = p.alias ? 1 : 2;
  const size_t sbuf = stage_floats(p.npad, p.alias);
  const int k_begin = kc * p.kchunk;
  const int k_end = min(p.n2, k_begin + p.kchunk);
  const int ngroups = k_end > k_begin ? (k_end - k_begin + kG - 1) / kG : 0;

  // ---- tensor memory: 512 columns for the block (one block per SM) --------
  if (warp == 0) {
    tmem_alloc(&s_tmem, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    s_err = 0;
    s_xsmem = p.force_xsmem;
  }

  // ---- prologue -------------------------------------------------------------
  for (int i = tid; i < S; i += kThreadsWs) {
    float s, c;
    sincospif(2.0f * static_cast<float>(i) / static_cast<float>(p.b), &s, &c);
    tlo[i] = make_float2(c, -s);
  }
  for (int i = tid; i < p.nhi; i += kThreadsWs) thi[i] = p.thi_g[i];
  if (tid < kItems) {
    const int w = tid / kItemsFe, j = tid % kItemsFe;
    const int side = j >> 2, gi = fe_group(p, t, w, j);
    const size_t ts = static_cast<size_t>(t) * 2 + side;
    const uint32_t gb = p.grp[(ts * (kC / 32) + gi) * 2];
    const uint32_t gy = p.grp[(ts * (kC / 32) + gi) * 2 + 1];
    wmeta[tid] = (gy & 0xFFu) | (static_cast<uint32_t>(side) << 8) | (((gy >> 16) & 0x7FFFu) << 9) |
                 (gy & 0x80000000u);
    ibase[tid] = static_cast<uint32_t>(side) * p.ecap + gb;
  }
  for (int i = tid; i < kFeWarps * 32 * kItemsFe; i += kThreadsWs) {
    const int w = i / (32 * kItemsFe), j = (i / 32) % kItemsFe, l = i % 32;   // [w][j][l]
    const int side = j >> 2, gi = fe_group(p, t, w, j);
    const size_t ts = static_cast<size_t>(t) * 2 + side;
    wdst[i] = static_cast<uint16_t>(side * kG * kRegion + p.dest[ts * kC + gi * 32 + l]);
  }
  for (int side = 0; side < 2; ++side) {
    const size_t ts = static_cast<size_t>(t) * 2 + side;
    for (int i = tid; i <= kC; i += kThreadsWs)
      ovf[side * (kC + 1) + i] = static_cast<uint16_t>(p.ovf_off[ts * (kC + 1) + i]);
  }
  for (int i = tid; i < kRows * kC; i += kThreadsWs) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  // zero the staging tails [n_side, npad) of both buffers: entries x >= n_side read zeros
  for (int bb = 0; bb < 2; ++bb)
    for (int s2 = 0; s2 < nside; ++s2) {
      const int ns = s2 == 0 ? p.n1 : p.n3;
      for (int g = 0; g < kG; ++g)
        for (int i = ns + tid; i < p.npad; i += kThreadsWs)
          stage[bb * sbuf + (s2 * kG + g) * p.npad + i] = 0.f;
    }
  if (tid == 0) {
    mbar_init(&full_stage[0], 1);
    mbar_init(&full_stage[1], 1);
    fence_proxy_async();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = s_tmem;
  // each front-end warp's items in order of decreasing count (stable), so
  // that its group loop runs one unrolled body per count class
  {
    int rank = 0;
    uint32_t pm_meta = 0, pm_base = 0;
    uint16_t pm_dst[32];
    if (tid < kItems) {
      const int w = tid / kItemsFe, j = tid % kItemsFe;
      const uint32_t cj = wmeta[tid] & 0xFFu;
#pragma unroll
      for (int i = 0; i < kItemsFe; ++i) {
        const uint32_t ci = wmeta[w * kItemsFe + i] & 0xFFu;
        rank += (ci > cj || (ci == cj && i < j)) ? 1 : 0;
      }
      pm_meta = wmeta[tid];
      pm_base = ibase[tid];
#pragma unroll
      for (int l = 0; l < 32; ++l) pm_dst[l] = wdst[(w * kItemsFe + j) * 32 + l];
    }
    __syncthreads();
    if (tid < kItems) {
      const int w = tid / kItemsFe;
      wmeta[w * kItemsFe + rank] = pm_meta;
      ibase[w * kItemsFe + rank] = pm_base;
#pragma unroll
      for (int l = 0; l < 32; ++l) wdst[(w * kItemsFe + rank) * 32 + l] = pm_dst[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    uint32_t s = 0;
    for (int i = 0; i < kItems; ++i) { istart[i] = s; s += wmeta[i] & 0xFFu; }
    istart[kItems] = s;
  }
  if (tid < kFeWarps) {
    uint32_t f = 0, cnt[kItemsFe];
#pragma unroll
    for (int j = 0; j < kItemsFe; ++j) {
      const uint32_t m = wmeta[tid * kItemsFe + j];
      f |= m >> 31;
      cnt[j] = m & 0xFFu;
    }
    wovf[tid] = f;
    int ncls[9];
#pragma unroll
    for (int c = 0; c <= 8; ++c) {
      int k = 0;
#pragma unroll
      for (int j = 0; j < kItemsFe; ++j) k += cnt[j] == static_cast<uint32_t>(c) ? 1 : 0;
      ncls[c] = k;
      wcls[tid * 16 + c] = static_cast<uint8_t>(k);
    }
    // tensor-memory columns of the items (decreasing count): 32 per item of
    // count >= 5, 16 per item of count 3 or 4, 16 per pair of count 2 and
    // per quad of count 1 (a lone pair or quad member at the start of its
    // block), so every chunk load starts on a multiple of its size; at most
    // 8 x 32 = 256 columns per warp
    uint32_t col = 0;
    int q = 0;
#pragma unroll
    for (int c = 8; c >= 1; --c)
      for (int i = 0; i < ncls[c]; ++i, ++q) {
        if (c >= 5) { wcol[tid * kItemsFe + q] = static_cast<uint16_t>(col); col += 32; }
        else if (c >= 3) { wcol[tid * kItemsFe + q] = static_cast<uint16_t>(col); col += 16; }
        else if (c == 2) {
          wcol[tid * kItemsFe + q] = static_cast<uint16_t>(col + 8 * (i & 1));
          if ((i & 1) || i + 1 == ncls[c]) col += 16;
        } else {
          wcol[tid * kItemsFe + q] = static_cast<uint16_t>(col + 4 * (i & 3));
          if ((i & 3) == 3 || i + 1 == ncls[c]) col += 16;
        }
      }
    for (; q < kItemsFe; ++q) wcol[tid * kItemsFe + q] = 0;
    wext[kItems + tid] = static_cast<uint16_t>(col);
    // more records than the warp's share of its quarter: this block keeps
    // the full halves for the records and swaps spectra in shared memory
    if (col > kFeColCap) atomicOr(&s_xsmem, 1);
  }
  __syncthreads();
  const bool xsmem = s_xsmem != 0;

  // TMA copies of group g into staging buffer g & 1 (thread 0 only)
  auto issue = [&](int g) {
    const int k0 = k_begin + g * kG;
    const int gl = min(kG, k_end - k0);
    float* st = stage + (g & 1) * sbuf;
    uint32_t bytes = 0;
    for (int gg = 0; gg < gl; ++gg) bytes += static_cast<uint32_t>(p.n1) * 4u;
    if (!p.alias)
      for (int gg = 0; gg < gl; ++gg) bytes += static_cast<uint32_t>(p.n3) * 4u;
    // the staging buffer was last read by generic loads that completed
    // before the front-end barrier; no proxy fence is needed for that order
    mbar_arrive_expect_tx(&full_stage[g & 1], bytes);
    for (int gg = 0; gg < gl; ++gg) {
      if (p.n1 > 0)
        bulk_g2s(st + gg * p.npad, p.A + static_cast<size_t>(k0 + gg) * p.lda, static_cast<uint32_t>(p.n1) * 4u,
                 &full_stage[g & 1]);
      if (!p.alias && p.n3 > 0)
        bulk_g2s(st + (kG + gg) * p.npad, p.B + static_cast<size_t>(k0 + gg) * p.ldb,
                 static_cast<uint32_t>(p.n3) * 4u, &full_stage[g & 1]);
    }
  };

  if (warp >= kFftWarps) {
    // ======================= front-end warps =================================
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsFe));
    const int w = warp - kFftWarps;
    const int fe_tid = tid - kFftThreads;
    // lane quarter w mod 4; columns [0, kFeColCap) or [kFeColCap, kXCol)
    // by w div 4 (halves of 256 when the block swaps spectra in shared memory)
    const uint32_t tq = tmem + ((32u * static_cast<uint32_t>(w & 3)) << 16) +
                        (xsmem ? 256u : kFeColCap) * static_cast<uint32_t>(w >> 2);
    // the first two groups' copies fly while the records are built
    if (fe_tid == 0) {
      if (ngroups > 0) issue(0);
      if (ngroups > 1) issue(1);
    }
    // records: staging index of x (shared memory, stream order) and
    // s(x) w_b^{(h(x) f1) mod b} for both rows (TMEM: entry r of item j at
    // column wcol[j] + 4 r); padding entries (x = n) read the zeroed staging
    // tail
    {
      const size_t tbase = static_cast<size_t>(t) * 2 * p.ecap;
#pragma unroll 1
      for (int j = 0; j < kItemsFe; ++j) {
        const uint32_t c = wmeta[w * kItemsFe + j] & 0xFFu;
        const uint32_t b0 = ibase[w * kItemsFe + j];
        const uint32_t s0 = istart[w * kItemsFe + j];
#pragma unroll 1
        for (uint32_t r = 0; r < c; ++r) {
          const uint32_t src = b0 + 32u * r + static_cast<uint32_t>(lane);
          const uint32_t side = src >= p.ecap ? 1u : 0u;
          const uint32_t x = p.rec_x[tbase + src];
          const uint32_t hv = p.rec_hs[tbase + src];
          float2 tw[kRows];
#pragma unroll
          for (int rr = 0; rr < kRows; ++rr) {
            tw[rr] = make_float2(0.f, 0.f);
            if (x < static_cast<uint32_t>(n)) {
              tw[rr] = wb(tlo, thi, mulmod(hv & kBucketMask, f1r[rr], modb), p.tw_shift);
              if (hv >> 31) { tw[rr].x = -tw[rr].x; tw[rr].y = -tw[rr].y; }
            }
          }
          tmem_st4(tq + static_cast<uint32_t>(wcol[w * kItemsFe + j]) + 4u * r,
                   make_float4(tw[0].x, tw[0].y, tw[1].x, tw[1].y));
          const uint32_t xs = min(x, static_cast<uint32_t>(n));
          rec_x[(s0 + r) * 32u + lane] =
              static_cast<uint16_t>((p.alias ? 0u : side * kG * static_cast<uint32_t>(p.npad)) + xs);
        }
      }
      tmem_wait_st();
    }
    // overflow records: the entries past the capped count of an item's
    // buckets, for items whose lists fit the warp's free tensor-memory
    // columns after its records (heavy draws leave many items empty): step r
    // of the item (entry r of each lane's list, zero-padded to a multiple of
    // 4 steps) has its twiddles at column e + 4 r and its staging index at
    // column e + 4 om4 + r, e a multiple of 16
    {
      const uint16_t* wdx = wdst + w * kItemsFe * 32 + lane;
      if (lane == 0) {
        const uint32_t capw = xsmem ? 256u : kFeColCap;
        uint32_t ec = (static_cast<uint32_t>(wext[kItems + w]) + 15u) & ~15u;
        for (int j = 0; j < kItemsFe; ++j) {
          const uint32_t om = (wmeta[w * kItemsFe + j] >> 9) & 0x7FFFu;
          const uint32_t om4 = (om + 3u) & ~3u;
          uint16_t e = 0xFFFFu;
          if (om > 0 && ec + 5u * om4 <= capw) {
            e = static_cast<uint16_t>(ec);
            ec = (ec + 5u * om4 + 15u) & ~15u;
          }
          wext[w * kItemsFe + j] = e;
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int j = 0; j < kItemsFe; ++j) {
        const uint32_t e = wext[w * kItemsFe + j];
        if (e == 0xFFFFu) continue;
        const uint32_t m = wmeta[w * kItemsFe + j];
        const uint32_t om4 = (((m >> 9) & 0x7FFFu) + 3u) & ~3u;
        const uint32_t side = (m >> 8) & 1u;
        const uint32_t z2 = static_cast<uint32_t>(wdx[32 * j]) - side * static_cast<uint32_t>(kG * kRegion);
        const size_t ts = static_cast<size_t>(t) * 2 + side;
        const uint32_t soff = p.alias ? 0u : side * static_cast<uint32_t>(kG * p.npad);
        uint32_t o0 = 0, o1 = 0;
        if (z2 < static_cast<uint32_t>(kC)) {
          o0 = ovf[side * (kC + 1) + z2];
          o1 = ovf[side * (kC + 1) + z2 + 1];
        }
#pragma unroll 1
        for (uint32_t r = 0; r < om4; ++r) {
          float4 tw = make_float4(0.f, 0.f, 0.f, 0.f);
          uint32_t xs = 0;
          if (o0 + r < o1) {
            const uint32_t o = o0 + r;
            const uint32_t x = p.ovf_x[ts * n + o];
            const uint32_t hv = p.ovf_hs[ts * n + o];
            float2 w0 = wb(tlo, thi, mulmod(hv & kBucketMask, f1r[0], modb), p.tw_shift);
            float2 w1 = wb(tlo, thi, mulmod(hv & kBucketMask, f1r[1], modb), p.tw_shift);
            if (hv >> 31) { w0.x = -w0.x; w0.y = -w0.y; w1.x = -w1.x; w1.y = -w1.y; }
            tw = make_float4(w0.x, w0.y, w1.x, w1.y);
            xs = soff + x;
          }
          __syncwarp();   // the tensor-memory stores are warp-collective
          tmem_st4(tq + e + 4u * r, tw);
          tmem_st1(tq + e + 4u * om4 + r, xs);
        }
      }
      tmem_wait_st();
    }
    // twiddles of the entries past the capped count (overflow lists of both
    // sides), cached for the whole task up to the shared-memory capacity
    const uint32_t novf_a = ovf[kC];
    const uint32_t nov = min(novf_a + static_cast<uint32_t>(ovf[(kC + 1) + kC]),
                             static_cast<uint32_t>(p.ovcap));
    for (uint32_t i = static_cast<uint32_t>(fe_tid); i < nov; i += kFeThreads) {
      const uint32_t side = i >= novf_a ? 1u : 0u;
      const size_t ts = static_cast<size_t>(t) * 2 + side;
      const uint32_t x = p.ovf_x[ts * n + (i - side * novf_a)];
      const uint32_t hv = p.ovf_hs[ts * n + (i - side * novf_a)];
      float2 w0 = wb(tlo, thi, mulmod(hv & kBucketMask, f1r[0], modb), p.tw_shift);
      float2 w1 = wb(tlo, thi, mulmod(hv & kBucketMask, f1r[1], modb), p.tw_shift);
      if (hv >> 31) { w0.x = -w0.x; w0.y = -w0.y; w1.x = -w1.x; w1.y = -w1.y; }
      ovtw[i] = make_float4(w0.x, w0.y, w1.x, w1.y);
      ovx[i] = static_cast<uint16_t>((p.alias ? 0u : side * kG * static_cast<uint32_t>(p.npad)) + x);
    }
    named_sync(kBarFeOvf, kFeThreads);
    const uint32_t* wm = wmeta + w * kItemsFe;
    const uint16_t* wd = wdst + w * kItemsFe * 32 + lane;   // item j of this lane at wd[32 j]
    const uint16_t* xbase = rec_x + istart[w * kItemsFe] * 32u + lane;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      if (!s_err && !mbar_wait_bounded_sleep(&full_stage[b], (g >> 1) & 1)) s_err = 1;
      // the FFT warps are done with Y buffer b (group g - 2)
      if (g >= 2) named_sync(kBarYFree + b, kThreadsWs);
      const float* st0 = stage + b * sbuf;
      const float* st1 = st0 + p.npad;
      float2* work = ybuf + static_cast<size_t>(b) * kFftWarps * kRegion;
      // the items by count class, largest first (the order of the records)
      const uint16_t* xp = xbase;
      uint32_t tc = tq;
      int pos = 0;
      const uint8_t* ncl = wcls + w * 16;
      fe_class<8>(ncl[8], xp, tc, pos, wd, work, st0, st1);
      fe_class<7>(ncl[7], xp, tc, pos, wd, work, st0, st1);
      fe_class<6>(ncl[6], xp, tc, pos, wd, work, st0, st1);
      fe_class<5>(ncl[5], xp, tc, pos, wd, work, st0, st1);
      fe_class<4>(ncl[4], xp, tc, pos, wd, work, st0, st1);
      fe_class<3>(ncl[3], xp, tc, pos, wd, work, st0, st1);
      fe_class<2>(ncl[2], xp, tc, pos, wd, work, st0, st1);
      fe_class<1>(ncl[1], xp, tc, pos, wd, work, st0, st1);
      // empty bucket groups: zeros
#pragma unroll 1
      for (; pos < kItemsFe; ++pos) {
        float2* dp = work + wd[32 * pos];
        const float2 z = make_float2(0.f, 0.f);
        dp[0] = z;
        dp[kRegion] = z;
        dp[2 * kG * kRegion] = z;
        dp[2 * kG * kRegion + kRegion] = z;
      }
      // entries past the capped count of some bucket (rare): the lane that
      // stored the bucket's Y adds them, with on-the-fly twiddles
      if (wovf[w]) {
#pragma unroll 1
        for (int j = 0; j < kItemsFe; ++j) {
          const uint32_t m = wm[j];
          if (!(m >> 31)) continue;
          const uint32_t dst = wd[32 * j];
          const int side = static_cast<int>((m >> 8) & 1u);
          const int z2 = static_cast<int>(dst) - side * kG * kRegion;
          const size_t ts = static_cast<size_t>(t) * 2 + side;
          const uint32_t obase = side ? novf_a : 0u;
          const uint32_t soff = p.alias ? 0u : static_cast<uint32_t>(side * kG * p.npad);
          float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
          const uint32_t e = wext[w * kItemsFe + j];
          if (e != 0xFFFFu) {
            // from the overflow records, 4 steps per load
            const uint32_t om4 = (((m >> 9) & 0x7FFFu) + 3u) & ~3u;
#pragma unroll 1
            for (uint32_t r0 = 0; r0 < om4; r0 += 4) {
              uint32_t tw[32], xr[4];
              __syncwarp();
              tmem_ld_part<16>(tq + e + 4u * r0, tw);
              tmem_ld_part<4>(tq + e + 4u * om4 + r0, xr);
              tmem_wait_ld16_4(tw, xr);
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float v0 = st0[xr[i]];
                const float v1 = st1[xr[i]];
                const float w0 = __uint_as_float(tw[4 * i]), w1 = __uint_as_float(tw[4 * i + 1]);
                const float w2 = __uint_as_float(tw[4 * i + 2]), w3 = __uint_as_float(tw[4 * i + 3]);
                a00.x = fmaf(v0, w0, a00.x); a00.y = fmaf(v0, w1, a00.y);
                a01.x = fmaf(v1, w0, a01.x); a01.y = fmaf(v1, w1, a01.y);
                a10.x = fmaf(v0, w2, a10.x); a10.y = fmaf(v0, w3, a10.y);
                a11.x = fmaf(v1, w2, a11.x); a11.y = fmaf(v1, w3, a11.y);
              }
            }
          } else {
          const uint32_t o1 = ovf[side * (kC + 1) + z2 + 1];
          for (uint32_t o = ovf[side * (kC + 1) + z2]; o < o1; ++o) {
            float4 w;
            uint32_t xi;
            if (obase + o < nov) {
              w = ovtw[obase + o];
              xi = ovx[obase + o];
            } else {
              // beyond the cache: twiddles on the fly (rows f1 and f1 + 1,
              // or the same row twice: one reduction, the second phase
              // is the first plus h mod b)
              const uint32_t x = p.ovf_x[ts * n + o];
              const uint32_t hv = p.ovf_hs[ts * n + o];
              const uint32_t hb = hv & kBucketMask, bb = static_cast<uint32_t>(p.b);
              const uint32_t e0 = mulmod(hb, f1r[0], modb);
              uint32_t e1 = f1r[1] != f1r[0] ? e0 + hb : e0;
              if (e1 >= bb) e1 -= bb;
              float2 w0 = wb(tlo, thi, e0, p.tw_shift);
              float2 w1 = wb(tlo, thi, e1, p.tw_shift);
              if (hv >> 31) { w0.x = -w0.x; w0.y = -w0.y; w1.x = -w1.x; w1.y = -w1.y; }
              w = make_float4(w0.x, w0.y, w1.x, w1.y);
              xi = soff + x;
            }
            const float v0 = st0[xi];
            const float v1 = st1[xi];
            a00.x = fmaf(v0, w.x, a00.x); a00.y = fmaf(v0, w.y, a00.y);
            a01.x = fmaf(v1, w.x, a01.x); a01.y = fmaf(v1, w.y, a01.y);
            a10.x = fmaf(v0, w.z, a10.x); a10.y = fmaf(v0, w.w, a10.y);
            a11.x = fmaf(v1, w.z, a11.x); a11.y = fmaf(v1, w.w, a11.y);
          }
          }
          float2* dp = work + dst;
          dp[0].x += a00.x; dp[0].y += a00.y;
          dp[kRegion].x += a01.x; dp[kRegion].y += a01.y;
          dp[2 * kG * kRegion].x += a10.x; dp[2 * kG * kRegion].y += a10.y;
          dp[2 * kG * kRegion + kRegion].x += a11.x; dp[2 * kG * kRegion + kRegion].y += a11.y;
        }
      }
      // Y of group g is complete, and so are this thread's reads of staging
      // buffer b (the FFT side refills it once all 256 have arrived)
      named_arrive(kBarYFull + b, kThreadsWs);
    }
  } else {
    // ========================== FFT warps ====================================
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsFft));
    // warp f: side f >> 2, row (f >> 1) & 1, k slot f & 1; its partner (same
    // row and k slot, other side) is warp f ^ 4, in the same tensor-memory
    // lane quarter
    const int f = warp;
    const int ftid = tid;
    const int side_w = f >> 2;
    const int row_w = (f >> 1) & 1;
    const int g_w = f & 1;
    const int own_m0 = side_w * 16;
    const int ri = (row_w * 2 + side_w) * kG + g_w;          // this warp's Y region
    const int ri_partner = (row_w * 2 + (side_w ^ 1)) * kG + g_w;
    const int pair_bar = kBarPair + (f & 3);
    const uint32_t tx = tmem + ((32u * static_cast<uint32_t>(f & 3)) << 16) + kXCol;
    // lane twiddle anchors w_1024^{lane * 8 q}, q = 0..3, and the step w_1024^lane
    float2 anchor[4];
    float2 step;
    {
      float s, c;
      sincospif(2.0f * static_cast<float>(lane) / static_cast<float>(kC), &s, &c);
      step = make_float2(c, -s);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sincospif(2.0f * static_cast<float>((lane * 8 * q) & (kC - 1)) / static_cast<float>(kC), &s, &c);
        anchor[q] = make_float2(c, -s);
      }
    }
    float2 part[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) part[m] = make_float2(0.f, 0.f);
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      const int gcnt = min(kG, k_end - (k_begin + g * kG));
      named_sync(kBarYFull + b, kThreadsWs);
      // every front-end read of staging buffer b is done: refill it with
      // group g + 2 (the first FFT thread issues the copies)
      if (ftid == 0 && g + 2 < ngroups && !s_err) issue(g + 2);
      float2* work = ybuf + static_cast<size_t>(b) * kFftWarps * kRegion;
      float2* region = work + ri * kRegion;
      const float2* partner = work + ri_partner * kRegion;
      // ---- FFT of length 1024 --------------------------------------------
      float2 x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = region[lane + 32 * j];
      dft32<false>(x);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 w = anchor[q];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (q + r > 0) x[8 * q + r] = cmul(x[8 * q + r], w);
          w = cmul(w, step);
        }
      }
      __syncwarp();
#pragma unroll
      for (int ff = 0; ff < 32; ++ff) region[ff * kPitch + lane] = x[ff];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = region[lane * kPitch + j];
      dft32<false>(x);
      __syncwarp();
      // hand the partner the half of the bins it accumulates (side 0 keeps
      // bins 0..15 of every lane, side 1 bins 16..31): through tensor memory
      // (the quarter's swap buffer g mod 2: side s writes its 32 columns at
      // 32 s), or through shared memory
      const uint32_t xb = tx + 64u * static_cast<uint32_t>(b);
      if (!xsmem) {
        float gv[32];
        if (side_w == 0) {
#pragma unroll
          for (int m = 0; m < 16; ++m) { gv[2 * m] = x[16 + m].x; gv[2 * m + 1] = x[16 + m].y; }
          tmem_st32(xb, gv);
        } else {
#pragma unroll
          for (int m = 0; m < 16; ++m) { gv[2 * m] = x[m].x; gv[2 * m + 1] = x[m].y; }
          tmem_st32(xb + 32u, gv);
        }
        tmem_wait_st();
        tmem_fence_before_sync();
        named_sync(pair_bar, 64);
        tmem_fence_after_sync();
      } else {
        if (side_w == 0) {
#pragma unroll
          for (int m = 16; m < 32; ++m) region[lane + 32 * m] = x[m];
        } else {
#pragma unroll
          for (int m = 0; m < 16; ++m) region[lane + 32 * m] = x[m];
        }
        named_sync(pair_bar, 64);
      }
      // the partner's bins own_m0 + 8 h .. + 7 (its columns 16 h ..)
      auto partner8 = [&](int h, float2 (&q)[8]) {
        if (!xsmem) {
          uint32_t r[32];
          tmem_ld16_nowait(xb + 32u * static_cast<uint32_t>(side_w ^ 1) + 16u * static_cast<uint32_t>(h), r);
          tmem_wait_ld16(r);
#pragma unroll
          for (int i = 0; i < 8; ++i) q[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) q[i] = partner[lane + 32 * (own_m0 + 8 * h + i)];
        }
      };
      // ---- spectral products: own half of the bins ------------------------
      if (g_w < gcnt) {
        if (side_w == 0) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 q[8];
            partner8(h, q);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int m = 8 * h + i;
              part[m].x = fmaf(x[m].x, q[i].x, part[m].x);
              part[m].x = fmaf(-x[m].y, q[i].y, part[m].x);
              part[m].y = fmaf(x[m].x, q[i].y, part[m].y);
              part[m].y = fmaf(x[m].y, q[i].x, part[m].y);
            }
          }
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 q[8];
            partner8(h, q);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int m = 8 * h + i;
              part[m].x = fmaf(x[16 + m].x, q[i].x, part[m].x);
              part[m].x = fmaf(-x[16 + m].y, q[i].y, part[m].x);
              part[m].y = fmaf(x[16 + m].x, q[i].y, part[m].y);
              part[m].y = fmaf(x[16 + m].y, q[i].x, part[m].y);
            }
          }
        }
      }
      // ---- fold the partial sums into the Kahan accumulators ---------------
      if ((g % kFlush) == kFlush - 1 || g + 1 == ngroups) {
        named_sync(kBarFft, kFftThreads);   // every partner read of buffer b is done
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          region[lane + 32 * (own_m0 + m)] = part[m];
          part[m] = make_float2(0.f, 0.f);
        }
        named_sync(kBarFft, kFftThreads);
#pragma unroll
        for (int u = 0; u < (kRows * kC) / kFftThreads; ++u) {
          const int idx = ftid + kFftThreads * u;
          const int r = idx / kC, fb = idx % kC;
          const int sd = fb >> 9;            // bins f < 512 live with side a, the rest with side b
          float2 s = work[((r * 2 + sd) * kG + 0) * kRegion + fb];
#pragma unroll
          for (int gg = 1; gg < kG; ++gg) {
            const float2 v = work[((r * 2 + sd) * kG + gg) * kRegion + fb];
            s.x += v.x;
            s.y += v.y;
          }
          float4 a = acc[idx];
          kahan_add(a.x, a.z, s.x);
          kahan_add(a.y, a.w, s.y);
          acc[idx] = a;
        }
      }
      // release Y buffer b to the front end (only if it refills it)
      if (g + 2 < ngroups) named_arrive(kBarYFree + b, kThreadsWs);
    }
    // ---- this block's partial spectra ------------------------------------------
    named_sync(kBarFft, kFftThreads);
#pragma unroll
    for (int u = 0; u < (kRows * kC) / kFftThreads; ++u) {
      const int idx = ftid + kFftThreads * u;
      const int r = idx / kC, fb = idx % kC;
      if (r == 1 && !row1_live) continue;
      const float4 a = acc[idx];
      const uint32_t frow = r ? f1r[1] : f1r[0];
      float2* out = p.partial + ((static_cast<size_t>(t) * p.nrows + frow) * p.nkc + kc) * kC;
      out[fb] = make_float2(a.x - a.z, a.y - a.w);
    }
  }

  // ---- teardown ----------------------------------------------------------------
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (tid == 0 && s_err) {
    atomicOr(&g_ws_error, 1u);
    // copies still in flight must land before the block's shared memory is
    // released: one more bounded wait on the phases the issues left open
    for (int bb = 0; bb < 2; ++bb) {
      const int issued = ngroups > bb ? (ngroups - bb + 1) / 2 : 0;   // groups bb, bb + 2, ...
      if (issued > 0) (void)mbar_wait_bounded(&full_stage[bb], (issued - 1) & 1);
    }
  }
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) mbar_inval(&bars[i]);
  }
}

}  // namespace

uint32_t read_clear_error_sketch_ws() {
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_ws_error, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) cudaMemcpyToSymbol(g_ws_error, &zero, sizeof(zero));
  return v;
}

// The register split (setmaxnreg) must fit the registers the block is
// launched with, or the FFT warps' request would never be granted; checked
// once against the compiled kernel's launch register count.
bool ws_kernel_usable() {
  static std::atomic<int> ok{-1};   // concurrent first calls store the same value
  int v = ok.load(std::memory_order_relaxed);
  if (v < 0) {
    cudaFuncAttributes fa{};
    v = cudaFuncGetAttributes(&fa, k_sketch_ws) == cudaSuccess && fa.maxThreadsPerBlock >= kThreadsWs &&
                static_cast<int64_t>(fa.numRegs) * kThreadsWs >=
                    static_cast<int64_t>(kFeThreads) * kRegsFe + static_cast<int64_t>(kFftThreads) * kRegsFft
            ? 1
            : 0;
    ok.store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

size_t ws_smem_bytes(int npad, uint32_t ecap, int alias, int tw_shift, int nhi, int ovcap) {
  return ws_layout(npad, ecap, alias, tw_shift, nhi, ovcap).total;
}

cudaError_t launch_sketch_ws(const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                             const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3,
                             float2* partial, float2* thi, cudaStream_t s) {
  WsArgs a{};
  a.A = static_cast<const float*>(A);
  a.lda = lda;
  a.B = static_cast<const float*>(B);
  a.ldb = ldb;
  a.n1 = static_cast<int>(n1); a.n2 = static_cast<int>(n2); a.n3 = static_cast<int>(n3);
  a.n = static_cast<int>(h->n);
  a.npad = plan.npad;
  a.b = plan.b;
  a.nrows = plan.nrows;
  a.nunits = (plan.nrows + 1) / 2;
  a.kchunk = static_cast<int>(plan.kchunk);
  a.nkc = plan.nkc;
  a.alias = plan.alias ? 1 : 0;
  a.ecap = h->fe_ecap;
  a.tw_shift = plan.tw_shift;
  a.nhi = plan.nhi;
  a.rec_x = h->d_fe_x;
  a.rec_hs = h->d_fe_hs;
  a.grp = h->d_fe_grp;
  a.dest = h->d_fe_dest;
  a.ovf_off = h->d_fe_ovf_off;
  a.ovf_x = h->d_fe_ovf_x;
  a.ovf_hs = h->d_fe_ovf_hs;
  a.assign = h->d_fe_assign;
  a.partial = partial;
  a.thi_g = thi;
  a.ovcap = plan.ovcap;
  // debug switch (environment): the partner FFT warps swap their half
  // spectra through shared memory, the path blocks take when the front-end
  // records leave no tensor-memory columns for the swap
  a.force_xsmem = std::getenv("CMS_WS_SMEM_SWAP") != nullptr ? 1 : 0;
  if (!ws_kernel_usable()) return cudaErrorInvalidConfiguration;
  const int smem = static_cast<int>(plan.smem);
  cudaError_t e = cudaFuncSetAttribute(k_sketch_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned ntask = static_cast<unsigned>(static_cast<int64_t>(plan.d) * a.nunits * plan.nkc);
  {
    ProfScope prof_scope("k_sketch_ws", s);
    k_sketch_ws<<<ntask, kThreadsWs, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace cms
