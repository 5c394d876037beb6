// k_sketch_wide.cu - the fused sketch kernel for long sketches: b a multiple
// of C = 2^16, one row of the b = R x C grid per thread-block cluster of 8
// CTAs (the computation of k_sketch.cu, see there for the four-step split of
// the length-b DFT and the pruned first stage).
//
// With the row length C = 65536 the rows are few (R/2 + 1 of them: 9 for
// b = 2^20), so each entry of a_k and b_k is visited by few rows, but a row
// of C complex bins does not fit one SM.  It is split over the cluster:
// with bucket z2 = u + 8 v (u = CTA rank, v < 8192) and bin
// f2 = f2a + 8192 f2b (f2a < 8192, f2b < 8),
//   PA[f1 + R (f2a + 8192 f2b)] = sum_u w_8^{u f2b} [w_C^{u f2a} L_u[f2a]],
//   L_u[f2a] = sum_v w_8192^{v f2a} Y[f1][u + 8 v].
// CTA u gathers its buckets (an eighth of the entries, records with their
// twiddles s(x) w_b^{f1 h(x)} in tensor memory) and runs the local length-
// 8192 FFT in shared memory: with v = m + 1024 r and f2a = f8 + 8 q,
//   L[f8 + 8 q] = sum_m w_1024^{m q} [w_8192^{m f8} sum_r Y[m + 1024 r] w_8^{r f8}],
// a radix-8 pass over r and then one length-1024 register FFT per warp and
// block f8.  After a cluster barrier CTA v reads L_u[v + 8 q] of every CTA u
// through distributed shared memory, applies w_C^{u f2a}, finishes the
// length-8 DFT over u, forms PA PB and adds it to Kahan-compensated
// accumulators of its 8192 bins kept in tensor memory.  A second cluster
// barrier (arrive after the remote reads, wait before the next front end)
// guards the Y buffers.  The copy of the next a_k / b_k (TMA bulk copy into
// the staging buffer) runs while the FFTs of the current one do.
//
// Bucket records are dealt to threads by k_wide_tables: buckets in order of
// decreasing size, thread by thread in alternating directions, at most
// kCap entries per thread; buckets that do not fit go to a spill list that
// every inner index walks from global memory (twiddles computed on the fly).
#include <algorithm>
#include <atomic>

#include "cms_internal.h"
#include "sketch_generic.cuh"
#include "warp_fft.cuh"

namespace cms {
namespace {

using namespace wfft;

constexpr int kCl = 8;                 // CTAs per cluster
constexpr int kL = 8192;               // local FFT length
constexpr int kCw = kCl * kL;          // row length C = 65536
constexpr int kThr = 256;               // threads per CTA
constexpr int kWarps = kThr / 32;
constexpr int kQ = 1024 / kThr;         // bin groups q per thread (8 bins each)
constexpr int kKeys = 2 * kL;           // (side, v) bucket keys per CTA
constexpr int kStageBytes = 65536;      // staging row(s) of a_k, b_k
// tensor memory: warp w reaches lanes 32 (w mod 4) .. +31 and the column
// chunk w / 4 (kWarps / 4 chunks of kChunk columns); per thread: records
// x|v at [0, kCap), w.x at [kCap, 2 kCap), w.y at [2 kCap, 3 kCap), the
// accumulators of its kQ bin groups (32 columns each) at the chunk's end
constexpr int kChunk = 512 / (kWarps / 4);
constexpr int kAccCol = kChunk - 32 * kQ;
constexpr int kCap = kAccCol / 3;       // records per thread
static_assert(3 * kCap <= kAccCol, "record columns overlap the accumulators");

__device__ uint32_t g_wide_error = 0;   // 1: a wait gave up

struct WideArgs {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  int n1, n2, n3, n;
  int64_t b;
  int nrows, kchunk, nkc;
  int alias;
  int esz;                 // 2 (BF16) or 4 (FP32)
  int n1s;                 // staging offset of b_k (elements) when not aliased
  const uint32_t* rec_xv;  // [d][8][kCap][kThr]
  const uint32_t* rec_h;   // [d][8][kCap][kThr]
  const uint32_t* nrec;    // [d][8][kThr]
  const uint32_t* sp_xv;   // [d][8][spstride]
  const uint32_t* sp_h;
  const uint32_t* sp_bkt;  // [d][8][spstride]: bucket starts, then the end
  const uint32_t* sp_cnt;  // [d][8][2]: buckets, entries
  int64_t spstride;
  float2* partial;
};

struct WideLayout {
  size_t stage, Y, tw8k, twlo, twhi, total;
};

__host__ __device__ inline WideLayout wide_layout() {
  WideLayout L{};
  size_t o = 0;
  L.stage = o; o += kStageBytes;
  L.Y = o;     o += static_cast<size_t>(2) * kL * sizeof(float2);
  L.tw8k = o;  o += 1024 * sizeof(float2);
  L.twlo = o;  o += 128 * sizeof(float2);
  L.twhi = o;  o += 64 * sizeof(float2);
  L.total = o;
  return L;
}

// w_M^m = exp(-2 pi i m / M), angle reduced to (-pi, pi] in integers first.
__device__ __forceinline__ float2 wpow(uint64_t m, int64_t M) {
  const int64_t mm = 2 * static_cast<int64_t>(m) > M ? static_cast<int64_t>(m) - M : static_cast<int64_t>(m);
  float s, c;
  sincospif(2.0f * static_cast<float>(mm) / static_cast<float>(M), &s, &c);
  return make_float2(c, -s);
}

// ------------------------------------------------------ cluster helpers --
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of `local` (a shared-memory address of this CTA)
// in the CTA of rank `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// w^1 .. w^7 from w by a product tree of depth 3.
__device__ __forceinline__ void powers7(float2 w1, float2 (&w)[8]) {
  w[0] = make_float2(1.f, 0.f);
  w[1] = w1;
  w[2] = cmul(w1, w1);
  w[3] = cmul(w[2], w1);
  w[4] = cmul(w[2], w[2]);
  w[5] = cmul(w[4], w1);
  w[6] = cmul(w[3], w[3]);
  w[7] = cmul(w[4], w[3]);
}

template <typename T>
__device__ __forceinline__ float stage_val(const unsigned char* stage, uint32_t x) {
  return generic::to_f32(reinterpret_cast<const T*>(stage)[x]);
}

template <typename T>
__global__ void __launch_bounds__(kThr, 1) k_sketch_wide(WideArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  const WideLayout Ly = wide_layout();
  unsigned char* stage = sm + Ly.stage;
  float2* Y = reinterpret_cast<float2*>(sm + Ly.Y);          // [2 sides][8 blocks f8][1024]
  float2* tw8k = reinterpret_cast<float2*>(sm + Ly.tw8k);    // w_8192^m, m < 1024
  float2* twlo = reinterpret_cast<float2*>(sm + Ly.twlo);    // w_C^i, i < 128
  float2* twhi = reinterpret_cast<float2*>(sm + Ly.twhi);    // w_C^{128 i}, i < 64

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const int cid = blockIdx.x / kCl;
  const int kc = cid % p.nkc;
  const int f1 = (cid / p.nkc) % p.nrows;
  const int t = cid / (p.nkc * p.nrows);
  const int ts = t * kCl + static_cast<int>(rank);
  const int k_begin = kc * p.kchunk;
  const int k_end = min(p.n2, k_begin + p.kchunk);
  const ModB modb = make_modb(p.b);

  if (warp == 0) {
    tmem_alloc(&s_tmem, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    s_err = 0;
    mbar_init(&s_bar, 1);
    fence_proxy_async();
  }
  for (int i = tid; i < 1024; i += kThr) {
    float s, c;
    sincospif(2.0f * static_cast<float>(i) / static_cast<float>(kL), &s, &c);
    tw8k[i] = make_float2(c, -s);
  }
  if (tid < 128) {
    float s, c;
    sincospif(2.0f * static_cast<float>(tid) / static_cast<float>(kCw), &s, &c);
    twlo[tid] = make_float2(c, -s);
  }
  if (tid < 64) {
    float s, c;
    sincospif(2.0f * static_cast<float>(128 * tid) / static_cast<float>(kCw), &s, &c);
    twhi[tid] = make_float2(c, -s);
  }
  // lane anchors of the length-1024 FFT twiddles w_1024^{lane * 8 q}, q < 4,
  // and the step w_1024^lane
  float2 anchor[4], step;
  {
    float s, c;
    sincospif(2.0f * static_cast<float>(lane) / 1024.0f, &s, &c);
    step = make_float2(c, -s);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sincospif(2.0f * static_cast<float>((lane * 8 * q) % 1024) / 1024.0f, &s, &c);
      anchor[q] = make_float2(c, -s);
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = s_tmem;
  // this thread's row of tensor memory: lane quarter (warp mod 4), column half (warp / 4)
  const uint32_t trow = tmem + ((static_cast<uint32_t>(warp & 3) * 32u) << 16) + static_cast<uint32_t>(warp >> 2) * static_cast<uint32_t>(kChunk);

  // ---- records of this (t, u) for row f1: x|v|side|last and s(x) w_b^{f1 h(x)}
  const int nr = static_cast<int>(p.nrec[static_cast<size_t>(ts) * kThr + tid]);
  const int mr = __reduce_max_sync(0xffffffffu, nr);
  for (int j = 0; j < kCap; ++j) {
    uint32_t xv = 0;
    float2 w = make_float2(0.f, 0.f);
    if (j < nr) {
      const size_t q = (static_cast<size_t>(ts) * kCap + j) * kThr + tid;
      xv = p.rec_xv[q];
      const uint32_t hw = p.rec_h[q];
      w = wpow(mulmod(hw & kBucketMask, static_cast<uint32_t>(f1), modb), p.b);
      if (hw >> 31) { w.x = -w.x; w.y = -w.y; }
    }
    __syncwarp();   // the tensor-memory stores are warp-collective
    tmem_st1(trow + j, xv);
    tmem_st1(trow + kCap + j, __float_as_uint(w.x));
    tmem_st1(trow + 2 * kCap + j, __float_as_uint(w.y));
  }
  {
    float z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0.f;
#pragma unroll
    for (int g = 0; g < kQ; ++g) tmem_st32(trow + kAccCol + 32 * g, z);
  }
  tmem_wait_st();
  const int sp_nb = static_cast<int>(p.sp_cnt[static_cast<size_t>(ts) * 2]);
  const uint32_t* spx = p.sp_xv + static_cast<size_t>(ts) * p.spstride;
  const uint32_t* sph = p.sp_h + static_cast<size_t>(ts) * p.spstride;
  const uint32_t* spb = p.sp_bkt + static_cast<size_t>(ts) * p.spstride;

  // TMA copy of a_k (and b_k) into the staging buffer (thread 0)
  auto issue = [&](int k) {
    const uint32_t ba = static_cast<uint32_t>(p.n1) * static_cast<uint32_t>(p.esz);
    const uint32_t bb = p.alias ? 0u : static_cast<uint32_t>(p.n3) * static_cast<uint32_t>(p.esz);
    fence_proxy_async();
    mbar_arrive_expect_tx(&s_bar, ba + bb);
    const unsigned char* A = static_cast<const unsigned char*>(p.A);
    const unsigned char* B = static_cast<const unsigned char*>(p.B);
    if (ba) bulk_g2s(stage, A + static_cast<size_t>(k) * p.lda * p.esz, ba, &s_bar);
    if (bb) bulk_g2s(stage + static_cast<size_t>(p.n1s) * p.esz, B + static_cast<size_t>(k) * p.ldb * p.esz, bb, &s_bar);
  };
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (tid == 0 && k_begin < k_end) issue(k_begin);

  uint32_t phase = 0;
  bool timed_out = false;
  // remote addresses of block f8 = rank in every CTA's Y (side 0; side 1 is + 8192 float2)
  const uint32_t yblk = smem_u32(Y + 1024 * rank);
  for (int k = k_begin; k < k_end; ++k) {
    if (k > k_begin) cluster_wait();   // every CTA has read this CTA's Y of the previous k
    {
      float4* Y4 = reinterpret_cast<float4*>(Y);
      for (int i = tid; i < kL; i += kThr) Y4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!timed_out) {
      const bool ok = mbar_wait_bounded(&s_bar, phase);
      timed_out = __syncthreads_or(!ok);
      if (!timed_out) phase ^= 1u;   // else the copy of this phase may still land
    } else {
      __syncthreads();
    }
    // ---- gather front end: Y[side][v] = sum over the bucket's entries -----
    {
      // records in batches of 8, the next batch's tensor-memory loads in
      // flight while this one is gathered
      float2 acc = make_float2(0.f, 0.f);
      uint32_t rx[8], rwx[8], rwy[8];
      __syncwarp();   // warp-collective loads after the lanes' own stores
      if (mr > 0) {
        tmem_ld8_nowait(trow, rx);
        tmem_ld8_nowait(trow + kCap, rwx);
        tmem_ld8_nowait(trow + 2 * kCap, rwy);
      }
#pragma unroll 1
      for (int j0 = 0; j0 < mr; j0 += 8) {
        tmem_wait_ld8x3(rx, rwx, rwy);
        uint32_t cx[8];
        float cwx[8], cwy[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          cx[i] = rx[i];
          cwx[i] = __uint_as_float(rwx[i]);
          cwy[i] = __uint_as_float(rwy[i]);
        }
        __syncwarp();
        if (j0 + 8 < mr) {
          tmem_ld8_nowait(trow + j0 + 8, rx);
          tmem_ld8_nowait(trow + kCap + j0 + 8, rwx);
          tmem_ld8_nowait(trow + 2 * kCap + j0 + 8, rwy);
        }
        // the batch's staged values first (independent loads in flight),
        // then the sums; records past nr read index 0 and add nothing
        float val[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) val[i] = stage_val<T>(stage, j0 + i < nr ? (cx[i] & 0xFFFFu) : 0u);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (j0 + i < nr) {
            const uint32_t xv = cx[i];
            acc.x = fmaf(val[i], cwx[i], acc.x);
            acc.y = fmaf(val[i], cwy[i], acc.y);
            if (xv >> 31) {
              Y[((xv >> 29) & 1u) * kL + ((xv >> 16) & 0x1FFFu)] = acc;
              acc = make_float2(0.f, 0.f);
            }
          }
        }
        __syncwarp();
      }
      // buckets that did not fit the records: from global memory
      for (int sb = tid; sb < sp_nb; sb += kThr) {
        const uint32_t e0 = spb[sb], e1 = spb[sb + 1];
        float2 a = make_float2(0.f, 0.f);
        uint32_t xv = 0;
        for (uint32_t e = e0; e < e1; ++e) {
          xv = spx[e];
          const uint32_t hw = sph[e];
          float2 w = wpow(mulmod(hw & kBucketMask, static_cast<uint32_t>(f1), modb), p.b);
          if (hw >> 31) { w.x = -w.x; w.y = -w.y; }
          const float val = stage_val<T>(stage, xv & 0xFFFFu);
          a.x = fmaf(val, w.x, a.x);
          a.y = fmaf(val, w.y, a.y);
        }
        if (e1 > e0) Y[((xv >> 29) & 1u) * kL + ((xv >> 16) & 0x1FFFu)] = a;
      }
    }
    __syncthreads();
    // staging consumed: fetch the next inner index while the FFTs run
    if (tid == 0 && k + 1 < k_end && !timed_out) issue(k + 1);
    // ---- local FFT, radix-8 pass over r (v = m + 1024 r), both sides ------
#pragma unroll 2
    for (int m = tid; m < 1024; m += kThr) {
      float2 w[8];
      powers7(tw8k[m], w);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        float2* ys = Y + side * kL + m;
        float2 a[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r] = ys[1024 * r];
        Dft<8, false, float2>::run(a);
#pragma unroll
        for (int f8 = 1; f8 < 8; ++f8) a[f8] = cmul(a[f8], w[f8]);
#pragma unroll
        for (int f8 = 0; f8 < 8; ++f8) ys[1024 * f8] = a[f8];
      }
    }
    __syncthreads();
    // ---- length-1024 FFT over m per (side, f8) block ------------------------
    static_assert(kWarps == 8, "warp w runs the block pair of f8 = w");
    // lane l holds B[l + 32 j]: DFT-32 over j, twiddle w_1024^{l q1}, transpose
    // (XOR-swizzled in place), DFT-32 over l: lane q1 ends with bins q1 + 32 q2.
    // Warp w runs blocks w and w + 8 (the two sides of f8 = w) side by side,
    // two independent streams of arithmetic for the scheduler
    {
      float2* blk0 = Y + warp * 1024;
      float2* blk1 = Y + (warp + 8) * 1024;
      float2 x0[32], x1[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { x0[j] = blk0[lane + 32 * j]; x1[j] = blk1[lane + 32 * j]; }
      dft32<false>(x0);
      dft32<false>(x1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 w = anchor[q];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (q + r > 0) { x0[8 * q + r] = cmul(x0[8 * q + r], w); x1[8 * q + r] = cmul(x1[8 * q + r], w); }
          w = cmul(w, step);
        }
      }
      __syncwarp();
#pragma unroll
      for (int f = 0; f < 32; ++f) { blk0[f * 32 + (lane ^ f)] = x0[f]; blk1[f * 32 + (lane ^ f)] = x1[f]; }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j) { x0[j] = blk0[lane * 32 + (j ^ lane)]; x1[j] = blk1[lane * 32 + (j ^ lane)]; }
      dft32<false>(x0);
      dft32<false>(x1);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j) { blk0[lane + 32 * j] = x0[j]; blk1[lane + 32 * j] = x1[j]; }
    }
    // ---- every CTA's L_u ready: length-8 DFT over u, products, Kahan -------
    cluster_arrive();
    cluster_wait();
    {
      // all remote loads first (16 kQ in flight per thread), then the arithmetic
      float2 ga[kQ][8], gb[kQ][8];
#pragma unroll
      for (int qi = 0; qi < kQ; ++qi) {
        const uint32_t la = yblk + static_cast<uint32_t>(tid + kThr * qi) * 8u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t ra = map_rank(la, static_cast<uint32_t>(u));
          ga[qi][u] = ld_cluster(ra);
          gb[qi][u] = ld_cluster(ra + static_cast<uint32_t>(kL) * 8u);
        }
      }
#pragma unroll
      for (int qi = 0; qi < kQ; ++qi) {
        const int f2a = static_cast<int>(rank) + 8 * (tid + kThr * qi);
        float2 w[8];
        powers7(cmul(twhi[f2a >> 7], twlo[f2a & 127]), w);
#pragma unroll
        for (int u = 1; u < 8; ++u) {
          ga[qi][u] = cmul(ga[qi][u], w[u]);
          gb[qi][u] = cmul(gb[qi][u], w[u]);
        }
        Dft<8, false, float2>::run(ga[qi]);
        Dft<8, false, float2>::run(gb[qi]);
        float a[32];
        tmem_ld32(trow + kAccCol + 32 * qi, a);
#pragma unroll
        for (int f2b = 0; f2b < 8; ++f2b) {
          const float2 pr = cmul(ga[qi][f2b], gb[qi][f2b]);
          kahan_add(a[4 * f2b + 0], a[4 * f2b + 2], pr.x);
          kahan_add(a[4 * f2b + 1], a[4 * f2b + 3], pr.y);
        }
        tmem_st32(trow + kAccCol + 32 * qi, a);
      }
    }
    tmem_wait_st();
    // the remote values are consumed (their loads complete): a relaxed
    // arrival suffices to order them before the other CTAs' next front end
    cluster_arrive_relaxed();
  }
  if (k_end > k_begin) cluster_wait();

  // ---- partial row: bins f2 = rank + 8 q + 8192 f2b ------------------------
  {
    float2* out = p.partial + ((static_cast<size_t>(t) * p.nrows + f1) * p.nkc + kc) * kCw;
#pragma unroll 1
    for (int qi = 0; qi < kQ; ++qi) {
      const int q = tid + kThr * qi;
      float a[32];
      tmem_ld32(trow + kAccCol + 32 * qi, a);
#pragma unroll
      for (int f2b = 0; f2b < 8; ++f2b)
        out[static_cast<int>(rank) + 8 * q + kL * f2b] =
            make_float2(a[4 * f2b + 0] - a[4 * f2b + 2], a[4 * f2b + 1] - a[4 * f2b + 3]);
    }
  }

  // ---- teardown ----------------------------------------------------------------
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (tid == 0 && timed_out) {
    atomicOr(&g_wide_error, 1u);
    // a copy still in flight must land before the shared memory is released
    (void)mbar_wait_bounded(&s_bar, phase);
  }
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (tid == 0) mbar_inval(&s_bar);
}

// ------------------------------------------------------------ tables ----
// One block per (t, u): the entries x of either side whose bucket h(x) has
// (h mod C) mod 8 = u, grouped by key (side, v = (h mod C) / 8) in x order,
// buckets dealt to the 256 threads in order of decreasing size (ties by key),
// alternating direction every round, each thread taking whole buckets while
// it has room for kCap records.
struct TabArgs {
  const uint32_t* hs;    // [d][2][n]
  int n, n1, n3, alias, n1s;
  uint32_t* ent;         // [d][8][entstride] scratch: x per sorted entry
  int64_t entstride;
  uint32_t* rec_xv;
  uint32_t* rec_h;
  uint32_t* nrec;
  uint32_t* sp_xv;
  uint32_t* sp_h;
  uint32_t* sp_bkt;
  uint32_t* sp_cnt;
  int64_t spstride;
};

constexpr int kTabThr = kThr;   // one table column per sketch-kernel thread

// exclusive scan over the block of one value per thread; returns the prefix
// and writes the total to *total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kTabThr / 32 ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kTabThr / 32) scratch[32 + lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp > 0 ? scratch[32 + warp - 1] : 0u;
  *total = scratch[32 + kTabThr / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kTabThr) k_wide_tables(TabArgs p) {
  extern __shared__ uint32_t tsm[];
  uint32_t* cnt = tsm;               // [kKeys] entries per key
  uint32_t* off = cnt + kKeys;       // [kKeys] first sorted entry of the key
  uint32_t* run = off + kKeys;       // [kKeys] fill counter, later the key at each dealing position
  __shared__ uint32_t scratch[64];
  __shared__ uint32_t s_maxc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ts = blockIdx.x;
  const int t = ts / kCl, u = ts % kCl;
  uint32_t* ent = p.ent + static_cast<size_t>(ts) * p.entstride;

  for (int i = tid; i < kKeys; i += kTabThr) { cnt[i] = 0; run[i] = 0; }
  if (tid == 0) s_maxc = 0;
  __syncthreads();
  for (int side = 0; side < 2; ++side) {
    const int ns = side ? p.n3 : p.n1;
    const uint32_t* tab = p.hs + (static_cast<size_t>(t) * 2 + side) * p.n;
    for (int x = tid; x < ns; x += kTabThr) {
      const uint32_t h = tab[x] & kBucketMask;
      if (static_cast<int>(h & 7u) == u) atomicAdd(&cnt[side * kL + ((h & 0xFFFFu) >> 3)], 1u);
    }
  }
  __syncthreads();
  // exclusive scan of the counts: keys [64 tid, 64 tid + 64)
  constexpr int kPer = kKeys / kTabThr;
  uint32_t loc = 0, cmax = 0;
  for (int i = 0; i < kPer; ++i) {
    const uint32_t c = cnt[tid * kPer + i];
    loc += c;
    cmax = max(cmax, c);
  }
  uint32_t total;
  uint32_t base = block_excl_scan(loc, scratch, &total);
  for (int i = 0; i < kPer; ++i) {
    off[tid * kPer + i] = base;
    base += cnt[tid * kPer + i];
  }
  atomicMax(&s_maxc, cmax);
  __syncthreads();
  // stable placement in x order: warp `side` walks that side's x in chunks of 32
  if (warp < 2) {
    const int side = warp;
    const int ns = side ? p.n3 : p.n1;
    const uint32_t* tab = p.hs + (static_cast<size_t>(t) * 2 + side) * p.n;
    const uint32_t lt = (1u << lane) - 1u;
    for (int x0 = 0; x0 < ns; x0 += 32) {
      const int x = x0 + lane;
      uint32_t key = 0xFFFFFFFFu;
      if (x < ns) {
        const uint32_t h = tab[x] & kBucketMask;
        if (static_cast<int>(h & 7u) == u) key = static_cast<uint32_t>(side * kL) + ((h & 0xFFFFu) >> 3);
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, key);
      uint32_t r0 = 0;
      if (key != 0xFFFFFFFFu) {
        r0 = run[key];
        ent[off[key] + r0 + __popc(peers & lt)] = static_cast<uint32_t>(x);
      }
      __syncwarp();
      if (key != 0xFFFFFFFFu && __popc(peers & lt) == __popc(peers) - 1) run[key] = r0 + __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();
  // dealing positions: sizes from the largest down, keys ascending
  const uint32_t maxc = s_maxc;
  uint32_t pbase = 0;
  for (uint32_t c = maxc; c >= 1; --c) {
    uint32_t lc = 0;
    for (int i = 0; i < kPer; ++i) lc += cnt[tid * kPer + i] == c;
    uint32_t tot;
    uint32_t pos = pbase + block_excl_scan(lc, scratch, &tot);
    for (int i = 0; i < kPer; ++i)
      if (cnt[tid * kPer + i] == c) run[pos++] = static_cast<uint32_t>(tid * kPer + i);
    pbase += tot;
  }
  const uint32_t nb = pbase;   // nonempty buckets
  __syncthreads();
  // placement: thread T takes position r * kThr + T (even rounds) or
  // r * kThr + kThr - 1 - T (odd rounds)
  {
    uint32_t fill = 0;
    for (uint32_t r = 0; r * kTabThr < nb; ++r) {
      const uint32_t pp = r * kTabThr + ((r & 1u) ? static_cast<uint32_t>(kTabThr - 1 - tid) : static_cast<uint32_t>(tid));
      if (pp >= nb) continue;
      const uint32_t key = run[pp];
      const uint32_t c = cnt[key];
      if (fill + c <= static_cast<uint32_t>(kCap)) {
        const uint32_t side = key >= static_cast<uint32_t>(kL) ? 1u : 0u;
        const uint32_t v = key & static_cast<uint32_t>(kL - 1);
        const uint32_t* tab = p.hs + (static_cast<size_t>(t) * 2 + side) * p.n;
        for (uint32_t i = 0; i < c; ++i) {
          const uint32_t x = ent[off[key] + i];
          const uint32_t xs = (side && !p.alias) ? x + static_cast<uint32_t>(p.n1s) : x;
          const uint32_t xv = xs | (v << 16) | (side << 29) | (i + 1 == c ? 0x80000000u : 0u);
          const size_t q = (static_cast<size_t>(ts) * kCap + fill + i) * kTabThr + tid;
          p.rec_xv[q] = xv;
          p.rec_h[q] = tab[x];
        }
        fill += c;
      } else {
        run[pp] = key | 0x80000000u;   // spilled
      }
    }
    p.nrec[static_cast<size_t>(ts) * kTabThr + tid] = fill;
  }
  __syncthreads();
  // spill list, in dealing order (warp 0)
  if (warp == 0) {
    uint32_t* sx = p.sp_xv + static_cast<size_t>(ts) * p.spstride;
    uint32_t* sh = p.sp_h + static_cast<size_t>(ts) * p.spstride;
    uint32_t* sbk = p.sp_bkt + static_cast<size_t>(ts) * p.spstride;
    uint32_t nent = 0, nbk = 0;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t pb = 0; pb < nb; pb += 32) {
      const uint32_t pp = pb + lane;
      const bool spl = pp < nb && (run[pp] >> 31);
      const uint32_t bal = __ballot_sync(0xffffffffu, spl);
      if (bal == 0) continue;
      const uint32_t key = spl ? (run[pp] & 0x7FFFFFFFu) : 0u;
      const uint32_t c = spl ? cnt[key] : 0u;
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
      if (spl) {
        const uint32_t e0 = nent + x - c;
        sbk[nbk + __popc(bal & lt)] = e0;
        const uint32_t side = key >= static_cast<uint32_t>(kL) ? 1u : 0u;
        const uint32_t v = key & static_cast<uint32_t>(kL - 1);
        const uint32_t* tab = p.hs + (static_cast<size_t>(t) * 2 + side) * p.n;
        for (uint32_t i = 0; i < c; ++i) {
          const uint32_t xe = ent[off[key] + i];
          const uint32_t xs = (side && !p.alias) ? xe + static_cast<uint32_t>(p.n1s) : xe;
          sx[e0 + i] = xs | (v << 16) | (side << 29) | (i + 1 == c ? 0x80000000u : 0u);
          sh[e0 + i] = tab[xe];
        }
      }
      nent += tot;
      nbk += __popc(bal);
    }
    if (lane == 0) {
      sbk[nbk] = nent;
      p.sp_cnt[static_cast<size_t>(ts) * 2] = nbk;
      p.sp_cnt[static_cast<size_t>(ts) * 2 + 1] = nent;
    }
  }
}

// ------------------------------------------------------------ inverse ----
// Row inverse for C = 65536 = 256 x 256 (f2 = a + 256 e2, z2 = c + 256 e):
//   x[c + 256 e] = sum_a w_256^{-a e} [w_C^{-a c} sum_e2 S[a + 256 e2] w_256^{-e2 c}],
// then V[f1][z2] = x[z2] w_b^{-f1 z2}.  Pass A (one block per row and a)
// sums the k-range partials in FP64 and runs the inner transforms; pass B
// (one block per row and c) the outer ones.
struct WinvArgs {
  int64_t b;
  int nrows, nkc;
  int nrad;
  int rad[8];
  const float2* partial;   // [units][nkc][C]
  const float2* tw256;     // w_256^m
  float2* T;               // [units][256 a][256 c]
  float2* V;               // [units][C]
};

__global__ void __launch_bounds__(256) k_winv_a(WinvArgs p) {
  __shared__ float2 P[256], Q[256], tw[256];
  const int a = blockIdx.x & 255;
  const int unit = blockIdx.x >> 8;
  tw[threadIdx.x] = p.tw256[threadIdx.x];
  const float2* part = p.partial + static_cast<size_t>(unit) * p.nkc * kCw;
  {
    const int e2 = threadIdx.x;
    double sx = 0.0, sy = 0.0;
    for (int kc = 0; kc < p.nkc; ++kc) {
      const float2 v = part[static_cast<size_t>(kc) * kCw + a + 256 * e2];
      sx += v.x;
      sy += v.y;
    }
    P[e2] = make_float2(static_cast<float>(sx), static_cast<float>(sy));
  }
  __syncthreads();
  const float2* X = fft_block<true>(P, Q, 256, 1, p.rad, p.nrad, tw);
  const int c = threadIdx.x;
  const float2 w = cconj(wpow(static_cast<uint64_t>(a) * static_cast<uint64_t>(c), kCw));
  p.T[(static_cast<size_t>(unit) * 256 + a) * 256 + c] = cmul(X[c], w);
}

__global__ void __launch_bounds__(256) k_winv_b(WinvArgs p) {
  __shared__ float2 P[256], Q[256], tw[256];
  const int c = blockIdx.x & 255;
  const int unit = blockIdx.x >> 8;
  const int f1 = unit % p.nrows;
  tw[threadIdx.x] = p.tw256[threadIdx.x];
  P[threadIdx.x] = p.T[(static_cast<size_t>(unit) * 256 + threadIdx.x) * 256 + c];
  __syncthreads();
  const float2* X = fft_block<true>(P, Q, 256, 1, p.rad, p.nrad, tw);
  const int e = threadIdx.x;
  const uint32_t z2 = static_cast<uint32_t>(c + 256 * e);
  const uint64_t m = (static_cast<uint64_t>(f1) * z2) % static_cast<uint64_t>(p.b);
  p.V[static_cast<size_t>(unit) * kCw + z2] = cmul(X[e], cconj(wpow(m, p.b)));
}

}  // namespace

// ------------------------------------------------------------ host side ----
size_t wide_smem_bytes() { return wide_layout().total; }

uint32_t read_clear_error_sketch_wide() {
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_wide_error, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) cudaMemcpyToSymbol(g_wide_error, &zero, sizeof(zero));
  return v;
}

WideTables wide_tables_layout(int d, int64_t n, size_t base) {
  WideTables w{};
  const size_t units = static_cast<size_t>(d) * kCl;
  size_t o = base;
  auto take = [&](size_t bytes) { const size_t r = o; o = (o + bytes + 255) & ~static_cast<size_t>(255); return r; };
  w.entstride = 2 * n;
  w.spstride = 2 * n + 1;
  w.off_ent = take(units * w.entstride * 4);
  w.off_rec_xv = take(units * kCap * kThr * 4);
  w.off_rec_h = take(units * kCap * kThr * 4);
  w.off_nrec = take(units * kThr * 4);
  w.off_sp_xv = take(units * w.spstride * 4);
  w.off_sp_h = take(units * w.spstride * 4);
  w.off_sp_bkt = take(units * w.spstride * 4);
  w.off_sp_cnt = take(units * 2 * 4);
  w.end = o;
  return w;
}

// Active clusters of the kernel's launch shape (0: it cannot run here).
int wide_max_clusters(int dt) {
  static std::atomic<int> cached[2] = {{-1}, {-1}};   // concurrent first calls store the same value
  const int i = dt == CMS_BF16 ? 1 : 0;
  const int c = cached[i].load(std::memory_order_relaxed);
  if (c >= 0) return c;
  const void* fn = i ? reinterpret_cast<const void*>(k_sketch_wide<__nv_bfloat16>)
                     : reinterpret_cast<const void*>(k_sketch_wide<float>);
  const int smem = static_cast<int>(wide_smem_bytes());
  int nc = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kCl, 1, 1);
    cfg.blockDim = dim3(kThr, 1, 1);
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kCl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
  }
  (void)cudaGetLastError();
  cached[i].store(nc, std::memory_order_relaxed);
  return nc;
}

cudaError_t launch_sketch_wide(const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                               const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3, char* ws,
                               float2* partial, cudaStream_t s) {
  const WideTables wt = wide_tables_layout(plan.d, h->n, plan.off_wtab);
  const int esz = plan.dt == CMS_BF16 ? 2 : 4;
  const int n1s = plan.alias ? 0 : static_cast<int>((n1 * esz + 15) / 16 * 16 / esz);
  TabArgs ta{};
  ta.hs = h->d_hs;
  ta.n = static_cast<int>(h->n);
  ta.n1 = static_cast<int>(n1);
  ta.n3 = static_cast<int>(n3);
  ta.alias = plan.alias ? 1 : 0;
  ta.n1s = n1s;
  ta.ent = reinterpret_cast<uint32_t*>(ws + wt.off_ent);
  ta.entstride = wt.entstride;
  ta.rec_xv = reinterpret_cast<uint32_t*>(ws + wt.off_rec_xv);
  ta.rec_h = reinterpret_cast<uint32_t*>(ws + wt.off_rec_h);
  ta.nrec = reinterpret_cast<uint32_t*>(ws + wt.off_nrec);
  ta.sp_xv = reinterpret_cast<uint32_t*>(ws + wt.off_sp_xv);
  ta.sp_h = reinterpret_cast<uint32_t*>(ws + wt.off_sp_h);
  ta.sp_bkt = reinterpret_cast<uint32_t*>(ws + wt.off_sp_bkt);
  ta.sp_cnt = reinterpret_cast<uint32_t*>(ws + wt.off_sp_cnt);
  ta.spstride = wt.spstride;
  const int tsmem = 3 * kKeys * 4;
  cudaError_t e = cudaFuncSetAttribute(k_wide_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof_scope("k_wide_tables", s);
    k_wide_tables<<<static_cast<unsigned>(plan.d * kCl), kTabThr, tsmem, s>>>(ta);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  WideArgs a{};
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
  a.n1 = static_cast<int>(n1); a.n2 = static_cast<int>(n2); a.n3 = static_cast<int>(n3);
  a.n = static_cast<int>(h->n);
  a.b = plan.b;
  a.nrows = plan.nrows;
  a.kchunk = static_cast<int>(plan.kchunk);
  a.nkc = plan.nkc;
  a.alias = plan.alias ? 1 : 0;
  a.esz = esz;
  a.n1s = n1s;
  a.rec_xv = ta.rec_xv; a.rec_h = ta.rec_h; a.nrec = ta.nrec;
  a.sp_xv = ta.sp_xv; a.sp_h = ta.sp_h; a.sp_bkt = ta.sp_bkt; a.sp_cnt = ta.sp_cnt;
  a.spstride = wt.spstride;
  a.partial = partial;
  const bool bf = plan.dt == CMS_BF16;
  const void* fn = bf ? reinterpret_cast<const void*>(k_sketch_wide<__nv_bfloat16>)
                      : reinterpret_cast<const void*>(k_sketch_wide<float>);
  const int smem = static_cast<int>(wide_smem_bytes());
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(static_cast<int64_t>(plan.d) * plan.nrows * plan.nkc * kCl), 1, 1);
  cfg.blockDim = dim3(kThr, 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    ProfScope prof_scope("k_sketch_wide", s);
    e = bf ? cudaLaunchKernelEx(&cfg, k_sketch_wide<__nv_bfloat16>, a) : cudaLaunchKernelEx(&cfg, k_sketch_wide<float>, a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_inverse_wide(const SketchPlan& plan, const float2* partial, float2* V, float2* T,
                                const float2* tw256, const float2* twR, float* c, cudaStream_t s) {
  WinvArgs w{};
  w.b = plan.b;
  w.nrows = plan.nrows;
  w.nkc = plan.nkc;
  w.nrad = factor_radices(256, w.rad, 8);
  w.partial = partial;
  w.tw256 = tw256;
  w.T = T;
  w.V = V;
  const unsigned blocks = static_cast<unsigned>(static_cast<int64_t>(plan.d) * plan.nrows * 256);
  {
    ProfScope prof_scope("k_winv_a", s);
    k_winv_a<<<blocks, 256, 0, s>>>(w);
  }
  {
    ProfScope prof_scope("k_winv_b", s);
    k_winv_b<<<blocks, 256, 0, s>>>(w);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_cols_inverse(plan, V, twR, c, s);
}

}  // namespace cms
