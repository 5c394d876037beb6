// k_sketch_sparse.cu - COMPRESSEDPRODUCT for sparse inputs (Sec. 2.2, "A and
// B sparse ... nonzeros of a column (row) retrieved in linear time";
// Theorem 5's setting): A given by columns (CSC: colptr, rowidx, val), B by
// rows (CSR: rowptr, colidx, val).  Only inner indices k with a nonzero
// column a_k AND a nonzero row b_k contribute; they are compacted first, in
// increasing k, by a deterministic scan.
//
// The per-k work is the same four-step split as the dense kernels
// (b = R * 1024, a block owns one row f1 for one repetition and a range of
// nonempty k): the pruned first stage scatters the few nonzeros of a_k / b_k
// into Y[f1][z2] = sum s(x) v_x w_b^{f1 h(x)}, one warp per (side, k), in a
// fixed order (lanes with distinct buckets add in parallel, colliding lanes
// in lane order), then the radix-32 x radix-32 warp FFT, the spectral
// product (split across the two sides' warps) and Kahan-compensated
// accumulation, exactly as in k_sketch_fast.cu.
#include <algorithm>
#include <cstdlib>

#include "cms_internal.h"
#include "warp_fft.cuh"

namespace cms {
namespace {

using namespace wfft;

constexpr int kC = kFeC;       // 1024
constexpr int kG = 4;          // nonempty inner indices per group
constexpr int kThreads = 256;  // 8 warps = 2 sides x kG
constexpr int kFlush = 16;     // groups between Kahan folds (64 products)
constexpr int kPitch = 33;
constexpr int kRegion = 32 * kPitch;
constexpr int kSplitBlocks = 1024;   // chunks of the inner-index split

struct SparseArgs {
  const int64_t* ptr0;         // colptr of A (side 0)
  const int64_t* ptr1;         // rowptr of B (side 1)
  const int32_t* idx0;         // row indices of A
  const int32_t* idx1;         // column indices of B
  const void* val0;
  const void* val1;
  int nside0, nside1;          // n1, n3
  int n;
  int64_t b;
  int nrows;
  int nkc;                     // k-chunks per (repetition, row): fixed by the launch
  const int32_t* klist;
  const int32_t* kcount;       // device: length of klist (written by the split kernels)
  int skip_empty;              // 1: a block returns at once when the list is empty
  int sepy;                    // 1: scatter into per-warp Y buffers kept zero between groups
  const uint32_t* hs;
  int tw_shift, nhi;
  float2* partial;
};

template <typename T> __device__ __forceinline__ float ld_val(const void* p, int64_t e);
template <> __device__ __forceinline__ float ld_val<float>(const void* p, int64_t e) {
  return __ldg(static_cast<const float*>(p) + e);
}
template <> __device__ __forceinline__ float ld_val<double>(const void* p, int64_t e) {
  return static_cast<float>(__ldg(static_cast<const double*>(p) + e));
}
template <> __device__ __forceinline__ float ld_val<__nv_bfloat16>(const void* p, int64_t e) {
  return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[e]);
}

size_t sparse_smem_bytes(int tw_shift, int nhi, bool sepy) {
  return static_cast<size_t>(2 * kG) * kRegion * 8 + static_cast<size_t>(kC) * 16 +
         (static_cast<size_t>(1) << tw_shift) * 8 + static_cast<size_t>(nhi) * 8 +
         (sepy ? static_cast<size_t>(2 * kG) * kC * 8 : 0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_sketch_sparse(SparseArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  float2* work = reinterpret_cast<float2*>(sm);
  float4* acc = reinterpret_cast<float4*>(sm + static_cast<size_t>(2 * kG) * kRegion * 8);
  float2* tlo = reinterpret_cast<float2*>(acc + kC);
  float2* thi = tlo + (1 << p.tw_shift);
  // per warp: the scatter target Y (kept zero between groups: each lane
  // clears what it wrote once the FFT has read it)
  float2* ysc = thi + p.nhi;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int task = blockIdx.x;
  const int kc = task % p.nkc;
  const int row = (task / p.nkc) % p.nrows;
  const int t = task / (p.nkc * p.nrows);
  const uint32_t f1 = static_cast<uint32_t>(row);
  const int S = 1 << p.tw_shift;
  const ModB modb = make_modb(p.b);
  // the chunking follows the list length found on the device: nkc chunks of
  // a whole number of groups; trailing chunks may be empty (zero partials)
  const int K = *p.kcount;
  if (p.skip_empty && K == 0) return;
  const int kchunk = max(kG, ((K + p.nkc - 1) / p.nkc + kG - 1) / kG * kG);
  const int l_begin = min(K, kc * kchunk);
  const int l_end = min(K, l_begin + kchunk);

  for (int i = tid; i < S; i += kThreads) {
    float s, c;
    sincospif(2.0f * static_cast<float>(i) / static_cast<float>(p.b), &s, &c);
    tlo[i] = make_float2(c, -s);
  }
  for (int i = tid; i < p.nhi; i += kThreads) {
    const double a = 2.0 * static_cast<double>(static_cast<int64_t>(i) * S) / static_cast<double>(p.b);
    double s, c;
    sincospi(a, &s, &c);
    thi[i] = make_float2(static_cast<float>(c), static_cast<float>(-s));
  }
  for (int i = tid; i < kC; i += kThreads) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p.sepy)
    for (int i = tid; i < 2 * kG * kC; i += kThreads) ysc[i] = make_float2(0.f, 0.f);
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
  __syncthreads();

  const int side_w = warp / kG;
  const int g_w = warp % kG;
  float2* region = work + warp * kRegion;
  float2* ybuf = p.sepy ? ysc + warp * kC : region;
  const float2* partner = work + (warp ^ kG) * kRegion;   // same k slot, other side
  const uint32_t* tab = p.hs + (static_cast<size_t>(t) * 2 + side_w) * p.n;
  const int64_t* ptr = side_w ? p.ptr1 : p.ptr0;
  const int32_t* idx = side_w ? p.idx1 : p.idx0;
  const void* val = side_w ? p.val1 : p.val0;
  const int nside = side_w ? p.nside1 : p.nside0;

  float2 part[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) part[m] = make_float2(0.f, 0.f);
  // the only per-group exchange is between the two warps of a k slot (its
  // two sides): they meet at a 64-thread barrier of their own (1 + k slot)
  auto pair_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + g_w) : "memory"); };

  // one nonzero of the warp's (side, k): its bucket and contribution
  // s(x) v w_b^{f1 h(x)} (a lane without one gets a unique sentinel bucket)
  auto contribution = [&](bool valid, int32_t x, float v, uint32_t w, uint32_t& z2, float2& c) {
    z2 = 0x80000000u | static_cast<uint32_t>(lane);
    c = make_float2(0.f, 0.f);
    if (valid && x >= 0 && x < nside) {
      const uint32_t h = w & kBucketMask;
      float2 tw = wb(tlo, thi, mulmod(h, f1, modb), p.tw_shift);
      if (w >> 31) { tw.x = -tw.x; tw.y = -tw.y; }
      c = make_float2(v * tw.x, v * tw.y);
      z2 = h & (kC - 1);
    }
  };
  // added to Y[z2]: lanes with distinct buckets in parallel, lanes sharing
  // a bucket in lane order (round q takes each bucket's q-th lane, so the
  // rounds are as many as the largest multiplicity)
  auto scatter = [&](uint32_t z2, float2 contrib) {
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, z2);
    const uint32_t rank = __popc(same & ((1u << lane) - 1u));
    const uint32_t nrank = __reduce_max_sync(0xFFFFFFFFu, rank);
    for (uint32_t q = 0; q <= nrank; ++q) {
      if (rank == q && !(z2 >> 31)) {
        float2 y = ybuf[z2];
        y.x += contrib.x;
        y.y += contrib.y;
        ybuf[z2] = y;
      }
      __syncwarp();
    }
  };
  // The first 32 nonzeros of each group's (side, k) are fetched during the
  // two previous groups' FFTs, one dependent level per FFT stage (inner
  // index and column bounds two groups ahead, row index and value and hash
  // one group ahead), and their buckets and contributions formed at the end
  // of the previous group, so the scatter finds them in registers; further
  // nonzeros of a long column are loaded when scattered.
  int64_t pe0 = 0, pe1 = 0;     // this group's column bounds
  int64_t ne0 = 0, ne1 = 0;     // the next group's
  uint32_t pz2;
  float2 pc;
  {
    int32_t px = -1;
    float pv = 0.f;
    uint32_t pw = 0;
    if (l_begin + g_w < l_end) {
      const int k = p.klist[l_begin + g_w];
      pe0 = ptr[k];
      pe1 = ptr[k + 1];
      if (pe0 + lane < pe1) {
        px = idx[pe0 + lane];
        pv = ld_val<T>(val, pe0 + lane);
        if (px >= 0 && px < nside) pw = __ldg(tab + px);
      }
    }
    contribution(pe0 + lane < pe1, px, pv, pw, pz2, pc);
    if (l_begin + kG + g_w < l_end) {
      const int k1 = p.klist[l_begin + kG + g_w];
      ne0 = ptr[k1];
      ne1 = ptr[k1 + 1];
    }
  }

  int group = 0;
  for (int l0 = l_begin; l0 < l_end; l0 += kG, ++group) {
    const int gcnt = min(kG, l_end - l0);
    // ---- scatter the nonzeros of this warp's (side, k) into its zero Y ---
    // (without separate buffers the FFT region is zeroed first)
    if (!p.sepy) {
      pair_sync();   // the partner has read this region's published half
      float4* r4 = reinterpret_cast<float4*>(region);
#pragma unroll
      for (int i = 0; i < kC / 2 / 32; ++i) r4[lane + 32 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncwarp();
    }
    if (g_w < gcnt) {
      scatter(pz2, pc);
      for (int64_t base = pe0 + 32; base < pe1; base += 32) {
        const int64_t e = base + lane;
        const bool valid = e < pe1;
        int32_t x = -1;
        float v = 0.f;
        uint32_t w = 0;
        if (valid) {
          x = idx[e];
          v = ld_val<T>(val, e);
          if (x >= 0 && x < nside) w = __ldg(tab + x);
        }
        uint32_t z2;
        float2 c;
        contribution(valid, x, v, w, z2, c);
        scatter(z2, c);
      }
    }
    __syncwarp();
    // first prefetch level, two groups ahead: the inner index
    const int ln2 = l0 + 2 * kG + g_w;
    const int nk2 = ln2 < l_end ? p.klist[ln2] : -1;
    // ---- FFT of length 1024 ----------------------------------------------
    float2 x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = ybuf[lane + 32 * j];
    __syncwarp();
    // leave Y zero for the next group: each lane clears the bucket of its
    // nonzero (a column of more than 32 nonzeros clears the whole buffer)
    if (p.sepy && g_w < gcnt) {
      if (pe1 - pe0 > 32) {
        float4* y4 = reinterpret_cast<float4*>(ybuf);
#pragma unroll
        for (int i = 0; i < kC / 2 / 32; ++i) y4[lane + 32 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else if (!(pz2 >> 31)) {
        ybuf[pz2] = make_float2(0.f, 0.f);
      }
    }
    dft32<false>(x);
    // third level, next group: the lane's nonzero (row index and value)
    int32_t nx = -1;
    float nv = 0.f;
    if (ne0 + lane < ne1) {
      nx = idx[ne0 + lane];
      nv = ld_val<T>(val, ne0 + lane);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 w = anchor[q];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (q + r > 0) x[8 * q + r] = cmul(x[8 * q + r], w);
        w = cmul(w, step);
      }
    }
    if (p.sepy) pair_sync();   // the partner has read this region's published half
    else __syncwarp();
#pragma unroll
    for (int f = 0; f < 32; ++f) region[f * kPitch + lane] = x[f];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = region[lane * kPitch + j];
    // fourth level, next group: its hash
    const uint32_t nw = (nx >= 0 && nx < nside) ? __ldg(tab + nx) : 0u;
    // second level, two groups ahead: the column bounds
    int64_t qe0 = 0, qe1 = 0;
    if (nk2 >= 0) {
      qe0 = ptr[nk2];
      qe1 = ptr[nk2 + 1];
    }
    dft32<false>(x);
    __syncwarp();
    if (side_w == 0) {
#pragma unroll
      for (int m = 16; m < 32; ++m) region[lane + 32 * m] = x[m];
    } else {
#pragma unroll
      for (int m = 0; m < 16; ++m) region[lane + 32 * m] = x[m];
    }
    pair_sync();   // the partner's half is published
    if (g_w < gcnt) {
      if (side_w == 0) {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float2 q = partner[lane + 32 * m];
          part[m].x = fmaf(x[m].x, q.x, part[m].x);
          part[m].x = fmaf(-x[m].y, q.y, part[m].x);
          part[m].y = fmaf(x[m].x, q.y, part[m].y);
          part[m].y = fmaf(x[m].y, q.x, part[m].y);
        }
      } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float2 q = partner[lane + 32 * (16 + m)];
          part[m].x = fmaf(x[16 + m].x, q.x, part[m].x);
          part[m].x = fmaf(-x[16 + m].y, q.y, part[m].x);
          part[m].y = fmaf(x[16 + m].x, q.y, part[m].y);
          part[m].y = fmaf(x[16 + m].y, q.x, part[m].y);
        }
      }
    }
    pe0 = ne0;
    pe1 = ne1;
    contribution(pe0 + lane < pe1, nx, nv, nw, pz2, pc);
    ne0 = qe0;
    ne1 = qe1;
    const bool last = l0 + kG >= l_end;
    if ((group % kFlush) == kFlush - 1 || last) {
      __syncthreads();
      const int own = side_w * 16;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        region[lane + 32 * (own + m)] = part[m];
        part[m] = make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kC / kThreads; ++u) {
        const int f = tid + kThreads * u;
        const int sd = f >> 9;          // bins f < 512 live with side a
        float2 s = work[(sd * kG + 0) * kRegion + f];
#pragma unroll
        for (int g = 1; g < kG; ++g) {
          const float2 v = work[(sd * kG + g) * kRegion + f];
          s.x += v.x;
          s.y += v.y;
        }
        float4 a = acc[f];
        kahan_add(a.x, a.z, s.x);
        kahan_add(a.y, a.w, s.y);
        acc[f] = a;
      }
      __syncthreads();   // every region read before any warp writes its own again
    }
  }
  __syncthreads();
  float2* out = p.partial + ((static_cast<size_t>(t) * p.nrows + f1) * p.nkc + kc) * kC;
  for (int f = tid; f < kC; f += kThreads) {
    const float4 a = acc[f];
    out[f] = make_float2(a.x - a.z, a.y - a.w);
  }
}

// Sparse-k hybrid: the nonempty inner indices split, in increasing k, into
// those whose outer product a_k b_k has at most `limit` terms (sketched
// directly, Sec. 2.2 "sketching a matrix product naively") and the rest
// (the FFT route); limit < 0 sends every nonempty index to the FFT route.
// Three passes over contiguous chunks of k (one block each): counts per
// chunk, an exclusive scan of the chunk counts, and an ordered write of
// every chunk from its offsets.  counts[0] = FFT list length, counts[1] =
// direct list length.
__device__ __forceinline__ void classify_k(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr,
                                           int64_t n2, int64_t limit, int64_t k, bool* fft, bool* direct) {
  int64_t na = 0, nb = 0;
  if (k < n2) {
    na = a_ptr[k + 1] - a_ptr[k];
    nb = b_ptr[k + 1] - b_ptr[k];
  }
  const bool live = na > 0 && nb > 0;
  *direct = live && limit >= 0 && na * nb <= limit;
  *fft = live && !*direct;
}

__global__ void __launch_bounds__(1024)
k_split_count(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr, int64_t n2, int64_t limit,
              int64_t chunk, int32_t* __restrict__ part) {
  __shared__ int32_t tot[2];
  if (threadIdx.x < 2) tot[threadIdx.x] = 0;
  __syncthreads();
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t k1 = min(n2, k0 + chunk);
  int cf = 0, cd = 0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    bool f, dr;
    classify_k(a_ptr, b_ptr, n2, limit, k, &f, &dr);
    cf += f;
    cd += dr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    cf += __shfl_down_sync(0xFFFFFFFFu, cf, o);
    cd += __shfl_down_sync(0xFFFFFFFFu, cd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&tot[0], cf);
    atomicAdd(&tot[1], cd);
  }
  __syncthreads();
  if (threadIdx.x < 2) part[2 * blockIdx.x + threadIdx.x] = tot[threadIdx.x];
}

// exclusive scan of the nblk chunk counts (nblk <= 1024) in place
__global__ void __launch_bounds__(1024) k_split_scan(int32_t* __restrict__ part, int nblk,
                                                     int32_t* __restrict__ counts) {
  __shared__ int32_t wsum[2][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int side = 0; side < 2; ++side) {
    const int32_t v = tid < nblk ? part[2 * tid + side] : 0;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[side][warp] = x;
    __syncthreads();
    int32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) before += wsum[side][w];
      total += wsum[side][w];
    }
    if (tid < nblk) part[2 * tid + side] = before + x - v;
    if (tid == 0) counts[side] = total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
k_split_write(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr, int64_t n2, int64_t limit,
              int64_t chunk, const int32_t* __restrict__ part, int32_t* __restrict__ flist,
              int32_t* __restrict__ dlist) {
  __shared__ int32_t warp_tot[2][32];
  __shared__ int32_t running[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 2) running[tid] = part[2 * blockIdx.x + tid];
  __syncthreads();
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t k1 = min(n2, k0 + chunk);
  for (int64_t base = k0; base < k1; base += 1024) {
    const int64_t k = base + tid;
    bool f = false, dr = false;
    if (k < k1) classify_k(a_ptr, b_ptr, n2, limit, k, &f, &dr);
    const unsigned bf = __ballot_sync(0xFFFFFFFFu, f);
    const unsigned bd = __ballot_sync(0xFFFFFFFFu, dr);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) { warp_tot[0][warp] = __popc(bf); warp_tot[1][warp] = __popc(bd); }
    __syncthreads();
    int before_f = 0, before_d = 0;
    for (int w = 0; w < warp; ++w) { before_f += warp_tot[0][w]; before_d += warp_tot[1][w]; }
    if (f) flist[running[0] + before_f + __popc(bf & lt)] = static_cast<int32_t>(k);
    if (dr) dlist[running[1] + before_d + __popc(bd & lt)] = static_cast<int32_t>(k);
    __syncthreads();
    if (tid < 2) {
      int tot = 0;
      for (int w = 0; w < 32; ++w) tot += warp_tot[tid][w];
      running[tid] += tot;
    }
    __syncthreads();
  }
}

template <typename T> __device__ __forceinline__ double val_f64(const T* v, int64_t i);
template <> __device__ __forceinline__ double val_f64<float>(const float* v, int64_t i) { return v[i]; }
template <> __device__ __forceinline__ double val_f64<double>(const double* v, int64_t i) { return v[i]; }
template <> __device__ __forceinline__ double val_f64<__nv_bfloat16>(const __nv_bfloat16* v, int64_t i) {
  return static_cast<double>(__bfloat162float(v[i]));
}

// Direct sketch of the outer products of the listed inner indices: for every
// nonzero pair (A_ik, B_kj) and repetition t, s1(i) s2(j) A_ik B_kj goes to
// bucket (h1(i) + h2(j)) mod b of an FP64 accumulator (products of two FP32
// or BF16 values are exact in FP64; the additions are atomic, so their order
// varies, at FP64 rounding).  One block per listed k at a time.
template <typename T>
__global__ void __launch_bounds__(256)
k_direct_scatter(const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const T* __restrict__ a_val,
                 const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_idx, const T* __restrict__ b_val,
                 int n1, int n3, int64_t n, const int32_t* __restrict__ dlist, const int32_t* __restrict__ counts,
                 const uint32_t* __restrict__ hs, int d, int64_t b, double* __restrict__ cd) {
  const int Kd = counts[1];
  for (int q = blockIdx.x; q < Kd; q += gridDim.x) {
    const int64_t k = dlist[q];
    const int64_t a0 = a_ptr[k], na = a_ptr[k + 1] - a0;
    const int64_t b0 = b_ptr[k], nb = b_ptr[k + 1] - b0;
    for (int64_t pr = threadIdx.x; pr < na * nb; pr += blockDim.x) {
      const int64_t ia = a0 + pr / nb, jb = b0 + pr % nb;
      const int i = a_idx[ia], j = b_idx[jb];
      if (i < 0 || i >= n1 || j < 0 || j >= n3) continue;
      const double v = val_f64<T>(a_val, ia) * val_f64<T>(b_val, jb);
      for (int t = 0; t < d; ++t) {
        const uint32_t w1 = hs[(static_cast<size_t>(t) * 2 + 0) * n + i];
        const uint32_t w2 = hs[(static_cast<size_t>(t) * 2 + 1) * n + j];
        uint64_t z = static_cast<uint64_t>(w1 & kBucketMask) + (w2 & kBucketMask);
        if (z >= static_cast<uint64_t>(b)) z -= static_cast<uint64_t>(b);
        const double sv = ((w1 ^ w2) >> 31) ? -v : v;
        atomicAdd(&cd[static_cast<size_t>(t) * b + z], sv);
      }
    }
  }
}

// c = FFT-route c + direct part (rounded once to FP32), or the direct part
// alone when no inner index took the FFT route.
__global__ void k_add_direct(float* __restrict__ c, const double* __restrict__ cd, int64_t len,
                             const int32_t* __restrict__ counts) {
  const bool fft = counts[0] > 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < len;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    c[i] = static_cast<float>(fft ? static_cast<double>(c[i]) + cd[i] : cd[i]);
}

}  // namespace

int make_sparse_plan(const cms_hashes* h, int64_t n2, int64_t K, int num_sms, size_t smem_optin,
                     SketchPlan* plan, size_t* off_klist, std::string* why) {
  SketchPlan p;
  p.b = h->b;
  p.d = h->d;
  if (h->C != kFeC) {
    *why = "the sparse path needs b to be a multiple of 1024 (b = R * 1024)";
    return CMS_ERR_UNSUPPORTED;
  }
  p.R = h->R;
  p.C = h->C;
  p.nrows = static_cast<int>(p.R / 2 + 1);
  p.nradC = factor_radices(p.C, p.radC, 16);
  int sh = 0;
  while ((static_cast<int64_t>(1) << (2 * sh)) < p.b) ++sh;
  p.tw_shift = sh;
  p.nhi = static_cast<int>((p.b + (static_cast<int64_t>(1) << sh) - 1) >> sh);
  // separate, zero-kept scatter buffers when they fit beside the rest (a
  // debug switch in the environment keeps the in-place form, the path of
  // sketches too long for them)
  p.sparse_sepy = sparse_smem_bytes(p.tw_shift, p.nhi, true) <= smem_optin &&
                  std::getenv("CMS_SPARSE_INPLACE_Y") == nullptr;
  p.smem = sparse_smem_bytes(p.tw_shift, p.nhi, p.sparse_sepy);
  p.G = kG;
  p.threads = kThreads;
  const int64_t units = static_cast<int64_t>(p.d) * p.nrows;
  const int64_t slots = num_sms;
  const int64_t lo = std::max<int64_t>(1, (2 * slots + units - 1) / units);
  const int64_t hi = std::max<int64_t>(lo, 4 * lo);
  // chunks over the list of nonempty k; the workspace covers the largest count
  int64_t nkc;
  if (K < 0) {
    nkc = hi;
  } else {
    nkc = 1;
    double best = -1.0;
    const int64_t maxc = std::max<int64_t>(1, (K + kG - 1) / kG);
    for (int64_t c2 = std::min(lo, maxc); c2 <= std::min(hi, maxc); ++c2) {
      const int64_t tasks = units * c2;
      const int64_t waves = (tasks + slots - 1) / slots;
      const double eff = static_cast<double>(tasks) / static_cast<double>(waves * slots);
      if (eff > best + 1e-9) { best = eff; nkc = c2; }
    }
  }
  const int64_t KK = K < 0 ? n2 : K;
  int64_t kchunk = KK > 0 ? (KK + nkc - 1) / nkc : kG;
  kchunk = ((kchunk + kG - 1) / kG) * kG;
  if (K >= 0) nkc = KK > 0 ? (KK + kchunk - 1) / kchunk : 1;
  p.kchunk = kchunk;
  p.nkc = static_cast<int>(nkc);
  auto align256 = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  size_t off = 0;
  p.off_partial = off; off = align256(off + static_cast<size_t>(units) * hi * p.C * 8);
  p.off_V = off;       off = align256(off + static_cast<size_t>(units) * p.C * 8);
  p.off_twC = off;     off = align256(off + static_cast<size_t>(p.C) * 8);
  p.off_twR = off;     off = align256(off + static_cast<size_t>(p.R) * 8);
  *off_klist = off;    off = align256(off + static_cast<size_t>(std::max<int64_t>(n2, 1) + 1) * 4);
  // sparse-k hybrid: the direct list, the list counts, the FP64 direct sketch
  p.off_dlist = off;   off = align256(off + (static_cast<size_t>(std::max<int64_t>(n2, 1)) + 2 + 2 * kSplitBlocks) * 4);
  p.off_cd = off;      off = align256(off + static_cast<size_t>(p.d) * p.b * 8);
  p.ws_bytes = off;
  (void)why;
  *plan = p;
  return CMS_OK;
}

cudaError_t launch_nonempty_split(const int64_t* a_ptr, const int64_t* b_ptr, int64_t n2, int64_t limit,
                                  int32_t* flist, int32_t* dlist, int32_t* counts, int32_t* scratch, cudaStream_t s) {
  if (n2 <= 0) return cudaMemsetAsync(counts, 0, 2 * sizeof(int32_t), s);
  const int64_t nblk = std::min<int64_t>(kSplitBlocks, (n2 + 1023) / 1024);
  const int64_t chunk = ((n2 + nblk - 1) / nblk + 1023) / 1024 * 1024;
  const unsigned g = static_cast<unsigned>((n2 + chunk - 1) / chunk);
  ProfScope prof_scope("k_nonempty_split", s);
  k_split_count<<<g, 1024, 0, s>>>(a_ptr, b_ptr, n2, limit, chunk, scratch);
  k_split_scan<<<1, 1024, 0, s>>>(scratch, static_cast<int>(g), counts);
  k_split_write<<<g, 1024, 0, s>>>(a_ptr, b_ptr, n2, limit, chunk, scratch, flist, dlist);
  return cudaGetLastError();
}

cudaError_t launch_direct_scatter(const cms_hashes* h, const SparseArgsHost& in, int dt, const int32_t* dlist,
                                  const int32_t* counts, int64_t n2, double* cd, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cd, 0, static_cast<size_t>(h->d) * h->b * sizeof(double), s);
  if (e != cudaSuccess || n2 <= 0) return e;
  // the list length is on the device: blocks stride over it and those past
  // its end return at once
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(n2, 4096));
  ProfScope prof_scope("k_direct_scatter", s);
  switch (dt) {
    case CMS_F32:
      k_direct_scatter<float><<<grid, 256, 0, s>>>(in.a_ptr, in.a_idx, static_cast<const float*>(in.a_val), in.b_ptr,
                                                   in.b_idx, static_cast<const float*>(in.b_val), in.n1, in.n3, h->n,
                                                   dlist, counts, h->d_hs, h->d, h->b, cd);
      break;
    case CMS_BF16:
      k_direct_scatter<__nv_bfloat16><<<grid, 256, 0, s>>>(
          in.a_ptr, in.a_idx, static_cast<const __nv_bfloat16*>(in.a_val), in.b_ptr, in.b_idx,
          static_cast<const __nv_bfloat16*>(in.b_val), in.n1, in.n3, h->n, dlist, counts, h->d_hs, h->d, h->b, cd);
      break;
    default:
      k_direct_scatter<double><<<grid, 256, 0, s>>>(in.a_ptr, in.a_idx, static_cast<const double*>(in.a_val), in.b_ptr,
                                                    in.b_idx, static_cast<const double*>(in.b_val), in.n1, in.n3, h->n,
                                                    dlist, counts, h->d_hs, h->d, h->b, cd);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_add_direct(float* c, const double* cd, int64_t len, const int32_t* counts, cudaStream_t s) {
  {
    ProfScope prof_scope("k_add_direct", s);
    k_add_direct<<<static_cast<unsigned>(std::min<int64_t>((len + 255) / 256, 4096)), 256, 0, s>>>(c, cd, len, counts);
  }
  return cudaGetLastError();
}

cudaError_t launch_sketch_sparse(const SketchPlan& plan, const cms_hashes* h, const SparseArgsHost& in,
                                 int dt, const int32_t* klist, const int32_t* kcount, int skip_empty,
                                 float2* partial, cudaStream_t s) {
  SparseArgs a{};
  a.ptr0 = in.a_ptr; a.ptr1 = in.b_ptr;
  a.idx0 = in.a_idx; a.idx1 = in.b_idx;
  a.val0 = in.a_val; a.val1 = in.b_val;
  a.n = static_cast<int>(h->n);
  a.nside0 = in.n1; a.nside1 = in.n3;
  a.b = plan.b;
  a.nrows = plan.nrows;
  a.nkc = plan.nkc;
  a.klist = klist;
  a.kcount = kcount;
  a.skip_empty = skip_empty;
  a.sepy = plan.sparse_sepy ? 1 : 0;
  a.hs = h->d_hs;
  a.tw_shift = plan.tw_shift;
  a.nhi = plan.nhi;
  a.partial = partial;
  const int smem = static_cast<int>(plan.smem);
  const unsigned ntask = static_cast<unsigned>(static_cast<int64_t>(plan.d) * plan.nrows * plan.nkc);
  cudaError_t e = cudaSuccess;
  switch (dt) {
    case CMS_F32:
      e = cudaFuncSetAttribute(k_sketch_sparse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) { ProfScope ps("k_sketch_sparse", s); k_sketch_sparse<float><<<ntask, kThreads, smem, s>>>(a); }
      break;
    case CMS_BF16:
      e = cudaFuncSetAttribute(k_sketch_sparse<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) { ProfScope ps("k_sketch_sparse", s); k_sketch_sparse<__nv_bfloat16><<<ntask, kThreads, smem, s>>>(a); }
      break;
    default:
      e = cudaFuncSetAttribute(k_sketch_sparse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) { ProfScope ps("k_sketch_sparse", s); k_sketch_sparse<double><<<ntask, kThreads, smem, s>>>(a); }
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace cms
