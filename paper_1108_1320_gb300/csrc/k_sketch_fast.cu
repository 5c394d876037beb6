// k_sketch_fast.cu - the fused FP32 kernel for C = 1024 (b = R * 1024),
// the same computation as k_sketch_fused in k_sketch.cu (see there for the
// four-step split of the length-b DFT and the pruned first stage) with a
// GB300-specific layout:
//
//  * a thread block owns TWO rows f1 of the R x C output grid (one
//    repetition t, a range of inner indices k), so every value of a_k / b_k
//    it gathers serves both rows;
//  * a_k (column k of A) and b_k (row k of B) for a group of G = 2 inner
//    indices are staged into shared memory by TMA bulk copies
//    (cp.async.bulk + mbarrier), issued as soon as the previous group's
//    front end has consumed the buffer, so the copy overlaps the FFTs;
//    when A = X^T and B = X are the same bytes the rows are staged once;
//  * the gather front end Y[f1][z2] = sum s(x) A_xk w_b^{f1 h(x)} walks
//    records (staging index of x and the two rows' twiddles) kept in shared
//    memory for the whole task, laid out as one contiguous stream per warp;
//    32 buckets of equal (capped) occupancy form a group whose lanes run in
//    lock step, placed so that the stores to Y are free of bank conflicts;
//  * each of the 8 warps runs one length-1024 FFT (one (row, side, k)):
//    radix-32 in registers, twiddle, one XOR-swizzled (conflict-free)
//    transpose through shared memory, radix-32 in registers; lane l ends
//    holding bins l + 32 m, m = 0..31;
//  * the side-b warps publish their spectra, the side-a warps multiply and
//    accumulate PA PB in registers; every kFlush groups the two inner
//    indices' partial sums are added (fixed order) and folded into
//    Kahan-compensated accumulators in shared memory.
#include <algorithm>
#include <cstring>

#include "cms_internal.h"
#include "warp_fft.cuh"
#include "sketch_generic.cuh"
#include "dft_codelets.cuh"

namespace cms {
namespace {

using namespace wfft;

constexpr int kC = kFeC;       // 1024: the largest C = P Q
constexpr int kG = 2;          // inner indices per group
constexpr int kRows = 2;       // rows f1 per block
constexpr int kThreads = 256;  // 8 warps = kRows x 2 sides x kG FFTs
constexpr int kFlush = 32;     // groups between Kahan folds (64 products)
constexpr int kPitch = 33;     // transpose row pitch (float2): conflict-free both ways
constexpr int kRegion = 32 * kPitch;   // float2 per warp region (>= kC)

__device__ uint32_t g_sketch_error = 0;   // 1: a TMA wait gave up

struct FastArgs {
  const void* A;      // FP32 or BF16 storage (the task body's template type)
  int64_t lda;
  const void* B;
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
  const uint32_t* ovf_off;   // [t][side][C + 1]: each bucket's overflow list
  const uint32_t* ovf_x;     // [t][side][n]: overflow entries (x), bucket by bucket
  const uint32_t* ovf_hs;    // [t][side][n]: their packed hashes
  float2* partial;
  int C, P, Q;        // FFT length C = P Q: P lanes x DFT-Q, then Q lanes x DFT-P
  int G;              // bucket groups per side, ceil(C / 32)
  int esz;            // bytes per stored element: 4 (FP32) or 2 (BF16)
  int unal;           // rows not 16-byte aligned: copy the aligned superset
  int zpos;           // (unal) staging index of the zero slot read by padding
  int tmem_rec;       // twiddle records in tensor memory (large n) instead of shared memory
};

}  // namespace

struct BatchDesc {
  int kind;                 // 1: fast task (FP32), 3: fast task (BF16), 0: generic task
  generic::SketchArgs g;
  FastArgs f;
};

namespace {

struct SmemLayout {
  size_t stage, rec_tw, rec_x, work, acc, tlo, thi, wmeta, wdst, wovb, ibase, istart, slot_src, bar, total;
};

constexpr int kWarps = kThreads / 32;
constexpr int kItems = 2 * (kC / 32) / kWarps;   // (side, bucket group) item slots per warp: 8
constexpr uint32_t kVoidItem = 1u << 30;          // wmeta flag: slot without an item (2 L < 64)

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

__host__ __device__ inline SmemLayout fast_layout(int npad, uint32_t ecap, int alias, int tw_shift, int nhi,
                                                  int esz, int tmem_rec) {
  SmemLayout L{};
  size_t o = 0;
  const int nstage = alias ? 1 : 2;
  L.stage = o;    o = al16(o + static_cast<size_t>(nstage) * kG * npad * esz);
  L.rec_tw = o;   o = al16(o + (tmem_rec ? 0 : static_cast<size_t>(2) * ecap * 16));
  L.rec_x = o;    o = al16(o + static_cast<size_t>(2) * ecap * 2);
  L.work = o;     o = al16(o + static_cast<size_t>(kRows * 2 * kG) * kRegion * 8);
  L.acc = o;      o = al16(o + static_cast<size_t>(kRows) * kC * 16);
  L.tlo = o;      o = al16(o + (static_cast<size_t>(1) << tw_shift) * 8);
  L.thi = o;      o = al16(o + static_cast<size_t>(nhi) * 8);
  L.wmeta = o;    o = al16(o + static_cast<size_t>(kWarps) * kItems * 4);
  L.wdst = o;     o = al16(o + static_cast<size_t>(kWarps) * 32 * kItems * 2);
  L.wovb = o;     o = al16(o + static_cast<size_t>(kWarps) * 32 * kItems * 4);
  L.ibase = o;    o = al16(o + static_cast<size_t>(kWarps) * kItems * 4);
  L.istart = o;   o = al16(o + static_cast<size_t>(kWarps * kItems + 1) * 4);
  L.slot_src = o; o = al16(o + (static_cast<size_t>(2) * ecap / 32 + 1) * 4);
  L.bar = o;      o = al16(o + 8);
  L.total = o;
  return L;
}

// One task (t, row pair, k-range) of the fast kernel; `sm` is the block's
// dynamic shared memory (fast_layout).
//
// The gather front end is laid out per warp: warp w owns kItems (side,
// bucket group) items, dealt in snake order so that the heavy (first)
// groups of each side spread over all warps.  The prologue copies the
// records of warp w's items, item after item, into one contiguous stream
// (slot s holds 32 lanes' records), and keeps per item its padded count
// (warp-uniform) and per lane the Y slot its bucket is stored to, so the
// per-group loop only walks the stream.
//
// With tmem_rec the twiddle records live in tensor memory instead (for
// hash domains whose records do not fit in shared memory): warp w's item j
// owns the 32 columns 32 j .. 32 j + 31 of its lane quarter (w mod 4) and
// column half (w / 4), entry e at columns 32 j + 4 e .. + 3 (an item holds
// at most 8 entries per lane: the capped bucket count); `trow` is the
// warp's tensor-memory row address.
template <typename T>
__device__ __forceinline__ void fast_task(const FastArgs& p, const int task, unsigned char* sm, uint32_t trow) {
  const SmemLayout L = fast_layout(p.npad, p.ecap, p.alias, p.tw_shift, p.nhi, static_cast<int>(sizeof(T)),
                                   p.tmem_rec);
  T* stage = reinterpret_cast<T*>(sm + L.stage);      // FP32 or BF16 as stored
  float4* rec_tw = reinterpret_cast<float4*>(sm + L.rec_tw);     // [slot][lane]: row 0 tw, row 1 tw
  uint16_t* rec_x = reinterpret_cast<uint16_t*>(sm + L.rec_x);   // [slot][lane]: staging index
  float2* work = reinterpret_cast<float2*>(sm + L.work);
  float4* acc = reinterpret_cast<float4*>(sm + L.acc);
  float2* tlo = reinterpret_cast<float2*>(sm + L.tlo);
  float2* thi = reinterpret_cast<float2*>(sm + L.thi);
  uint32_t* wmeta = reinterpret_cast<uint32_t*>(sm + L.wmeta);   // [warp][item]: cnt | side << 8 | overflow steps << 9
  uint16_t* wdst = reinterpret_cast<uint16_t*>(sm + L.wdst);     // [warp][item][lane]: Y slot (row 0, k 0)
  // [warp][item][lane]: the lane's overflow list, start | length << 16 (both
  // below n, which the planner keeps under 2^16 for this kernel: 3 npad <= 65535)
  uint32_t* wovb = reinterpret_cast<uint32_t*>(sm + L.wovb);
  uint32_t* ibase = reinterpret_cast<uint32_t*>(sm + L.ibase);   // [warp][item]: side * ecap + first record
  uint32_t* istart = reinterpret_cast<uint32_t*>(sm + L.istart); // [warp][item]: first stream slot; [64]: total
  uint32_t* slot_src = reinterpret_cast<uint32_t*>(sm + L.slot_src);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = task % p.nkc;
  const int unit = (task / p.nkc) % p.nunits;
  const int t = task / (p.nkc * p.nunits);
  // rows of this block: 2 unit, 2 unit + 1 (the odd last unit repeats its row)
  uint32_t f1r[kRows];
  f1r[0] = static_cast<uint32_t>(2 * unit);
  f1r[1] = static_cast<uint32_t>(min(2 * unit + 1, p.nrows - 1));
  const bool row1_live = 2 * unit + 1 < p.nrows;
  const int n = p.n;
  const int S = 1 << p.tw_shift;
  const ModB modb = make_modb(p.b);
  const float w2pi = static_cast<float>(6.283185307179586 / static_cast<double>(p.b));
  const int nstage = p.alias ? 1 : 2;
  const int k_begin = kc * p.kchunk;
  const int k_end = min(p.n2, k_begin + p.kchunk);

  // ---- prologue: tables, item streams, staging tails, accumulators -------
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
  const int C = p.C, Pq = p.P, Qq = p.Q, Gq = p.G;   // C = Pq Qq buckets in Gq groups per side
  if (tid < kWarps * kItems) {
    const int w = tid / kItems, j = tid % kItems;
    const int slot = (j & 1) ? (kWarps - 1 - w) : w;
    const int item = j * kWarps + slot;
    const int side = item & 1, gi = item >> 1;
    if (item < 2 * Gq) {
      const size_t ts = static_cast<size_t>(t) * 2 + side;
      const uint32_t gb = p.grp[(ts * Gq + gi) * 2];
      const uint32_t gy = p.grp[(ts * Gq + gi) * 2 + 1];
      wmeta[tid] = (gy & 0xFFu) | (static_cast<uint32_t>(side) << 8) | (((gy >> 16) & 0x7FFFu) << 9);
      ibase[tid] = static_cast<uint32_t>(side) * p.ecap + gb;
    } else {
      wmeta[tid] = kVoidItem;
      ibase[tid] = 0;
    }
  }
  for (int i = tid; i < kWarps * 32 * kItems; i += kThreads) {
    const int w = i / (32 * kItems), j = (i / 32) % kItems, l = i % 32;   // [w][j][l]: one item's lanes together
    const int slot = (j & 1) ? (kWarps - 1 - w) : w;
    const int item = j * kWarps + slot;
    const int side = item & 1, gi = item >> 1;
    const size_t ts = static_cast<size_t>(t) * 2 + side;
    const uint32_t z = item < 2 * Gq ? p.dest[(ts * Gq + gi) * 32 + l] : 0u;
    wdst[i] = item < 2 * Gq ? static_cast<uint16_t>(side * kG * kRegion + z) : 0;
    // the lane's overflow list (the same for every inner index)
    uint32_t ob = 0;
    if (item < 2 * Gq && z < static_cast<uint32_t>(C) && ((p.grp[(ts * Gq + gi) * 2 + 1] >> 16) & 0x7FFFu)) {
      const uint32_t o = p.ovf_off[ts * (C + 1) + z];
      ob = o | ((p.ovf_off[ts * (C + 1) + z + 1] - o) << 16);
    }
    wovb[i] = ob;
  }
  for (int i = tid; i < kRows * kC; i += kThreads) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  // zero the staging tails [n_side, npad): entries x >= n_side read zeros.
  // Rows that are not 16-byte aligned are copied as their aligned superset
  // (starting up to 16 bytes early, ending up to 16 bytes late), so that
  // staged row k begins at element shift(k); such entries then read the zero
  // slot zpos instead, past anything a copy writes
  for (int s2 = 0; s2 < nstage; ++s2) {
    const int nside = p.unal ? p.zpos : (s2 == 0 ? p.n1 : p.n3);
    for (int g = 0; g < kG; ++g)
      for (int i = nside + tid; i < p.npad; i += kThreads) stage[(s2 * kG + g) * p.npad + i] = T(0.f);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t s = 0;
    for (int i = 0; i < kWarps * kItems; ++i) { istart[i] = s; s += wmeta[i] & 0xFFu; }
    istart[kWarps * kItems] = s;
  }
  __syncthreads();
  if (tid < kWarps * kItems) {
    const uint32_t c = wmeta[tid] & 0xFFu, s0 = istart[tid], b0 = ibase[tid];
    for (uint32_t r = 0; r < c; ++r) slot_src[s0 + r] = b0 + 32u * r;
  }
  __syncthreads();
  // records in stream order: staging index of x and s(x) w_b^{(h(x) f1) mod b}
  // for both rows; padding entries (x = n) read the zeroed staging tail
  const size_t tbase = static_cast<size_t>(t) * 2 * p.ecap;
  auto rec_twiddles = [&](uint32_t i) {
    const uint32_t src = slot_src[i >> 5] + (i & 31u);
    const uint32_t x = p.rec_x[tbase + src];
    const uint32_t w = p.rec_hs[tbase + src];
    float2 tw[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      tw[r] = make_float2(0.f, 0.f);
      if (x < static_cast<uint32_t>(n)) {
        tw[r] = wb(tlo, thi, mulmod(w & kBucketMask, f1r[r], modb), p.tw_shift);
        if (w >> 31) { tw[r].x = -tw[r].x; tw[r].y = -tw[r].y; }
      }
    }
    return make_float4(tw[0].x, tw[0].y, tw[1].x, tw[1].y);
  };
  {
    const uint32_t nrec = istart[kWarps * kItems] * 32u;
    for (uint32_t i = tid; i < nrec; i += kThreads) {
      const uint32_t src = slot_src[i >> 5] + (i & 31u);
      const uint32_t side = src >= p.ecap ? 1u : 0u;
      const uint32_t x = p.rec_x[tbase + src];
      if (!p.tmem_rec) rec_tw[i] = rec_twiddles(i);
      const uint32_t nsd = static_cast<uint32_t>(side ? p.n3 : p.n1);
      const uint32_t xs = p.unal ? (x < nsd ? x : static_cast<uint32_t>(p.zpos)) : min(x, static_cast<uint32_t>(n));
      rec_x[i] = static_cast<uint16_t>((p.alias ? 0u : side * kG * static_cast<uint32_t>(p.npad)) + xs);
    }
  }
  if (p.tmem_rec) {
    // each warp writes its own items' twiddles to its tensor-memory row
#pragma unroll 1
    for (int j = 0; j < kItems; ++j) {
      const uint32_t cnt = wmeta[warp * kItems + j] & 0xFFu;
      const uint32_t s0 = istart[warp * kItems + j];
      float v[32];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (static_cast<uint32_t>(e) < cnt) w4 = rec_twiddles((s0 + e) * 32u + lane);
        v[4 * e + 0] = w4.x; v[4 * e + 1] = w4.y; v[4 * e + 2] = w4.z; v[4 * e + 3] = w4.w;
      }
      __syncwarp();   // the tensor-memory store is warp-collective
      tmem_st32(trow + 32u * static_cast<uint32_t>(j), v);
    }
    tmem_wait_st();
  }
  // lane twiddle anchors w_1024^{lane * 8 q}, q = 0..3, and the step w_1024^lane
  float2 anchor[4];
  float2 step;
  {
    float s, c;
    sincospif(2.0f * static_cast<float>(lane) / static_cast<float>(C), &s, &c);
    step = make_float2(c, -s);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sincospif(2.0f * static_cast<float>((lane * 8 * q) % C) / static_cast<float>(C), &s, &c);
      anchor[q] = make_float2(c, -s);
    }
  }

  // issue the TMA copies of the group starting at k0 (thread 0 only)
  auto issue = [&](int k0) {
    uint32_t bytes = 0;
    const int gl = min(kG, k_end - k0);
    const T* A = static_cast<const T*>(p.A);
    const T* B = static_cast<const T*>(p.B);
    // the 16-byte aligned superset of each row (the row itself when aligned)
    auto span = [&](const T* row, int len, uintptr_t* a0) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(row);
      *a0 = a & ~static_cast<uintptr_t>(15);
      return static_cast<uint32_t>(((a + static_cast<uintptr_t>(len) * sizeof(T) + 15) & ~static_cast<uintptr_t>(15)) - *a0);
    };
    uintptr_t a0;
    for (int g = 0; g < gl; ++g) {
      if (p.n1 > 0) bytes += span(A + static_cast<size_t>(k0 + g) * p.lda, p.n1, &a0);
      if (!p.alias && p.n3 > 0) bytes += span(B + static_cast<size_t>(k0 + g) * p.ldb, p.n3, &a0);
    }
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, bytes);
    for (int g = 0; g < gl; ++g) {
      if (p.n1 > 0) {
        const uint32_t nb = span(A + static_cast<size_t>(k0 + g) * p.lda, p.n1, &a0);
        bulk_g2s(stage + (0 * kG + g) * p.npad, reinterpret_cast<const void*>(a0), nb, bar);
      }
      if (!p.alias && p.n3 > 0) {
        const uint32_t nb = span(B + static_cast<size_t>(k0 + g) * p.ldb, p.n3, &a0);
        bulk_g2s(stage + (1 * kG + g) * p.npad, reinterpret_cast<const void*>(a0), nb, bar);
      }
    }
  };

  // Each warp accumulates the spectral product of its (row, k-slot) pair for
  // 16 of its 32 bins: side-a warps own m = 0..15, side-b warps m = 16..31.
  float2 part[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) part[m] = make_float2(0.f, 0.f);

  if (tid == 0 && k_begin < k_end) issue(k_begin);
  __syncthreads();

  // warp -> (row, side, inner index of the group); region = warp
  const int side_w = (warp >> 1) & 1;
  const int g_w = warp & 1;
  float2* region = work + warp * kRegion;
  // partner: same row and k slot, other side
  const float2* partner = work + (warp ^ 2) * kRegion;
  const int own_m0 = side_w * 16;       // bins this warp accumulates: m in [own_m0, own_m0 + 16)
  uint32_t phase = 0;
  int group = 0;
  bool timed_out = false;

  for (int k0 = k_begin; k0 < k_end; k0 += kG, ++group) {
    const int gcnt = min(kG, k_end - k0);
    // ---- wait for this group's staging ----------------------------------
    const bool ok = mbar_wait_bounded(bar, phase);
    if (__syncthreads_or(!ok)) { timed_out = true; break; }
    phase ^= 1u;
    // ---- gather front end (both rows, both inner indices) ----------------
    {
      const uint32_t s0 = istart[warp * kItems];
      const float4* twp = rec_tw + s0 * 32u + lane;
      const uint16_t* xp = rec_x + s0 * 32u + lane;
      const T* st1 = stage + p.npad;
      // element offsets of the staged rows inside their aligned copies
      int shA0 = 0, shA1 = 0, shB0 = 0, shB1 = 0;
      if (p.unal) {
        const T* A = static_cast<const T*>(p.A);
        const T* B = static_cast<const T*>(p.B);
        const int k1 = min(k0 + 1, p.n2 - 1);
        shA0 = static_cast<int>((reinterpret_cast<uintptr_t>(A + static_cast<size_t>(k0) * p.lda) & 15) / sizeof(T));
        shA1 = static_cast<int>((reinterpret_cast<uintptr_t>(A + static_cast<size_t>(k1) * p.lda) & 15) / sizeof(T));
        shB0 = p.alias ? shA0 : static_cast<int>((reinterpret_cast<uintptr_t>(B + static_cast<size_t>(k0) * p.ldb) & 15) / sizeof(T));
        shB1 = p.alias ? shA1 : static_cast<int>((reinterpret_cast<uintptr_t>(B + static_cast<size_t>(k1) * p.ldb) & 15) / sizeof(T));
      }
      // neither loop is unrolled: the smaller loop body keeps the hot code
      // in the instruction cache (measured faster than unrolled forms)
#pragma unroll 1
      for (int j = 0; j < kItems; ++j) {
        const uint32_t m = wmeta[warp * kItems + j];
        const uint32_t dst = wdst[(warp * kItems + j) * 32 + lane];
        const uint32_t cnt = m & 0xFFu;
        const bool sb = (m >> 8) & 1u;
        const T* sg0 = stage + (sb ? shB0 : shA0);
        const T* sg1 = st1 + (sb ? shB1 : shA1);
        float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;   // [row][k]
        if (p.tmem_rec) {
          // the item's (at most 8) entries' twiddles in one tensor-memory load
          float wr[32];
          __syncwarp();
          tmem_ld32(trow + 32u * static_cast<uint32_t>(j), wr);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if (static_cast<uint32_t>(e) < cnt) {
              const int x = xp[32 * e];
              const float v0 = generic::to_f32(sg0[x]);
              const float v1 = generic::to_f32(sg1[x]);
              const float4 w = make_float4(wr[4 * e], wr[4 * e + 1], wr[4 * e + 2], wr[4 * e + 3]);
              a00.x = fmaf(v0, w.x, a00.x); a00.y = fmaf(v0, w.y, a00.y);
              a01.x = fmaf(v1, w.x, a01.x); a01.y = fmaf(v1, w.y, a01.y);
              a10.x = fmaf(v0, w.z, a10.x); a10.y = fmaf(v0, w.w, a10.y);
              a11.x = fmaf(v1, w.z, a11.x); a11.y = fmaf(v1, w.w, a11.y);
            }
          }
        } else {
#pragma unroll 1
          for (uint32_t e = 0; e < cnt; ++e) {
            const int x = xp[32 * e];
            const float4 w = twp[32 * e];
            const float v0 = generic::to_f32(sg0[x]);
            const float v1 = generic::to_f32(sg1[x]);
            a00.x = fmaf(v0, w.x, a00.x); a00.y = fmaf(v0, w.y, a00.y);
            a01.x = fmaf(v1, w.x, a01.x); a01.y = fmaf(v1, w.y, a01.y);
            a10.x = fmaf(v0, w.z, a10.x); a10.y = fmaf(v0, w.w, a10.y);
            a11.x = fmaf(v1, w.z, a11.x); a11.y = fmaf(v1, w.w, a11.y);
          }
        }
        // the entries of the lane's bucket past the capped count (the
        // bucket's overflow list; the table builder groups buckets of
        // similar totals, so the lanes' lists are of similar length), with
        // on-the-fly twiddles (wb_sfu)
        const uint32_t om = (m >> 9) & 0x7FFFu;
        if (om) {
          const size_t ts = static_cast<size_t>(t) * 2 + (sb ? 1 : 0);
          const uint32_t ob = wovb[(warp * kItems + j) * 32 + lane];
          uint32_t o = ob & 0xFFFFu;
          const uint32_t o1 = o + (ob >> 16);
          const uint32_t* ox = p.ovf_x + ts * n;
          const uint32_t* oh = p.ovf_hs + ts * n;
          const uint32_t soff = p.alias || !sb ? 0u : static_cast<uint32_t>(kG * p.npad);
          const uint32_t nsd = static_cast<uint32_t>(sb ? p.n3 : p.n1);
          // the two rows are f1 and f1 + 1 (or the same row twice for the
          // last unit of an odd count), so the second phase is the first
          // plus h (mod b) or the first itself
          const uint32_t bb = static_cast<uint32_t>(p.b);
          const bool step1 = f1r[1] != f1r[0];
          uint32_t nx = 0, nh = 0;
          if (o < o1) { nx = ox[o]; nh = oh[o]; }
#pragma unroll 1
          for (; o < o1; ++o) {
            const uint32_t x = nx, hv = nh;
            if (o + 1 < o1) { nx = ox[o + 1]; nh = oh[o + 1]; }
            const uint32_t hb = hv & kBucketMask;
            const uint32_t e0 = mulmod(hb, f1r[0], modb);
            uint32_t e1 = step1 ? e0 + hb : e0;
            if (e1 >= bb) e1 -= bb;
            float2 w0 = wb_sfu(e0, bb, w2pi);
            float2 w1 = wb_sfu(e1, bb, w2pi);
            if (hv >> 31) { w0.x = -w0.x; w0.y = -w0.y; w1.x = -w1.x; w1.y = -w1.y; }
            const uint32_t xr = soff + (p.unal && x >= nsd ? static_cast<uint32_t>(p.zpos) : x);
            const float v0 = generic::to_f32(sg0[xr]);
            const float v1 = generic::to_f32(sg1[xr]);
            a00.x = fmaf(v0, w0.x, a00.x); a00.y = fmaf(v0, w0.y, a00.y);
            a01.x = fmaf(v1, w0.x, a01.x); a01.y = fmaf(v1, w0.y, a01.y);
            a10.x = fmaf(v0, w1.x, a10.x); a10.y = fmaf(v0, w1.y, a10.y);
            a11.x = fmaf(v1, w1.x, a11.x); a11.y = fmaf(v1, w1.y, a11.y);
          }
        }
        xp += 32u * cnt;
        twp += 32u * cnt;
        if (m & kVoidItem) continue;
        float2* dp = work + dst;
        dp[0] = a00;
        dp[kRegion] = a01;
        dp[2 * kG * kRegion] = a10;
        dp[2 * kG * kRegion + kRegion] = a11;
      }
    }
    __syncthreads();
    // staging consumed: fetch the next group while the FFTs run
    if (tid == 0 && k0 + kG < k_end) issue(k0 + kG);
    // ---- FFT of length C = P Q, one per warp -------------------------------
    // lane l < P holds Y[l + P j], j < Q: DFT of length Q over j in
    // registers, twiddle w_C^{l f1}, transpose, then lanes f1 < Q run the DFT
    // of length P over l: lane f1 ends holding bins f1 + Q f2 in x[f2]
    float2 x[32];
    if (Pq == 32 && Qq == 32) {
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = region[lane + 32 * j];
      dft32<false>(x);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        x[j] = (j < Qq && lane < Pq) ? region[lane + Pq * j] : make_float2(0.f, 0.f);
      if (Qq == 32) dft32<false>(x);
      else dft_reg(x, Qq);
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
    __syncwarp();
    // transpose through the padded region: T[f][lane] at f * 33 + lane
#pragma unroll
    for (int f = 0; f < 32; ++f)
      if (f < Qq) region[f * kPitch + lane] = x[f];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j)
      x[j] = (lane < Qq && j < Pq) ? region[lane * kPitch + j] : make_float2(0.f, 0.f);
    if (Pq == 32) dft32<false>(x);
    else dft_reg(x, Pq);
    __syncwarp();
    // hand the partner the half of the bins it accumulates (register indices
    // must stay compile-time constants: one branch per side)
    if (side_w == 0) {
#pragma unroll
      for (int m = 16; m < 32; ++m) region[lane + 32 * m] = x[m];
    } else {
#pragma unroll
      for (int m = 0; m < 16; ++m) region[lane + 32 * m] = x[m];
    }
    // only the partner warp (same row and k slot, other side) must be done;
    // named barrier 1 + pair index, 64 threads
    asm volatile("bar.sync %0, 64;" ::"r"(1 + ((warp & 1) | ((warp >> 2) << 1))) : "memory");
    // ---- spectral products: own half of the bins -------------------------
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
    // ---- fold the partial sums into the Kahan accumulators ---------------
    const bool last = k0 + kG >= k_end;
    if ((group % kFlush) == kFlush - 1 || last) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        region[lane + 32 * (own_m0 + m)] = part[m];
        part[m] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int idx = tid; idx < kRows * C; idx += kThreads) {
        const int r = idx / C, f = idx % C;
        const int f2 = f / Qq;             // bin f = f1 + Q f2 sits at lane f1, register f2
        const int widx = (f - f2 * Qq) + 32 * f2;
        const int sd = f2 >> 4;            // registers < 16 live with side a, the rest with side b
        float2 s = work[((r * 2 + sd) * kG + 0) * kRegion + widx];
#pragma unroll
        for (int g = 1; g < kG; ++g) {
          const float2 v = work[((r * 2 + sd) * kG + g) * kRegion + widx];
          s.x += v.x;
          s.y += v.y;
        }
        float4 a = acc[r * kC + f];
        kahan_add(a.x, a.z, s.x);
        kahan_add(a.y, a.w, s.y);
        acc[r * kC + f] = a;
      }
    }
    // the next group's __syncthreads_or orders these reads of the regions
    // before the front end overwrites them
  }

  if (timed_out) {
    if (tid == 0) atomicOr(&g_sketch_error, 1u);
    __syncthreads();
    return;
  }
  __syncthreads();
  for (int idx = tid; idx < kRows * C; idx += kThreads) {
    const int r = idx / C, f = idx % C;
    if (r == 1 && !row1_live) continue;
    const float4 a = acc[r * kC + f];
    const uint32_t frow = r ? f1r[1] : f1r[0];
    float2* out = p.partial + ((static_cast<size_t>(t) * p.nrows + frow) * p.nkc + kc) * C;
    out[f] = make_float2(a.x - a.z, a.y - a.w);
  }
  // the shared memory (and the mbarrier in it) is reused by the next task
  __syncthreads();
  if (tid == 0) mbar_inval(bar);
  __syncthreads();
}

// Tensor memory for the records of tmem_rec tasks: 512 columns per block
// (the launch asks for enough shared memory that one block fits per SM, so
// the allocation never waits on another block); returns this warp's row.
__device__ __forceinline__ uint32_t tmem_take(uint32_t* slot) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tmem_alloc(slot, 512);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  return *slot + ((static_cast<uint32_t>(warp & 3) * 32u) << 16) + static_cast<uint32_t>(warp >> 2) * 256u;
}

__device__ __forceinline__ void tmem_give(uint32_t* slot) {
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(*slot, 512);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_sketch_fast(FastArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint32_t s_tmem;
  const uint32_t trow = p.tmem_rec ? tmem_take(&s_tmem) : 0u;
  fast_task<T>(p, blockIdx.x, sm, trow);
  if (p.tmem_rec) tmem_give(&s_tmem);
}

// ------------------------------------------------------------- batched ----
// One persistent launch over the tasks of many instances (sketches of
// different (A, B) pairs, shapes and storage types).  Blocks take tasks from
// an atomic counter in the order the host laid them out (longest first);
// each task runs the fast or the generic body and writes only its own
// partial row, so the result does not depend on which block ran which task.
__global__ void __launch_bounds__(kThreads, 1)
k_sketch_batched(const BatchDesc* __restrict__ desc, const int* __restrict__ start, int ninst,
                 int total, int* next, int use_tmem) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ int s_task;
  __shared__ uint32_t s_tmem;
  const uint32_t trow = use_tmem ? tmem_take(&s_tmem) : 0u;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = atomicAdd(next, 1);
    __syncthreads();
    const int gtask = s_task;
    if (gtask >= total) break;
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= gtask) lo = mid; else hi = mid - 1;
    }
    const BatchDesc& d = desc[lo];
    const int task = gtask - start[lo];
    if (d.kind == 1) {
      fast_task<float>(d.f, task, sm, trow);
    } else if (d.kind == 3) {
      fast_task<__nv_bfloat16>(d.f, task, sm, trow);
    } else {
      float4* sm4 = reinterpret_cast<float4*>(sm);
      switch (d.g.dt) {
        case CMS_F32: generic::generic_task<float>(d.g, task, sm4); break;
        case CMS_BF16: generic::generic_task<__nv_bfloat16>(d.g, task, sm4); break;
        default: generic::generic_task<double>(d.g, task, sm4); break;
      }
      __syncthreads();
    }
  }
  if (use_tmem) tmem_give(&s_tmem);
}

}  // namespace

uint32_t read_clear_error_sketch() {
  uint32_t v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_sketch_error, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
  if (v) cudaMemcpyToSymbol(g_sketch_error, &zero, sizeof(zero));
  return v;
}

size_t fast_smem_bytes(int npad, uint32_t ecap, int alias, int tw_shift, int nhi, int esz, int tmem_rec) {
  return fast_layout(npad, ecap, alias, tw_shift, nhi, esz, tmem_rec).total;
}

size_t batch_desc_bytes() { return sizeof(BatchDesc); }

size_t batch_smem_bytes(const SketchPlan& plan) { return plan.smem; }

// Descriptor of one instance of a batched launch (host memory `dst`).
void fill_batch_desc(void* dst, const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                     const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3, int dt, char* ws) {
  BatchDesc d{};
  float2* partial = reinterpret_cast<float2*>(ws + plan.off_partial);
  if (plan.fast) {
    d.kind = dt == CMS_BF16 ? 3 : 1;
    FastArgs& a = d.f;
    a.A = A; a.lda = lda;
    a.B = B; a.ldb = ldb;
    a.esz = dt == CMS_BF16 ? 2 : 4;
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
    a.rec_x = h->d_fe_x; a.rec_hs = h->d_fe_hs; a.grp = h->d_fe_grp; a.dest = h->d_fe_dest;
    a.ovf_off = h->d_fe_ovf_off; a.ovf_x = h->d_fe_ovf_x; a.ovf_hs = h->d_fe_ovf_hs;
    a.partial = partial;
    a.C = static_cast<int>(plan.C);
    fe_pq(plan.C, &a.P, &a.Q);
    a.G = static_cast<int>((plan.C + 31) / 32);
    a.unal = plan.unal ? 1 : 0;
    a.zpos = plan.zpos;
    a.tmem_rec = plan.tmem_rec ? 1 : 0;
  } else {
    d.kind = 0;
    generic::SketchArgs& a = d.g;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
    a.n1 = static_cast<int>(n1); a.n2 = static_cast<int>(n2); a.n3 = static_cast<int>(n3);
    a.n = static_cast<int>(h->n);
    a.b = plan.b; a.R = static_cast<int>(plan.R); a.C = static_cast<int>(plan.C);
    a.nrows = plan.nrows; a.d = plan.d;
    a.nradC = plan.nradC;
    for (int i = 0; i < 16; ++i) a.radC[i] = plan.radC[i];
    a.G = plan.G; a.kchunk = static_cast<int>(plan.kchunk); a.nkc = plan.nkc;
    a.perm = h->d_perm; a.off = h->d_off;
    a.twfe = reinterpret_cast<const float2*>(ws + plan.off_twfe);
    a.twC = reinterpret_cast<const float2*>(ws + plan.off_twC);
    a.partial = partial;
    a.dt = dt;
  }
  std::memcpy(dst, &d, sizeof(d));
}

int batch_tasks(const SketchPlan& plan) {
  const int units = plan.fast ? plan.d * ((plan.nrows + 1) / 2) : plan.d * plan.nrows;
  return units * plan.nkc;
}

cudaError_t launch_sketch_batched(const void* d_desc, const int* d_start, int ninst, int total,
                                  int* d_next, size_t smem, int grid, int use_tmem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_sketch_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof_scope("k_sketch_batched", s);
    k_sketch_batched<<<grid, kThreads, smem, s>>>(static_cast<const BatchDesc*>(d_desc), d_start, ninst,
                                                  total, d_next, use_tmem);
  }
  return cudaGetLastError();
}

cudaError_t launch_sketch_fast(const SketchPlan& plan, const cms_hashes* h, const void* A,
                               int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                               int64_t n3, float2* partial, cudaStream_t s) {
  FastArgs a{};
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.esz = plan.dt == CMS_BF16 ? 2 : 4;
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
  a.partial = partial;
  a.C = static_cast<int>(plan.C);
  fe_pq(plan.C, &a.P, &a.Q);
  a.G = static_cast<int>((plan.C + 31) / 32);
  a.unal = plan.unal ? 1 : 0;
  a.zpos = plan.zpos;
  a.tmem_rec = plan.tmem_rec ? 1 : 0;
  const int smem = static_cast<int>(plan.smem);
  const bool bf = plan.dt == CMS_BF16;
  cudaError_t e = bf ? cudaFuncSetAttribute(k_sketch_fast<__nv_bfloat16>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                     : cudaFuncSetAttribute(k_sketch_fast<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned ntask = static_cast<unsigned>(static_cast<int64_t>(plan.d) * a.nunits * plan.nkc);
  {
    ProfScope prof_scope("k_sketch_fast", s);
    if (bf) k_sketch_fast<__nv_bfloat16><<<ntask, kThreads, smem, s>>>(a);
    else k_sketch_fast<float><<<ntask, kThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace cms
