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
// (t, side), C <= 1024.  Counts use integer shared atomics (exact); the
// placement orders equal keys by warp, then by lane, i.e. by increasing x:
// the result does not depend on scheduling.
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
  // exclusive scan of the counts, 1024 buckets per round (warp shuffles,
  // then the 32 warp totals); cnt becomes the placement cursor
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ uint32_t wsum[kSortThreads / 32];
  __shared__ uint32_t rtot;
  uint32_t run = 0;
  for (uint32_t z0 = 0; z0 < C; z0 += kSortThreads) {
    const uint32_t z = z0 + threadIdx.x;
    const uint32_t v = z < C ? cnt[z] : 0u;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t wv = wsum[lane];
      uint32_t wi = wv;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (lane >= o) wi += u;
      }
      wsum[lane] = wi - wv;
      if (lane == 31) rtot = wi;
    }
    __syncthreads();
    const uint32_t ex = run + wsum[warp] + incl - v;
    if (z < C) { of[z] = ex; cnt[z] = ex; }
    run += rtot;
    __syncthreads();
  }
  if (threadIdx.x == 0) of[C] = run;
  __syncthreads();
  // placement, 1024 indices per round: per warp, the count of each key
  // among its 32 indices (match_any); per key, the offsets of the warps'
  // runs in warp order; each index then lands at cursor + warp offset +
  // its rank among the equal keys of its warp (x order within a key)
  uint32_t* tot = cnt + C;                                        // C
  uint16_t* wc = reinterpret_cast<uint16_t*>(tot + C);            // [warp][C]
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t nwc = (kSortThreads / 32) * C;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t x = base + threadIdx.x;
    const bool valid = x < n;
    const uint32_t key = valid ? (tab[x] & kBucketMask) % C : 0xFFFFFFFFu;
    for (uint32_t i = threadIdx.x; i < nwc; i += blockDim.x) wc[i] = 0;
    __syncthreads();
    const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key);
    const uint32_t rank = __popc(grp & lt_mask);
    if (valid && lane == __ffs(grp) - 1) wc[warp * C + key] = static_cast<uint16_t>(__popc(grp));
    __syncthreads();
    for (uint32_t z = threadIdx.x; z < C; z += blockDim.x) {
      uint32_t acc = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t v = wc[w * C + z];
        wc[w * C + z] = static_cast<uint16_t>(acc);
        acc += v;
      }
      tot[z] = acc;
    }
    __syncthreads();
    if (valid) pm[cnt[key] + wc[warp * C + key] + rank] = x;
    __syncthreads();
    for (uint32_t z = threadIdx.x; z < C; z += blockDim.x) cnt[z] += tot[z];
    __syncthreads();
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
  if (C < 1 || C > kSortThreads) return cudaErrorInvalidValue;
  // cursors and round totals (u32) and per-warp key counts (u16)
  const size_t smem = static_cast<size_t>(C) * (2 * sizeof(uint32_t) + (kSortThreads / 32) * sizeof(uint16_t));
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

namespace cms {
namespace {

// Scrambled 10-bit key of a bucket index: buckets of equal count are grouped
// in this order, not by z2, because the x of neighbouring buckets of a linear
// hash fall into the same shared-memory banks (x mod 32) in lock step.
__device__ __forceinline__ uint32_t bucket_scramble(uint32_t z) {
  z *= 0x9E3779B1u;
  z ^= z >> 15;
  z *= 0x85EBCA6Bu;
  z ^= z >> 13;
  return z >> 22;
}

// Front-end tables for the C = 1024 fused kernel, one block per (t, side).
// Buckets z2 = h mod C are ordered by capped count (<= kFeCap) descending,
// then so that each run of 32 buckets of a class holds every residue
// z2 mod 16 twice (scrambled order within a residue; in the full class,
// order of total count within a residue, so that a group's overflow lists
// are of similar length).  Consecutive runs of
// 32 buckets form a group whose lanes walk their buckets in lock step:
// entry r of the bucket at group position l sits at base[group] + 32 r + l
// (padding entries point at x = n, the fill this kernel writes).  Entries
// past the kFeCap-th of a bucket (in x order) go to a per-bucket overflow
// list.  This kernel writes each group's base, count and longest overflow
// list (count | longest << 16 | overflow flag << 31), each group
// position's bucket, the overflow offsets (warp and block scans over the
// bucket counts of the stable bucket sort (perm, off)) and the dealing of
// the groups to the front-end warps; k_frontend_records then places the
// entries of each group.
__global__ void __launch_bounds__(1024, 1)
k_frontend_tables(const uint32_t* __restrict__ hs, const uint32_t* __restrict__ perm,
                  const uint32_t* __restrict__ off, uint32_t n, uint32_t ecap,
                  uint32_t* __restrict__ rec_x, uint32_t* __restrict__ rec_hs,
                  uint32_t* __restrict__ grp, uint16_t* __restrict__ dest,
                  uint32_t* __restrict__ ovf_off, uint32_t* __restrict__ ovf_x,
                  uint8_t* __restrict__ assign, int C) {
  // C <= 1024 buckets in L = ceil(C / 32) groups; the block has kFeC = 1024
  // threads, thread z < C owning bucket z and warp g < L group g.  The slots
  // of the last group without a bucket (sort key all ones) hold no entries
  // and store their zero sums to Y[C + lane], past the buckets
  constexpr int kMax = kFeC;
  constexpr uint32_t kCap = static_cast<uint32_t>(kFeCap);
  __shared__ uint32_t cnt[kMax];        // entries per bucket
  __shared__ uint32_t key[kMax];
  __shared__ uint32_t used[kMax];       // greedy bank counters, 32 per warp
  __shared__ uint32_t gword[kMax / 32];  // group count | longest overflow list << 16 | overflow flag << 31
  __shared__ uint32_t wtot[32];
  __shared__ uint32_t gcost[kMax / 32];  // slots + longest overflow list of a group
  const int L = (C + 31) / 32;
  const int ts = blockIdx.x;
  const uint32_t* of = off + static_cast<size_t>(ts) * (C + 1);
  uint32_t* rx = rec_x + static_cast<size_t>(ts) * ecap;
  uint32_t* rh = rec_hs + static_cast<size_t>(ts) * ecap;
  uint32_t* gp = grp + static_cast<size_t>(ts) * ((C + 31) / 32) * 2;
  uint16_t* ds = dest + static_cast<size_t>(ts) * ((C + 31) / 32) * 32;
  uint32_t* oo = ovf_off + static_cast<size_t>(ts) * (C + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // bucket sizes from the stable bucket sort (perm lists each bucket's x in
  // increasing order)
  cnt[tid] = tid < C ? of[tid + 1] - of[tid] : 0u;
  used[tid] = bucket_scramble(static_cast<uint32_t>(tid));   // scrambled bucket order, read by the rank loop
  for (uint32_t e = tid; e < ecap; e += blockDim.x) { rx[e] = n; rh[e] = 0u; }
  __syncthreads();
  if (tid < C) {
    // rank of this bucket among the buckets of its class (capped count) and
    // residue z2 mod 16, in scrambled order; sorting by (class, rank / 2,
    // residue, rank % 2) makes every run of 32 buckets of a class hold each
    // residue twice (the Y stores of a group then need 2 wavefronts)
    const uint32_t z = static_cast<uint32_t>(tid);
    const uint32_t cc = min(cnt[z], kCap);
    const uint32_t sk = used[z];
    uint32_t rank = 0;
    if (cc < kCap) {
      for (uint32_t o = z & 15u; o < static_cast<uint32_t>(C); o += 16u) {
        const uint32_t so = used[o];
        if (min(cnt[o], kCap) == cc && (so < sk || (so == sk && o < z))) ++rank;
      }
    } else {
      // full buckets by total count, largest first, so that the buckets of
      // a group have overflow lists of similar length
      const uint32_t ck = cnt[z];
      for (uint32_t o = z & 15u; o < static_cast<uint32_t>(C); o += 16u) {
        const uint32_t co = cnt[o], so = used[o];
        if (co >= kCap && (co > ck || (co == ck && (so < sk || (so == sk && o < z))))) ++rank;
      }
    }
    key[tid] = ((kCap - cc) << 20) | ((rank >> 1) << 15) | ((z & 15u) << 11) | ((rank & 1u) << 10) | z;
  } else {
    key[tid] = 0xFFFFFFFFu;   // sorts after every bucket
  }
  __syncthreads();
  for (int size = 2; size <= kMax; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int partner = tid ^ stride;
      if (partner > tid) {
        const bool up = (tid & size) == 0;
        const uint32_t a = key[tid], b2 = key[partner];
        if ((a > b2) == up) { key[tid] = b2; key[partner] = a; }
      }
      __syncthreads();
    }
  }
  // Within each group of 32 buckets, place buckets so that each half-warp
  // holds distinct z2 mod 16 where possible: the front end's 8-byte stores
  // to Y[z2] are then free of bank conflicts.  The group's bucket set (and
  // so its padded length) is unchanged.
  // One warp per group, lane i holding the group's i-th key: the first
  // bucket of each residue (in group order) goes to the first half, the
  // second to the second half, the rest fill the first half up to 16 and
  // then the second, all in group order.
  if (warp < L) {
    uint32_t* grpkey = key + 32 * warp;
    const uint32_t kv = grpkey[lane];
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, (kv & 0x3FFu) & 15u);
    const uint32_t occ = __popc(same & lt);          // earlier keys of this residue
    const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, occ == 0);
    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, occ == 1);
    const uint32_t bp = __ballot_sync(0xFFFFFFFFu, occ >= 2);
    const uint32_t n0 = __popc(b0), n1 = __popc(b1);
    uint32_t slot;
    if (occ == 0) {
      slot = __popc(b0 & lt);
    } else if (occ == 1) {
      slot = 16u + __popc(b1 & lt);
    } else {
      const uint32_t pp = __popc(bp & lt);
      slot = n0 + pp < 16u ? n0 + pp : 16u + n1 + (pp - (16u - n0));
    }
    __syncwarp();
    grpkey[slot] = kv;
  }
  __syncthreads();
  // thread tid = group warp, lane: its bucket, the group's padded count
  const bool live = warp < L;                         // warp-uniform
  const bool real = key[tid] != 0xFFFFFFFFu;          // the sorted slot holds a bucket
  const uint32_t zs = real ? key[tid] & 0x3FFu : 0u;
  if (live) ds[tid] = static_cast<uint16_t>(real ? zs : static_cast<uint32_t>(C + lane));
  const uint32_t cz = real ? cnt[zs] : 0u;
  const uint32_t c = min(cz, kCap);
  uint32_t cm = c;
  for (int o = 16; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xFFFFFFFFu, cm, o));
  const bool any_ovf = __any_sync(0xFFFFFFFFu, cz > kCap);
  uint32_t om = cz > kCap ? cz - kCap : 0u;
  for (int o = 16; o > 0; o >>= 1) om = max(om, __shfl_xor_sync(0xFFFFFFFFu, om, o));
  if (lane == 0 && live) {
    gword[warp] = cm | (min(om, 0x7FFFu) << 16) | (any_ovf ? 0x80000000u : 0u);
    gcost[warp] = cm + om;
  }
  // overflow list offsets, by bucket index: block-wide exclusive scan
  const uint32_t ov = cnt[tid] > kCap ? cnt[tid] - kCap : 0u;
  uint32_t incl = ov;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t2 = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += t2;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    // group bases: exclusive scan of 32 x count over the L groups
    const uint32_t gw = lane < L ? gword[lane] : 0u;
    const uint32_t v = 32u * (gw & 0xFFFFu);
    uint32_t gi = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t2 = __shfl_up_sync(0xFFFFFFFFu, gi, o);
      if (lane >= o) gi += t2;
    }
    if (lane < L) {
      gp[2 * lane] = gi - v;
      gp[2 * lane + 1] = gw;
    }
    // warp offsets of the overflow scan
    const uint32_t wv = wtot[lane];
    uint32_t wi = wv;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t2 = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += t2;
    }
    wtot[lane] = wi - wv;
    if (lane == 31) oo[C] = wi;
  }
  if (warp == 1 && C == kMax) {
    // the 32 groups dealt to 8 front-end warps x 4 slots, heaviest first
    // (equal costs: lower group first) to the least-loaded warp with a free
    // slot (equal loads: lower warp); the warp-specialised kernel, C = 1024
    // only, takes 4 groups of each side per warp.  Lane g holds group g's
    // cost and its rank in that order; lanes 0..7 hold the warps' loads.
    uint8_t* as = assign + static_cast<size_t>(ts) * (kMax / 32);
    const uint32_t myc = gcost[lane];
    uint32_t rk = 0;
    for (int o = 0; o < 32; ++o) {
      const uint32_t co = __shfl_sync(0xFFFFFFFFu, myc, o);
      rk += (co > myc || (co == myc && o < lane)) ? 1u : 0u;
    }
    uint32_t load = 0, fill = 0;
    for (uint32_t i = 0; i < 32; ++i) {
      const int g = __ffs(__ballot_sync(0xFFFFFFFFu, rk == i)) - 1;
      const uint32_t cg = __shfl_sync(0xFFFFFFFFu, myc, g);
      uint64_t key = (lane < 8 && fill < 4) ? ((static_cast<uint64_t>(load) << 8) | static_cast<uint64_t>(lane))
                                            : ~0ull;
      for (int o = 4; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(0xFFFFFFFFu, key, o));
      if (lane < 8 && static_cast<uint64_t>(lane) == (key & 0xFFu)) {
        as[lane * 4 + fill] = static_cast<uint8_t>(g);
        ++fill;
        load += cg;
      }
    }
  }
  __syncthreads();
  const uint32_t my_oof = wtot[warp] + incl - ov;   // bucket tid's first overflow slot
  if (tid < C) oo[tid] = my_oof;
  // the records themselves are placed by k_frontend_records

}

// Records of one bucket group (one warp per (t, side, group)): each lane's
// entries (the first kFeCap of its bucket in x order) and the overflow
// entries of its bucket (x and its packed hash).  The entries are ordered bank-aware: step r gives
// each lane, in order of ascending count, its remaining entry whose bank
// (x mod 32) is least used at this step so far; padding lanes all read
// x = n (one address).  The order is sequential over the lanes, so the
// groups run as separate warps spread over the SMs.
__global__ void __launch_bounds__(32)
k_frontend_records(const uint32_t* __restrict__ hs, const uint32_t* __restrict__ perm,
                   const uint32_t* __restrict__ off, uint32_t n, uint32_t ecap, uint32_t* __restrict__ rec_x,
                   uint32_t* __restrict__ rec_hs, const uint32_t* __restrict__ grp, const uint16_t* __restrict__ dest,
                   const uint32_t* __restrict__ ovf_off, uint32_t* __restrict__ ovf_x,
                   uint32_t* __restrict__ ovf_hs, int C) {
  constexpr uint32_t kCap = static_cast<uint32_t>(kFeCap);
  __shared__ uint32_t ub[32];
  const int L = (C + 31) / 32;
  const int ts = blockIdx.x / L, g = blockIdx.x % L;
  const int lane = threadIdx.x;
  const uint32_t* tab = hs + static_cast<size_t>(ts) * n;
  const uint32_t* pm = perm + static_cast<size_t>(ts) * n;
  const uint32_t* of = off + static_cast<size_t>(ts) * (C + 1);
  uint32_t* rx = rec_x + static_cast<size_t>(ts) * ecap;
  uint32_t* rh = rec_hs + static_cast<size_t>(ts) * ecap;
  const uint32_t gb = grp[(static_cast<size_t>(ts) * L + g) * 2];
  const uint32_t cm = grp[(static_cast<size_t>(ts) * L + g) * 2 + 1] & 0xFFFFu;
  const uint32_t zd = dest[static_cast<size_t>(ts) * L * 32 + 32 * g + lane];
  const bool real = zd < static_cast<uint32_t>(C);
  const uint32_t zs = real ? zd : 0u;
  const uint32_t cz = real ? of[zs + 1] - of[zs] : 0u;
  const uint32_t c = min(cz, kCap);
  const uint32_t o0 = of[zs];
  const uint32_t oz = ovf_off[static_cast<size_t>(ts) * (C + 1) + zs];
  uint32_t* ox = ovf_x + static_cast<size_t>(ts) * n;
  uint32_t* oh = ovf_hs + static_cast<size_t>(ts) * n;
  uint32_t xs[kFeCap], wsv[kFeCap];
#pragma unroll
  for (uint32_t r = 0; r < kCap; ++r)
    if (r < c) xs[r] = pm[o0 + r];
#pragma unroll
  for (uint32_t r = 0; r < kCap; ++r)
    if (r < c) wsv[r] = tab[xs[r]];
  for (uint32_t r = kCap; r < cz; ++r) {
    const uint32_t x = pm[o0 + r];
    ox[oz + (r - kCap)] = x;
    oh[oz + (r - kCap)] = tab[x];
  }
  uint32_t rank = 0;
  for (int o = 0; o < 32; ++o) {
    const uint32_t co = __shfl_sync(0xFFFFFFFFu, c, o);
    rank += (co < c || (co == c && o < lane)) ? 1u : 0u;
  }
  // steps r unrolled so that every index into xs / wsv is a constant (the
  // arrays stay in registers); the lanes with no entry left at step r have
  // the lowest ranks and take no turn
#pragma unroll
  for (uint32_t r = 0; r < kCap; ++r) {
    if (r >= cm) break;
    ub[lane] = 0;
    const uint32_t done = __ballot_sync(0xFFFFFFFFu, c <= r);
    __syncwarp();
    if (lane == 0 && done) ub[n & 31u] = 1;
    __syncwarp();
    for (uint32_t k = __popc(done); k < 32; ++k) {
      if (rank == k) {
        uint32_t best = r, bu = ub[xs[r] & 31u];
#pragma unroll
        for (uint32_t i = r + 1; i < kCap; ++i) {
          if (i < c) {
            const uint32_t u = ub[xs[i] & 31u];
            if (u < bu) { bu = u; best = i; }
          }
        }
#pragma unroll
        for (uint32_t i = r + 1; i < kCap; ++i) {
          if (best == i) {
            const uint32_t tx = xs[r], tw = wsv[r];
            xs[r] = xs[i]; wsv[r] = wsv[i];
            xs[i] = tx; wsv[i] = tw;
          }
        }
        ub[xs[r] & 31u] += 1;
      }
      __syncwarp();
    }
  }
#pragma unroll
  for (uint32_t r = 0; r < kCap; ++r) {
    if (r < c) {
      rx[gb + 32u * r + lane] = xs[r];
      rh[gb + 32u * r + lane] = wsv[r];
    }
  }
}

}  // namespace

cudaError_t launch_frontend_tables(const uint32_t* hs, const uint32_t* perm, const uint32_t* off, int d,
                                   int64_t n, int64_t C, uint32_t ecap, uint32_t* rec_x, uint32_t* rec_hs,
                                   uint32_t* grp, uint16_t* dest, uint32_t* ovf_off, uint32_t* ovf_x,
                                   uint8_t* assign, uint32_t* ovf_hs, cudaStream_t s) {
  {
    ProfScope prof_scope("k_frontend_tables", s);
    k_frontend_tables<<<2 * d, kFeC, 0, s>>>(hs, perm, off, static_cast<uint32_t>(n), ecap, rec_x, rec_hs,
                                             grp, dest, ovf_off, ovf_x, assign, static_cast<int>(C));
  }
  {
    ProfScope prof_scope("k_frontend_records", s);
    const unsigned groups = static_cast<unsigned>(2 * d * ((C + 31) / 32));
    k_frontend_records<<<groups, 32, 0, s>>>(hs, perm, off, static_cast<uint32_t>(n), ecap, rec_x, rec_hs, grp,
                                              dest, ovf_off, ovf_x, ovf_hs, static_cast<int>(C));
  }
  return cudaGetLastError();
}

}  // namespace cms
