// k_significant.cu - FINDSIGNIFICANTENTRIES (Sec. 4, Fig. 3).
//
// 2 l sketches of AB are taken with the same hash functions: for r < l the
// sketch of (I_{E_r} A) B (rows i of A with bit r of E(i) equal to 0 set to
// zero), for r >= l the sketch of A (B I_{E_{r-l}}) (columns j of B masked by
// E(j)).  For every repetition t and bucket k the string of bits
// |p^(t,r)[k]| > Delta/2 is decoded into a position (i, j), and positions
// decoded for at least d/2 of the (t, k) are returned.
//
// The code E: the paper asks for an expander code and defines none.  Here E
// is a balanced repetition code: for each of the L = ceil(log2 max(n1, n3))
// bits of x (least significant first), rho copies of the bit followed by rho
// copies of its complement, l = 2 rho L.  DECODE takes a majority vote per
// bit (a tie rejects the string) and rejects strings farther than l/4 from
// the decoded codeword, so an empty bucket (all bits 0) decodes to nothing.
//
// Kernels: the masked copy of A or B (one pass over the operand), the
// ordinary sketch path for each of the 2 l products, the decode (one thread
// per (t, k), keys i n3 + j + 1), and the multiset count: an open-addressing
// table of at least twice as many slots as keys (atomicCAS on the key,
// atomicAdd on its count); positions with a count of at least d/2 are
// appended to the output (their order is that of the atomic appends).
#include <algorithm>

#include "cms_internal.h"

namespace cms {
namespace {

__device__ __forceinline__ uint32_t code_bit(uint32_t x, int r, int rho) {
  const int q = r / (2 * rho), e = r - q * 2 * rho;
  const uint32_t bit = (x >> q) & 1u;
  return e < rho ? bit : 1u - bit;
}

template <typename T>
__global__ void k_mask_copy(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd, int64_t nx,
                            int64_t n2, int r, int rho) {
  for (int64_t k = blockIdx.y; k < n2; k += gridDim.y) {
    for (int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < ldd;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      T v = static_cast<T>(0.f);
      if (x < nx && code_bit(static_cast<uint32_t>(x), r, rho)) v = src[k * lds + x];
      dst[k * ldd + x] = v;
    }
  }
}

// decode one side: bits r0 .. r0 + l of the (t, k) column; -1 when rejected
__device__ __forceinline__ int64_t decode_side(const float* __restrict__ P, size_t stride, int r0, int L, int rho,
                                               float half) {
  int64_t x = 0;
  int dist = 0;
  for (int q = 0; q < L; ++q) {
    int votes = 0;
    for (int e = 0; e < 2 * rho; ++e) {
      const int bit = fabsf(P[static_cast<size_t>(r0 + q * 2 * rho + e) * stride]) > half ? 1 : 0;
      votes += e < rho ? bit : 1 - bit;
    }
    if (votes == rho) return -1;
    const int bit = votes > rho ? 1 : 0;
    x |= static_cast<int64_t>(bit) << q;
    dist += bit ? 2 * rho - votes : votes;
  }
  return 4 * dist <= 2 * rho * L ? x : -1;
}

__global__ void k_sig_decode(const float* __restrict__ P, int d, int64_t b, int64_t n1, int64_t n3, float delta,
                             int L, int rho, uint64_t* __restrict__ keys) {
  const int ell = 2 * rho * L;
  const size_t stride = static_cast<size_t>(d) * b;   // between consecutive sketches r
  const float half = delta * 0.5f;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < static_cast<int64_t>(d) * b;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* col = P + q;   // sketch r of (t, k) at col[r * stride]
    uint64_t key = 0;
    const int64_t i = decode_side(col, stride, 0, L, rho, half);
    if (i >= 0 && i < n1) {
      const int64_t j = decode_side(col, stride, ell, L, rho, half);
      if (j >= 0 && j < n3) key = static_cast<uint64_t>(i) * static_cast<uint64_t>(n3) + static_cast<uint64_t>(j) + 1u;
    }
    keys[q] = key;
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// the table has at least twice as many slots as keys, so a probe sequence
// always reaches the key's slot or an empty one within tsize steps
__global__ void k_sig_count(const uint64_t* __restrict__ keys, int64_t nkeys, unsigned long long* __restrict__ tkey,
                            unsigned int* __restrict__ tcnt, uint64_t tmask) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < nkeys;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint64_t key = keys[q];
    if (key == 0) continue;
    uint64_t slot = mix64(key) & tmask;
    for (uint64_t step = 0; step <= tmask; ++step) {
      const unsigned long long prev = atomicCAS(&tkey[slot], 0ull, static_cast<unsigned long long>(key));
      if (prev == 0ull || prev == key) {
        atomicAdd(&tcnt[slot], 1u);
        break;
      }
      slot = (slot + 1) & tmask;
    }
  }
}

__global__ void k_sig_collect(const unsigned long long* __restrict__ tkey, const unsigned int* __restrict__ tcnt,
                              uint64_t tsize, int d, int64_t n3, int64_t* __restrict__ ij, int64_t capacity,
                              unsigned long long* __restrict__ count) {
  for (uint64_t s = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < tsize;
       s += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long key = tkey[s];
    if (key == 0ull || 2 * static_cast<int64_t>(tcnt[s]) < d) continue;
    const unsigned long long pos = atomicAdd(count, 1ull);
    if (static_cast<int64_t>(pos) < capacity) {
      const uint64_t v = key - 1;
      ij[2 * pos] = static_cast<int64_t>(v / static_cast<uint64_t>(n3));
      ij[2 * pos + 1] = static_cast<int64_t>(v % static_cast<uint64_t>(n3));
    }
  }
}

size_t a256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

uint64_t table_slots(int d, int64_t b) {
  uint64_t t = 1;
  while (t < 2 * static_cast<uint64_t>(d) * static_cast<uint64_t>(b)) t <<= 1;
  return t;
}

}  // namespace

int significant_code_length(int64_t n1, int64_t n3, int rho, int* L) {
  int bits = 1;
  while ((static_cast<int64_t>(1) << bits) < std::max<int64_t>(std::max(n1, n3), 2)) ++bits;
  if (L) *L = bits;
  return 2 * rho * bits;
}

size_t significant_decode_ws_bytes(int d, int64_t b) {
  return a256(static_cast<size_t>(d) * b * 8) + a256(table_slots(d, b) * 8) + a256(table_slots(d, b) * 4);
}

cudaError_t launch_decode_significant(const float* P, const cms_hashes* h, int64_t n1, int64_t n3, float delta,
                                      int rho, int64_t* ij, int64_t capacity, int64_t* count, char* ws,
                                      cudaStream_t s) {
  int L = 0;
  significant_code_length(n1, n3, rho, &L);
  const int d = h->d;
  const int64_t b = h->b;
  const uint64_t ts = table_slots(d, b);
  uint64_t* keys = reinterpret_cast<uint64_t*>(ws);
  unsigned long long* tkey = reinterpret_cast<unsigned long long*>(ws + a256(static_cast<size_t>(d) * b * 8));
  unsigned int* tcnt = reinterpret_cast<unsigned int*>(ws + a256(static_cast<size_t>(d) * b * 8) + a256(ts * 8));
  cudaError_t e = cudaMemsetAsync(tkey, 0, ts * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tcnt, 0, ts * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const int64_t nk = static_cast<int64_t>(d) * b;
  const unsigned g1 = static_cast<unsigned>(std::min<int64_t>((nk + 255) / 256, 8192));
  {
    ProfScope prof_scope("k_sig_decode", s);
    k_sig_decode<<<g1, 256, 0, s>>>(P, d, b, n1, n3, delta, L, rho, keys);
  }
  {
    ProfScope prof_scope("k_sig_count", s);
    k_sig_count<<<g1, 256, 0, s>>>(keys, nk, tkey, tcnt, ts - 1);
  }
  {
    ProfScope prof_scope("k_sig_collect", s);
    const unsigned g2 = static_cast<unsigned>(std::min<uint64_t>((ts + 255) / 256, 8192));
    k_sig_collect<<<g2, 256, 0, s>>>(tkey, tcnt, ts, d, n3, ij, capacity,
                                     reinterpret_cast<unsigned long long*>(count));
  }
  return cudaGetLastError();
}

cudaError_t launch_mask_copy(const void* src, int64_t lds, void* dst, int64_t ldd, int64_t nx, int64_t n2, int r,
                             int rho, int dt, cudaStream_t s) {
  if (n2 == 0) return cudaSuccess;
  dim3 g(static_cast<unsigned>(std::min<int64_t>((ldd + 255) / 256, 64)),
         static_cast<unsigned>(std::min<int64_t>(n2, 65535)));
  ProfScope prof_scope("k_mask_copy", s);
  switch (dt) {
    case CMS_F32:
      k_mask_copy<float><<<g, 256, 0, s>>>(static_cast<const float*>(src), lds, static_cast<float*>(dst), ldd, nx, n2,
                                           r, rho);
      break;
    case CMS_BF16:
      k_mask_copy<__nv_bfloat16><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(src), lds,
                                                   static_cast<__nv_bfloat16*>(dst), ldd, nx, n2, r, rho);
      break;
    default:
      k_mask_copy<double><<<g, 256, 0, s>>>(static_cast<const double*>(src), lds, static_cast<double*>(dst), ldd, nx,
                                            n2, r, rho);
      break;
  }
  return cudaGetLastError();
}

}  // namespace cms
