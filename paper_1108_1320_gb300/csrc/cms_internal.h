// cms_internal.h - host-side declarations shared by the library's
// translation units (kernel launchers, the hash-set object, the plan).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "cms_common.cuh"

struct cms_hashes {
  int64_t n = 0;            // hash domain {0..n-1}
  int64_t b = 0;            // sketch length
  int32_t d = 0;            // repetitions
  uint64_t seed = 0;
  bool from_tables = false;
  cms::Coeffs coef{};       // host copy of the coefficients
  // factorisation b = R * C of the fused path (C = 0: b not 5-smooth)
  int64_t R = 0, C = 0;
  int device = 0;
  uint32_t* d_hs = nullptr;     // [d][2][n] packed bucket | sign
  uint32_t* d_perm = nullptr;   // [d][2][n] indices sorted by (bucket mod C), stable
  uint32_t* d_off = nullptr;    // [d][2][C+1] bucket-class offsets into d_perm
  // front-end records of the C = 1024 fused kernel (present when fe_ecap > 0)
  uint32_t fe_ecap = 0;
  uint32_t* d_fe_x = nullptr;      // [d][2][fe_ecap]
  uint32_t* d_fe_hs = nullptr;     // [d][2][fe_ecap]
  uint32_t* d_fe_grp = nullptr;    // [d][2][C/32][2] (base, count)
  uint16_t* d_fe_dest = nullptr;   // [d][2][C]
  uint32_t* d_fe_ovf_off = nullptr;  // [d][2][C+1]
  uint32_t* d_fe_ovf_x = nullptr;    // [d][2][n]
  uint8_t* d_fe_assign = nullptr;    // [d][2][32]: bucket group of each (warp, slot), cost-balanced
  uint32_t* d_fe_ovf_hs = nullptr;   // [d][2][n]: packed hash of each d_fe_ovf_x entry
};

namespace cms {

// Thread-local error text (set by the C entry points).
void set_error(const std::string& msg);

// Argument checks of the dense sketch entry points (cms_sketch_product and
// cms_sketch_product_noalloc share them, so both refuse the same inputs with
// the same text): hashes present, 0 <= n1, n3 <= hash domain n,
// 0 <= n2 < 2^31 (inner indices are 32-bit in the kernels), lda >= n1,
// ldb >= n3, a known dtype, c non-NULL, A and B non-NULL when they have
// entries, and the current device the one the hashes live on.  Sets the
// error text and returns its status, or CMS_OK.
int check_dense_call(const cms_hashes* h, const void* A, int64_t lda, const void* B, int64_t ldb,
                     int64_t n1, int64_t n2, int64_t n3, int32_t dt, const float* c);

// Brackets the launches in its scope with CUDA events on stream s while
// profiling is enabled (cms_profile_enable); a no-op otherwise.
// NVTX range around one C entry point, named after it: visible in a
// profiler's timeline (Nsight Systems, ncu's NVTX filters); without an
// attached tool the push and pop return at once (NVTX 3 is header-only and
// loads a tool library only when the profiler injects one).
class NvtxRange {
 public:
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Device error words: one per translation unit that owns kernels which can
// raise it.  Each reader returns the word and clears it.
uint32_t read_clear_error_decode();

// ------------------------------------------------------------- launchers --
// Fill d_hs from coefficients (hash evaluation on the device).
cudaError_t launch_hash_tables(const Coeffs& co, int d, int64_t n, int64_t b,
                               uint32_t* hs, cudaStream_t s);
// Stable counting sort of each [t][side] table by (bucket mod C).
cudaError_t launch_bucket_sort(const uint32_t* hs, int d, int64_t n, int64_t C,
                               uint32_t* perm, uint32_t* off, cudaStream_t s);

// Front-end record tables of the C = 1024 fused kernel.
constexpr int kFeC = 1024;        // FFT length of the specialised kernel
constexpr int kFeCap = 8;         // bucket entries kept in the padded layout
cudaError_t launch_frontend_tables(const uint32_t* hs, const uint32_t* perm, const uint32_t* off, int d,
                                   int64_t n, int64_t C, uint32_t ecap, uint32_t* rec_x, uint32_t* rec_hs,
                                   uint32_t* grp, uint16_t* dest, uint32_t* ovf_off, uint32_t* ovf_x,
                                   uint8_t* assign, uint32_t* ovf_hs, cudaStream_t s);
// Lengths of the in-register DFT codelets (and 32, the radix-32 DFT).
inline bool fe_supported_L(int64_t L) {
  return L == 16 || L == 18 || L == 20 || L == 24 || L == 25 || L == 27 || L == 30 || L == 32;
}
// The register-FFT kernels take C = P Q with P and Q codelet lengths: P
// lanes each run a DFT of length Q, then Q lanes a DFT of length P.  P = 32
// when possible (every lane busy in the first pass), else the largest P.
inline bool fe_pq(int64_t C, int* P, int* Q) {
  for (int p = 32; p >= 16; --p) {
    if (fe_supported_L(p) && C % p == 0 && fe_supported_L(C / p)) {
      if (P) *P = p;
      if (Q) *Q = static_cast<int>(C / p);
      return true;
    }
  }
  return false;
}
uint32_t read_clear_error_sketch();

// Plan of the fused sketch path for one call.
struct SketchPlan {
  int64_t b = 0, R = 0, C = 0;
  int nrows = 0;            // rows f1 = 0..floor(R/2) of the b = R*C grid
  int d = 0;
  int nradC = 0;
  int radC[16] = {0};
  int G = 1;                // inner indices per group in the fused kernel
  int64_t kchunk = 0;       // inner indices per task
  int nkc = 0;              // number of inner-index chunks
  int threads = 256;
  size_t smem = 0;          // dynamic shared memory of the fused kernel
  bool fast = false;        // a C = P Q register-FFT kernel applies
  int dt = 0;               // storage type of A and B (cms_dtype)
  bool ws = false;          // ... in its warp-specialised form (k_sketch_ws)
  int ovcap = 0;            // overflow entries whose twiddles k_sketch_ws caches
  bool alias = false;       // A and B are the same bytes (stage once)
  int npad = 0;             // staging row length of the fast kernel (elements)
  bool unal = false;        // rows not 16-byte aligned (the fast kernel copies aligned supersets)
  int zpos = 0;             // (unal) staging index of the zero slot
  int tw_shift = 0, nhi = 0;  // two-level w_b table: S = 2^tw_shift, nhi high entries
  bool wide = false;        // the cluster kernel for C = 2^16 rows (k_sketch_wide)
  bool tmem_rec = false;    // the lock-step kernel keeps its twiddle records in tensor memory
  bool sparse_sepy = false; // the sparse kernel scatters into Y buffers of its own (kept zero)
  // workspace layout (byte offsets)
  size_t off_partial = 0, off_V = 0, off_twfe = 0, off_twC = 0, off_twR = 0;
  size_t off_thi = 0;   // warp-specialised kernel: w_b^{i 2^tw_shift}, i < nhi
  size_t off_T = 0, off_wtab = 0;   // (wide) inverse pass buffer, bucket tables
  size_t off_dlist = 0, off_cd = 0; // (sparse) direct list + counts, FP64 direct sketch
  size_t ws_bytes = 0;
};

// Bucket tables of the cluster kernel in the workspace (byte offsets).
struct WideTables {
  int64_t entstride = 0, spstride = 0;
  size_t off_ent = 0, off_rec_xv = 0, off_rec_h = 0, off_nrec = 0;
  size_t off_sp_xv = 0, off_sp_h = 0, off_sp_bkt = 0, off_sp_cnt = 0;
  size_t end = 0;
};
constexpr int64_t kWideC = 65536;   // row length of the cluster kernel
WideTables wide_tables_layout(int d, int64_t n, size_t base);
size_t wide_smem_bytes();
int wide_max_clusters(int dt);
cudaError_t launch_sketch_wide(const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                               const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3, char* ws,
                               float2* partial, cudaStream_t s);
cudaError_t launch_inverse_wide(const SketchPlan& plan, const float2* partial, float2* V, float2* T,
                                const float2* tw256, const float2* twR, float* c, cudaStream_t s);
uint32_t read_clear_error_sketch_wide();
// K2b alone: real inverse length-R DFT over the rows, 1/b.
cudaError_t launch_cols_inverse(const SketchPlan& plan, const float2* V, const float2* twR, float* c,
                                cudaStream_t s,
                                const int32_t* skip_if_zero = nullptr);

bool choose_factorisation(int64_t b, int64_t* R, int64_t* C);
int make_sketch_plan(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3,
                     int dt, int num_sms, size_t smem_optin, SketchPlan* plan,
                     std::string* why, const void* A = nullptr, int64_t lda = 0,
                     const void* B = nullptr, int64_t ldb = 0, bool allow_fast = true,
                     int nkc_override = 0, int G_override = 0, bool allow_ws = true,
                     bool allow_wide = true);
size_t fast_smem_bytes(int npad, uint32_t ecap, int alias, int tw_shift, int nhi, int esz, int tmem_rec);
// Shared memory that keeps a block alone on its SM (a tensor-memory
// allocation of 512 columns then never waits on another block).
constexpr size_t kSmemOneBlockPerSm = 116 * 1024;
size_t ws_smem_bytes(int npad, uint32_t ecap, int alias, int tw_shift, int nhi, int ovcap);
bool ws_kernel_usable();
// thi: the kernel's high twiddle table w_b^{i 2^tw_shift}, i < nhi, already
// filled (k_twiddle_table with a high table; SketchPlan::off_thi)
cudaError_t launch_sketch_ws(const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                             const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3,
                             float2* partial, float2* thi, cudaStream_t s);
uint32_t read_clear_error_sketch_ws();
// Failure-detection self-test: one bounded wait on an mbarrier phase that
// nothing completes; *outcome = 1 when it gave up (designed), 2 when it
// completed.  Synchronous on s.
cudaError_t run_selftest_wait(cudaStream_t s, uint32_t* outcome);
cudaError_t launch_sketch_fast(const SketchPlan& plan, const cms_hashes* h, const void* A,
                               int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                               int64_t n3, float2* partial, cudaStream_t s);

cudaError_t launch_sketch(const SketchPlan& plan, const cms_hashes* h,
                          const void* A, int64_t lda, const void* B, int64_t ldb,
                          int64_t n1, int64_t n2, int64_t n3, int dt, float* c,
                          char* ws, cudaStream_t s);

// Fixed-order reduction of the k-range partials, inverse FFT, 1/b (K2a, K2b);
// twC / twR must hold w_C^m and w_R^m (launch_twiddle_tables).
// skip_if_zero (device, optional): when it holds 0 every block returns and c
// is left as it is.
cudaError_t launch_inverse(const SketchPlan& plan, const float2* partial, float2* V, const float2* twC,
                           const float2* twR, float* c, cudaStream_t s,
                           const int32_t* skip_if_zero = nullptr);
cudaError_t launch_twiddle_tables(float2* twC, int C, float2* twR, int R, cudaStream_t s);

// Reduction + inverse of many products in two launches (a batch): each
// instance's plan, partial rows, row spectra, twiddle tables and output.
struct InverseSpec {
  const SketchPlan* plan;
  const float2* partial;
  float2* V;
  const float2* twC;
  const float2* twR;
  float* c;
};
struct InverseBatch {
  void* buf = nullptr;      // device arguments (inverse_batch_bytes)
  int count = 0, row_blocks = 0, col_blocks = 0;
  size_t smem = 0;
  size_t o_rows = 0, o_cols = 0, o_rs = 0, o_cs = 0;
};
size_t inverse_batch_bytes(int count);
// Uploads the instances' arguments into d_buf (waits for the stream).
cudaError_t build_inverse_batch(const std::vector<InverseSpec>& specs, void* d_buf, InverseBatch* out,
                                cudaStream_t s);
cudaError_t launch_inverse_batched(const InverseBatch& ib, cudaStream_t s);
cudaError_t launch_frontend_twiddles(const SketchPlan& plan, const cms_hashes* h, char* ws, cudaStream_t s);

// Batched persistent launch (descriptors built on the host, copied to the device).
size_t batch_desc_bytes();
void fill_batch_desc(void* dst, const SketchPlan& plan, const cms_hashes* h, const void* A, int64_t lda,
                     const void* B, int64_t ldb, int64_t n1, int64_t n2, int64_t n3, int dt, char* ws);
int batch_tasks(const SketchPlan& plan);
cudaError_t launch_sketch_batched(const void* d_desc, const int* d_start, int ninst, int total,
                                  int* d_next, size_t smem, int grid, int use_tmem, cudaStream_t s);

// Sparse inputs (A by columns, B by rows).
struct SparseArgsHost {
  const int64_t* a_ptr; const int32_t* a_idx; const void* a_val;
  const int64_t* b_ptr; const int32_t* b_idx; const void* b_val;
  int n1, n3;
};
int make_sparse_plan(const cms_hashes* h, int64_t n2, int64_t K, int num_sms, size_t smem_optin,
                     SketchPlan* plan, size_t* off_klist, std::string* why);
// Ordered split of the nonempty inner indices into the FFT list (flist)
// and the direct list (dlist; limit < 0: none); counts[0..1] their lengths;
// scratch holds 2 x 1024 ints.
cudaError_t launch_nonempty_split(const int64_t* a_ptr, const int64_t* b_ptr, int64_t n2, int64_t limit,
                                  int32_t* flist, int32_t* dlist, int32_t* counts, int32_t* scratch, cudaStream_t s);
// The direct list's length is read on the device (counts[1]); n2 bounds it.
cudaError_t launch_direct_scatter(const cms_hashes* h, const SparseArgsHost& in, int dt, const int32_t* dlist,
                                  const int32_t* counts, int64_t n2, double* cd, cudaStream_t s);
cudaError_t launch_add_direct(float* c, const double* cd, int64_t len, const int32_t* counts, cudaStream_t s);
// FFT route over the nonempty inner indices klist[0..*kcount) (the length is
// read on the device, so the call needs no host wait); plan.nkc chunks per
// (repetition, row), trailing ones empty.  skip_empty: blocks return at once
// when the list is empty (the caller's inverse then skips too).
cudaError_t launch_sketch_sparse(const SketchPlan& plan, const cms_hashes* h, const SparseArgsHost& in,
                                 int dt, const int32_t* klist, const int32_t* kcount, int skip_empty,
                                 float2* partial, cudaStream_t s);

cudaError_t launch_decode_pairs_f32(const float* c, const cms_hashes* h,
                                    const int64_t* ij, int64_t q, float* out,
                                    cudaStream_t s);
cudaError_t launch_decode_pairs_f64(const double* c, const cms_hashes* h,
                                    const int64_t* ij, int64_t q, double* out,
                                    cudaStream_t s);
cudaError_t launch_decode_dense_f32(const float* c, const cms_hashes* h,
                                    int64_t n1, int64_t n3, float* out,
                                    int64_t ldo, cudaStream_t s);
cudaError_t launch_decode_threshold(const float* c, const cms_hashes* h, int64_t n1, int64_t n3, float tau,
                                    int skip_diagonal, int64_t* ij, float* val, int64_t capacity,
                                    int64_t* count, int64_t* rowcnt, cudaStream_t s);
cudaError_t launch_remove_diagonal(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                                   int64_t n3, int dt, const cms_hashes* h, float* c, cudaStream_t s);
size_t frobenius_ws_bytes(int64_t n1, int64_t n2, int64_t n3, int d);
int significant_code_length(int64_t n1, int64_t n3, int rho, int* L);
size_t significant_decode_ws_bytes(int d, int64_t b);
cudaError_t launch_decode_significant(const float* P, const cms_hashes* h, int64_t n1, int64_t n3, float delta,
                                      int rho, int64_t* ij, int64_t capacity, int64_t* count, char* ws,
                                      cudaStream_t s);
cudaError_t launch_mask_copy(const void* src, int64_t lds, void* dst, int64_t ldd, int64_t nx, int64_t n2, int r,
                             int rho, int dt, cudaStream_t s);
size_t nnz_ws_bytes(int d, int64_t b_max);
cudaError_t run_nnz_doubling(const SparseArgsHost& in, int dt, int64_t n2, const Coeffs& co, uint64_t seed,
                             int d, int64_t b_max, char* ws, int64_t* b_out, int64_t* worst_out, cudaStream_t s);
cudaError_t launch_frobenius(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2,
                             int64_t n3, int dt, uint64_t seed, int d, double* est, double* bound, char* ws,
                             cudaStream_t s);
cudaError_t launch_merge(const float* const* parts, int count, int64_t len,
                         float* out, cudaStream_t s);

// Plain FP64 path.
struct PlainPlan {
  int64_t b = 0;
  int nrad = 0;
  int rad[24] = {0};
  int64_t kc = 0;           // inner indices per scatter/FFT batch
  size_t off_Z = 0, off_Z2 = 0, off_S = 0, off_tw = 0;
  size_t ws_bytes = 0;
};
int make_plain_plan(const cms_hashes* h, int64_t n2, PlainPlan* plan, std::string* why);
cudaError_t launch_plain(const PlainPlan& plan, const cms_hashes* h,
                         const double* A, int64_t lda, const double* B, int64_t ldb,
                         int64_t n1, int64_t n2, int64_t n3, double* c, char* ws,
                         cudaStream_t s);

}  // namespace cms
