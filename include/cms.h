/*
 * cms.h - C ABI of the GB300 (sm_103a) compressed matrix multiplication
 * library (Pagh, "Compressed Matrix Multiplication", arXiv 1108.1320).
 *
 * The library computes the count sketch c[t][0..b-1], t = 0..d-1, of a matrix
 * product AB without forming AB (COMPRESSEDPRODUCT, Fig. 1), and decodes
 * entries as the median over t of s1_t(i) s2_t(j) c_t[(h1_t(i)+h2_t(j)) mod b]
 * (DECOMPRESS, Fig. 1).
 *
 * Conventions shared by every entry point:
 *  - Indices are 0-based.  A is n1 x n2, B is n2 x n3; k indexes n2.
 *  - Every matrix, sketch, output and workspace pointer is caller-owned
 *    DEVICE memory unless the parameter says "host".  The library owns only
 *    cms_hashes objects (host coefficients plus device tables).
 *  - Calls that take a stream are asynchronous on that stream (a
 *    cudaStream_t passed as void*; NULL means the legacy default stream).
 *    They allocate nothing: scratch comes from the caller's workspace.
 *  - Every call returns a cms_status; no call throws or aborts.  The text of
 *    the last error on the calling thread is returned by cms_last_error().
 *  - Device-side error words (a kernel that detects an impossible internal
 *    state) are surfaced by cms_check_async().
 *  - Threads: calls may come from several host threads.  A cms_hashes object
 *    is read by the compute calls and written by cms_reseed_hashes: reseeding
 *    while another call that reads the same object is in flight (on another
 *    stream or thread) races, as does freeing it; order them on one stream or
 *    synchronise.  Workspaces and outputs follow the same rule as any device
 *    buffer: one in-flight writer at a time.
 *  - Environment (for tests of alternative code paths; both give the same
 *    results as the default paths): CMS_WS_SMEM_SWAP makes the warp-
 *    specialised kernel swap half spectra through shared memory instead of
 *    tensor memory; CMS_SPARSE_INPLACE_Y makes the sparse-input route scatter
 *    into its FFT regions (zeroed every group) instead of per-warp buffers.
 *    Both are read at each call.
 */
#ifndef CMS_H
#define CMS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CMS_API __attribute__((visibility("default")))
#else
#define CMS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CMS_OK = 0,
    CMS_ERR_INVALID_ARG = 1,   /* bad pointer, size, stride or dtype       */
    CMS_ERR_UNSUPPORTED = 2,   /* valid but not implemented (e.g. b not 5-smooth) */
    CMS_ERR_CUDA = 3,          /* a CUDA runtime call failed               */
    CMS_ERR_WORKSPACE = 4,     /* workspace NULL or smaller than required  */
    CMS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up       */
    CMS_ERR_DEVICE = 6         /* a kernel raised its device error word    */
} cms_status;

typedef enum {
    CMS_F32 = 0,               /* IEEE binary32                            */
    CMS_BF16 = 1,              /* bfloat16 storage, computed in FP32       */
    CMS_F64 = 2                /* IEEE binary64 (rounded to FP32 by the fused path) */
} cms_dtype;

/* Opaque hash-function set: d repetitions of (h1, s1, h2, s2) over {0..n-1}. */
typedef struct cms_hashes cms_hashes;

/*
 * cms_make_hashes - draw d independent repetitions of the splitting and
 * sign functions (Fig. 1, first lines of COMPRESSEDPRODUCT; Sec. 2.2).
 *   h1_t, h2_t : {0..n-1} -> {0..b-1},  h(x) = ((a x + c) mod p) mod b,
 *   s1_t, s2_t : {0..n-1} -> {-1,+1},   s(x) = 1 - 2 (((a x + c) mod p) mod 2),
 * with p = 2^31 - 1 (the polynomial family of ref. [13], degree 1).  The
 * coefficients come from splitmix64 over `seed`: for t = 0..d-1, in the
 * order h1.a, h1.c, s1.a, s1.c, h2.a, h2.c, s2.a, s2.c, a = 1 + (r mod (p-1)),
 * c = r mod p.
 *   seed : any 64-bit value.
 *   n    : domain size, n = max(n1, n3) (h1/s1 index rows of A, h2/s2
 *          columns of B); 1 <= n <= 2^24.
 *   b    : sketch length, 1 <= b <= 2^24.  The fused FFT path needs b
 *          5-smooth (2^x 3^y 5^z); other b still hash and decode.
 *   d    : repetitions, 1 <= d <= 64.
 *   out  : host pointer receiving the new object.
 * Allocates device tables on the current device and fills them
 * synchronously.  Errors: CMS_ERR_INVALID_ARG, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_make_hashes(uint64_t seed, int64_t n, int64_t b, int32_t d,
                           cms_hashes** out);

/*
 * cms_reseed_hashes - redraw the functions of an existing object for a new
 * seed (same n, b, d), on the device, asynchronously on `stream`, without
 * allocating.  Calls using the object must be ordered after it on the
 * stream.  Errors: CMS_ERR_INVALID_ARG, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_reseed_hashes(cms_hashes* h, uint64_t seed, void* stream);

/*
 * cms_make_hashes_from_tables - build an object from explicit host tables
 * (test use: e.g. an injective splitting function, Sec. 2.2 special case).
 *   h1, h2 : host uint32 [d][n], values < b.   s1, s2 : host int8 [d][n], +-1.
 * Errors: CMS_ERR_INVALID_ARG, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_make_hashes_from_tables(int64_t n, int64_t b, int32_t d,
                                       const uint32_t* h1, const int8_t* s1,
                                       const uint32_t* h2, const int8_t* s2,
                                       cms_hashes** out);

/* Free an object and its device tables (synchronises the device). */
CMS_API cms_status cms_free_hashes(cms_hashes* h);

/*
 * cms_hashes_info - n, b, d and the FFT factorisation b = R * C chosen for
 * the fused path (R = 0, C = 0 when b is not 5-smooth).  Host outputs; any
 * may be NULL.
 */
CMS_API cms_status cms_hashes_info(const cms_hashes* h, int64_t* n, int64_t* b,
                           int32_t* d, int64_t* R, int64_t* C);

/*
 * cms_hashes_coeffs - the eight coefficients of repetition t, host out[8] in
 * the order h1.a, h1.c, s1.a, s1.c, h2.a, h2.c, s2.a, s2.c (all zero for an
 * object built from tables).
 */
CMS_API cms_status cms_hashes_coeffs(const cms_hashes* h, int32_t t, uint32_t out[8]);

/*
 * cms_hashes_tables - copy the tables to host buffers (synchronous):
 * h1, h2 uint32 [d][n]; s1, s2 int8 [d][n].  Any pointer may be NULL.
 */
CMS_API cms_status cms_hashes_tables(const cms_hashes* h, uint32_t* h1, int8_t* s1,
                             uint32_t* h2, int8_t* s2);

/*
 * cms_hashes_buckets - copy the bucket lists of repetition t and side
 * (0: h1 over rows of A, 1: h2 over columns of B) to host buffers
 * (synchronous; test and inspection use).  With C from cms_hashes_info:
 *   perm uint32 [n]: 0..n-1 stably sorted by h(x) mod C (equal keys keep
 *                    increasing x), the order the fused kernels' gather
 *                    front ends read a bucket class in (Sec. 2.2 scatter);
 *   off  uint32 [C + 1]: start of class z in perm; off[C] = n.
 * Either pointer may be NULL.  Errors: CMS_ERR_INVALID_ARG (t or side out
 * of range), CMS_ERR_UNSUPPORTED (C = 0: b is not 5-smooth, no lists).
 */
CMS_API cms_status cms_hashes_buckets(const cms_hashes* h, int32_t t, int32_t side, uint32_t* perm,
                              uint32_t* off);

/*
 * cms_workspace_size - bytes of device workspace cms_sketch_product needs
 * for these shapes (A n1 x n2, B n2 x n3, storage dtype dt).  Host output.
 * Errors: CMS_ERR_INVALID_ARG, CMS_ERR_UNSUPPORTED.
 */
CMS_API cms_status cms_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2,
                              int64_t n3, int32_t dt, size_t* bytes);

/*
 * cms_plan_kernel - which fused kernel cms_sketch_product would run for
 * these arguments (the choice depends on b, n, the storage type, the
 * alignment of A and B and whether they alias), without running it:
 *   CMS_KERNEL_SHARED_MEMORY      shared-memory Stockham FFTs (any 5-smooth b)
 *   CMS_KERNEL_LOCKSTEP           register FFTs, C = P Q, records in shared memory
 *   CMS_KERNEL_LOCKSTEP_TMEM      the same with the records in tensor memory
 *   CMS_KERNEL_WARP_SPECIALISED   register FFTs, C = 1024, FP32, front-end
 *                                 and FFT warps apart
 *   CMS_KERNEL_CLUSTER            rows of 2^16 bins over 8-CTA clusters
 * Errors: those of cms_sketch_product's argument checks.
 */
enum {
  CMS_KERNEL_SHARED_MEMORY = 0,
  CMS_KERNEL_LOCKSTEP = 1,
  CMS_KERNEL_LOCKSTEP_TMEM = 2,
  CMS_KERNEL_WARP_SPECIALISED = 3,
  CMS_KERNEL_CLUSTER = 4
};
CMS_API cms_status cms_plan_kernel(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                                   int64_t n2, int64_t n3, int32_t dt, const cms_hashes* h,
                                   int32_t* kernel_out);

/*
 * cms_sketch_product - COMPRESSEDPRODUCT(A, B, b, d) of Fig. 1 (Lemma 1):
 *   c[t][z] = sum over (i,j) with (h1_t(i)+h2_t(j)) mod b = z of
 *             s1_t(i) s2_t(j) (AB)_ij,
 * computed as in Sec. 2.2: per inner index k, count-sketch column k of A and
 * row k of B, FFT both, multiply pointwise and accumulate over k
 * (compensated FP32), then one inverse FFT per repetition.
 *   A   : n1 x n2, column-major, column k at A + k*lda (lda >= n1), so a
 *         single pass reads each a_k contiguously (Sec. 2.2, "single pass").
 *   B   : n2 x n3, row-major, row k at B + k*ldb (ldb >= n3).
 *   dt  : storage type of A and B (CMS_F32, CMS_BF16 or CMS_F64).
 *   h   : hashes with n >= max(n1, n3).
 *   c   : device float [d][b], written (not accumulated).
 *   ws  : device workspace of at least cms_workspace_size() bytes,
 *         256-byte aligned.
 * Errors: CMS_ERR_INVALID_ARG, CMS_ERR_UNSUPPORTED (b not 5-smooth or shape
 * beyond the kernels' limits), CMS_ERR_WORKSPACE, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_sketch_product(const void* A, int64_t lda, const void* B,
                              int64_t ldb, int64_t n1, int64_t n2, int64_t n3,
                              int32_t dt, const cms_hashes* h, float* c,
                              void* ws, size_t ws_bytes, void* stream);

/*
 * cms_sketch_product_noalloc - the same sketch as cms_sketch_product, for
 * callers that cannot allocate device memory or pass a workspace (for
 * example code running inside another application whose allocator owns all
 * device memory, or a path that must not call cudaMalloc/cudaFree because
 * they can synchronise the device).  The paper has no counterpart: this is a
 * memory-management variant of COMPRESSEDPRODUCT, not a different method.
 *   Arguments are those of cms_sketch_product without ws / ws_bytes; the
 *   caller still passes A, B, the hashes and the output c.
 *   Scratch: a fixed 32 MiB device array owned by the library (held on every
 *   GPU that loads it until the process exits).  Shapes whose
 *   cms_workspace_size() exceeds 32 MiB are rejected with CMS_ERR_WORKSPACE
 *   (the covariance shape n = 2048, b = 65536, d = 5 needs about 18 MiB).
 *   The call allocates nothing.  Its first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current;
 *   make that first call before any stream capture.  The address is cached
 *   per device for the life of the process; it does not survive a
 *   cudaDeviceReset (after one, reload the library before calling again).
 *   All calls on a device share the array, which keeps the previous call's
 *   contents (no part of it needs to start at zero): calls that overlap on
 *   the GPU (other streams or host threads) race and must be serialised by
 *   the caller.
 * Errors: those of cms_sketch_product, CMS_ERR_WORKSPACE above the limit.
 */
CMS_API cms_status cms_sketch_product_noalloc(const void* A, int64_t lda, const void* B,
                                              int64_t ldb, int64_t n1, int64_t n2, int64_t n3,
                                              int32_t dt, const cms_hashes* h, float* c,
                                              void* stream);

/*
 * cms_sparse_workspace_size / cms_sketch_product_csr - COMPRESSEDPRODUCT for
 * sparse inputs (Sec. 2.2: time O(N + n2 b lg b) when the nonzeros of a
 * column of A and of a row of B can be listed in linear time; Theorem 5's
 * exact recovery of sparse products).  Only inner indices k whose column
 * a_k and row b_k both have nonzeros contribute; they are compacted on the
 * device in increasing k.  Result as cms_sketch_product.
 *   a_colptr : device int64 [n2 + 1], CSC column pointers of A (n1 x n2).
 *   a_rowidx : device int32, row index of each nonzero of A (< n1).
 *   a_val    : device values of A, storage type dt.
 *   b_rowptr : device int64 [n2 + 1], CSR row pointers of B (n2 x n3).
 *   b_colidx : device int32, column index of each nonzero of B (< n3).
 *   b_val    : device values of B, storage type dt.
 *   Indices outside [0, n1) / [0, n3) contribute nothing.
 *   b must be a multiple of 1024 (CMS_ERR_UNSUPPORTED otherwise).
 *   Asynchronous: the list of nonempty k and its length stay on the device
 *   (the FFT route runs the workspace's worst-case chunking and reads the
 *   length there), so the call never waits for the stream and can be
 *   captured in a CUDA graph.
 */
CMS_API cms_status cms_sparse_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2,
                                             int64_t n3, size_t* bytes);
CMS_API cms_status cms_sketch_product_csr(const int64_t* a_colptr, const int32_t* a_rowidx,
                                          const void* a_val, const int64_t* b_rowptr,
                                          const int32_t* b_colidx, const void* b_val,
                                          int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                          const cms_hashes* h, float* c, void* ws,
                                          size_t ws_bytes, void* stream);

/*
 * cms_sketch_product_csr_hybrid - cms_sketch_product_csr with the sparse-k
 * hybrid: by linearity (Sec. 2.2, eq. (1)) c is the sum of the sketches of
 * the outer products a_k b_k; inner indices whose outer product has at
 * most `direct_max_pairs` terms (nnz(a_k) nnz(b_k)) are sketched directly
 * ("sketching a matrix product naively", Sec. 2.2: each term
 * s1(i) s2(j) A_ik B_kj added to bucket (h1(i) + h2(j)) mod b, in FP64),
 * the others through the FFT route of cms_sketch_product_csr; the two parts
 * are added and rounded once to FP32.
 *   direct_max_pairs : the split; < 0 selects 5 b log2(b) / 64, 0 sends
 *                      every inner index through the FFT route.
 *   The FP64 additions of the direct part are atomic: their order varies
 *   between calls (results agree to FP64 rounding, exactly when the values
 *   are integers).  Workspace: cms_sparse_workspace_size.  Other arguments,
 *   errors and asynchrony as cms_sketch_product_csr (the split is made on
 *   the device; the route whose list is empty returns at once).
 */
CMS_API cms_status cms_sketch_product_csr_hybrid(const int64_t* a_colptr, const int32_t* a_rowidx,
                                                 const void* a_val, const int64_t* b_rowptr,
                                                 const int32_t* b_colidx, const void* b_val,
                                                 int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                                 const cms_hashes* h, int64_t direct_max_pairs,
                                                 float* c, void* ws, size_t ws_bytes, void* stream);

/*
 * Batches: the paper treats one product; a batch runs COMPRESSEDPRODUCT on
 * many independent (A, B) pairs in one persistent launch.
 *
 * cms_instance - one product of a batch: the arguments of
 * cms_sketch_product (A column-major, B row-major, device pointers) plus its
 * hashes and its output c (device float [d][b]).
 */
typedef struct {
    const void* A;
    int64_t lda;
    const void* B;
    int64_t ldb;
    int64_t n1, n2, n3;
    int32_t dt;
    int32_t reserved;
    const cms_hashes* h;
    float* c;
} cms_instance;

typedef struct cms_batch cms_batch;

#define CMS_BATCH_AUTOTUNE 1

/*
 * Batches: many products of uneven shapes in one persistent launch (a
 * handle API: create once, run or replay many times, free).
 *
 * cms_batch_create - plan a batch of `count` instances (Fig. 1 for each):
 * allocates one device workspace for all of them, computes their constant
 * twiddle tables and uploads one task descriptor per instance (synchronous
 * on `stream`).  With flags & CMS_BATCH_AUTOTUNE, shapes not found in the
 * cache file `tune_cache` (may be NULL) are tuned by timing candidate
 * inner-index chunkings (and group sizes of the generic kernel) on the
 * instance's own data; results are written back to the file, one line per
 * key "b,n1,n2,n3,dt,d,SM count,kernel".
 * The instances' pointers are captured: the same buffers are used by every
 * run.  Errors: CMS_ERR_INVALID_ARG, CMS_ERR_UNSUPPORTED, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_batch_create(const cms_instance* items, int32_t count, int32_t flags,
                                    const char* tune_cache, void* stream, cms_batch** out);

/*
 * cms_batch_run - compute every instance's sketch c: one persistent kernel
 * over all instances' tasks (longest first, taken from an atomic work
 * counter; each task writes only its own partial row, so results do not
 * depend on scheduling), then the fixed-order reduction and inverse FFT of
 * every instance in two launches (rows, then columns).  Asynchronous,
 * allocates nothing.
 */
CMS_API cms_status cms_batch_run(cms_batch* b, void* stream);

/*
 * cms_batch_run_graph - the same, through a CUDA graph captured on the
 * first call (stream must not be the legacy default stream) and replayed
 * afterwards.  Hash tables reseeded after the capture are picked up (the
 * graph reads them at replay).
 */
CMS_API cms_status cms_batch_run_graph(cms_batch* b, void* stream);

/* Counts of instances, persistent-kernel tasks, kernel launches per run,
 * workspace bytes and instances served by the C = 1024 kernel (any NULL). */
CMS_API cms_status cms_batch_info(const cms_batch* b, int32_t* instances, int32_t* tasks,
                                  int32_t* launches, size_t* ws_bytes, int32_t* fast_instances);

/* Free a batch (synchronises the device). */
CMS_API cms_status cms_batch_free(cms_batch* b);

/*
 * cms_plain_workspace_size / cms_sketch_product_plain_f64 - the same sketch
 * (Fig. 1) in plain form: FP64 throughout, one instance per call, unfused
 * passes (scatter, FFT, spectral product, inverse FFT each a separate
 * kernel; spectra stored in device memory).  Same argument meanings as
 * cms_sketch_product with A, B double and c double [d][b].
 */
CMS_API cms_status cms_plain_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2,
                                    int64_t n3, size_t* bytes);
CMS_API cms_status cms_sketch_product_plain_f64(const double* A, int64_t lda,
                                        const double* B, int64_t ldb,
                                        int64_t n1, int64_t n2, int64_t n3,
                                        const cms_hashes* h, double* c,
                                        void* ws, size_t ws_bytes, void* stream);

/*
 * cms_decode - DECOMPRESS(i, j) of Fig. 1 for q index pairs:
 *   out[p] = median_t s1_t(i) s2_t(j) c_t[(h1_t(i) + h2_t(j)) mod b],
 * (i, j) = (ij[2p], ij[2p+1]).  An even d takes the mean of the two middle
 * values.
 *   c  : device float [d][b] from cms_sketch_product.
 *   ij : device int64 [q][2], 0 <= i < n, 0 <= j < n (out-of-range pairs
 *        produce NaN and raise the device error word).
 *   out: device float [q].
 * Errors: CMS_ERR_INVALID_ARG, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_decode(const float* c, const cms_hashes* h, const int64_t* ij,
                      int64_t q, float* out, void* stream);
CMS_API cms_status cms_decode_f64(const double* c, const cms_hashes* h,
                          const int64_t* ij, int64_t q, double* out,
                          void* stream);

/*
 * cms_decode_dense - every estimate C_ij, 0 <= i < n1, 0 <= j < n3
 * (Sec. 2.2: all entries in O(n^2) time): out[i*ldo + j] (row-major,
 * ldo >= n3), device float.  Errors: CMS_ERR_INVALID_ARG, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_decode_dense(const float* c, const cms_hashes* h, int64_t n1,
                            int64_t n3, float* out, int64_t ldo, void* stream);

/*
 * cms_sketch_remove_diagonal - covariance post-step (Sec. 3.2): a linear
 * sketch of Q gives one of Q~, Q with its diagonal set to zero.  With c the
 * sketch of AB (cms_sketch_product with the same operands and hashes), each
 * entry (AB)_ii = sum_k A_ik B_ki, i < min(n1, n3), formed in FP64, is
 * subtracted with sign s1_t(i) s2_t(i) from bucket (h1_t(i) + h2_t(i)) mod b
 * of every repetition t, in place.  For A = X^T, B = X this removes the
 * variances sum_k X_ki^2 (Fig. 2: "subtracting the contribution of diagonal
 * elements").
 *   A, lda, B, ldb, n1, n2, n3, dt : as cms_sketch_product.
 *   c : device float [d][b], updated in place (FP32 atomic subtractions:
 *       when several i share a bucket their order is unspecified).
 * Errors: CMS_ERR_INVALID_ARG for bad shapes, dtype or NULL pointers.
 */
CMS_API cms_status cms_sketch_remove_diagonal(const void* A, int64_t lda, const void* B, int64_t ldb,
                                              int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                              const cms_hashes* h, float* c, void* stream);

/*
 * cms_decode_threshold - the thresholding of Fig. 2: every (i, j), i < n1,
 * j < n3, whose estimate DECOMPRESS(i, j) (as cms_decode_dense) has
 * |estimate| > tau, skipping i = j when skip_diagonal is nonzero, without
 * forming the dense n1 x n3 matrix.
 *   ij_out    : device int64 [capacity][2], the hits in row-major order
 *               (i ascending, then j ascending), the first `capacity` of them.
 *   val_out   : device float [capacity], their estimates.
 *   count_out : device int64, the number of hits (may exceed capacity: call
 *               again with a larger buffer).
 *   ws        : device scratch of at least 8 (n1 + 1) bytes, 8-byte aligned.
 * The estimates are formed in FP32 (the even-d median is 0.5 (a + b) in
 * FP32), as is the comparison with tau.  Asynchronous on `stream`.
 * Errors: CMS_ERR_INVALID_ARG (bad sizes, tau < 0 or NaN, NULL pointers),
 * CMS_ERR_WORKSPACE (ws too small or misaligned).
 */
CMS_API cms_status cms_decode_threshold(const float* c, const cms_hashes* h, int64_t n1, int64_t n3,
                                        float tau, int32_t skip_diagonal, int64_t* ij_out,
                                        float* val_out, int64_t capacity, int64_t* count_out,
                                        void* ws, size_t ws_bytes, void* stream);

/*
 * cms_frobenius_workspace_size / cms_frobenius_estimate - Sec. 5.2: an upper
 * bound on ||AB||_F^2 (hence on the sketch's error scale ||AB||_F / sqrt(b))
 * from d AMS sketches of AB,
 *   X_t = sum_ij s1_t(i) s2_t(j) (AB)_ij = sum_k (s1_t . a_k)(b_k . s2_t),
 * with 4-wise independent signs s(x) = 1 - 2 (((a3 x^3 + a2 x^2 + a1 x + a0)
 * mod p) mod 2), p = 2^31 - 1, whose coefficients are drawn by splitmix64
 * from `seed` (order: t, then s1 and s2, then a0..a3; each r mod p).  X_t^2
 * estimates ||AB||_F^2 without bias; the bound is 32 times the median of the
 * X_t^2 (even d: mean of the two middle ones).  One pass over A and B;
 * sums in FP64.
 *   A, lda, B, ldb, n1, n2, n3, dt : as cms_sketch_product.
 *   est_out   : device double [d], the X_t.
 *   bound_out : device double [1], 32 median X_t^2.
 *   ws        : device scratch of cms_frobenius_workspace_size bytes,
 *               256-byte aligned.
 * Errors: CMS_ERR_INVALID_ARG (sizes, d outside [1, 64], NULL pointers),
 * CMS_ERR_WORKSPACE.
 */
CMS_API cms_status cms_frobenius_workspace_size(int64_t n1, int64_t n2, int64_t n3, int32_t d,
                                                size_t* bytes);
CMS_API cms_status cms_frobenius_estimate(const void* A, int64_t lda, const void* B, int64_t ldb,
                                          int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                          uint64_t seed, int32_t d, double* est_out,
                                          double* bound_out, void* ws, size_t ws_bytes,
                                          void* stream);

/*
 * cms_nnz_workspace_size / cms_nnz_estimate - Sec. 5.1: the doubling search
 * for the number of nonzero entries of AB (sparse A by columns, B by rows,
 * as cms_sketch_product_csr).  For b = 2, 4, 8, ... up to b_max it sketches
 * (D1 A)(B D2), D1 and D2 random diagonal scalings in [1, 2) (so that, by
 * the Schwartz-Zippel lemma, a bucket sums to zero only when every entry of
 * AB hashed to it is zero), with the d splitting and sign functions of
 * Fig. 1 drawn from `seed` (as cms_make_hashes; range b), every term added
 * in FP64; a bucket counts as zero when |sum| <= 1e-9 (sum of |terms|).  It
 * stops at the first b where every repetition has at most b/5 nonzero
 * buckets: then b bounds the number of nonzeros from above with
 * probability 1 - (3/4)^d, and b <= 10 nnz(AB).
 *   b_out       : host int64, that b, or -1 when b_max was passed first.
 *   buckets_out : host int64, the largest count of nonzero buckets at b.
 *   ws          : device scratch of cms_nnz_workspace_size(d, b_max) bytes.
 * The call waits for the stream once per doubling step.
 * Errors: CMS_ERR_INVALID_ARG (sizes, d outside [1, 64], b_max outside
 * [2, 2^30], NULL pointers), CMS_ERR_WORKSPACE.
 */
CMS_API cms_status cms_nnz_workspace_size(int32_t d, int64_t b_max, size_t* bytes);
CMS_API cms_status cms_nnz_estimate(const int64_t* a_colptr, const int32_t* a_rowidx, const void* a_val,
                                    const int64_t* b_rowptr, const int32_t* b_colidx, const void* b_val,
                                    int64_t n1, int64_t n2, int64_t n3, int32_t dt, uint64_t seed,
                                    int32_t d, int64_t b_max, int64_t* b_out, int64_t* buckets_out,
                                    void* ws, size_t ws_bytes, void* stream);

/*
 * FINDSIGNIFICANTENTRIES (Sec. 4, Fig. 3).
 *
 * cms_find_significant - 2 l sketches of AB with the hashes h: for r < l of
 * (I_{E_r} A) B (rows i of A kept when bit r of E(i) is 1), for r >= l of
 * A (B I_{E_{r-l}}); for every repetition t and bucket k the bits
 * |p^(t,r)[k]| > delta/2 are decoded into a position (i, j); positions
 * decoded for at least d/2 of the (t, k) are returned.  E is a balanced
 * repetition code (the paper's expander code is not defined there): for
 * each of the L = ceil(log2 max(n1, n3)) bits of x, least significant
 * first, rho copies of the bit then rho copies of its complement,
 * l = 2 rho L; decoding is a majority vote per bit, a tie or a string
 * farther than l/4 from the decoded codeword decodes to nothing.  Cost:
 * 2 l sketch products.
 *   A, lda, B, ldb, n1, n2, n3, dt : as cms_sketch_product (n1, n3 >= 1).
 *   delta     : the magnitude threshold Delta (>= 0).
 *   rho       : copies per bit, 1..8.
 *   ij_out    : device int64 [capacity][2], the positions (in the order of
 *               the device's atomic appends; sort for a canonical order).
 *   count_out : device int64, the number of positions (may exceed capacity).
 *   ws        : device scratch of cms_significant_workspace_size bytes,
 *               256-byte aligned.
 * cms_decode_significant - the decode and vote alone, on 2 l given
 * sketches (device float [2 l][d][b], as above), with a scratch of
 * cms_significant_decode_workspace_size bytes.
 * Errors: CMS_ERR_INVALID_ARG, CMS_ERR_WORKSPACE, and those of
 * cms_sketch_product.
 */
CMS_API cms_status cms_significant_workspace_size(const cms_hashes* h, int64_t n1, int64_t n2, int64_t n3,
                                                  int32_t dt, int32_t rho, size_t* bytes);
CMS_API cms_status cms_find_significant(const void* A, int64_t lda, const void* B, int64_t ldb,
                                        int64_t n1, int64_t n2, int64_t n3, int32_t dt,
                                        const cms_hashes* h, float delta, int32_t rho, int64_t* ij_out,
                                        int64_t capacity, int64_t* count_out, void* ws, size_t ws_bytes,
                                        void* stream);
CMS_API cms_status cms_significant_decode_workspace_size(const cms_hashes* h, size_t* bytes);
CMS_API cms_status cms_decode_significant(const float* sketches, const cms_hashes* h, int64_t n1,
                                          int64_t n3, float delta, int32_t rho, int64_t* ij_out,
                                          int64_t capacity, int64_t* count_out, void* ws,
                                          size_t ws_bytes, void* stream);

/*
 * cms_merge - c_out[t][z] = sum over the `count` partial sketches (device
 * float [d][b] each, pointers in a host array) in index order.  The sketch
 * is linear in the outer products of eq. (1) (Sec. 2.2), so sketches of
 * disjoint inner-index ranges add up to the sketch of the whole product.
 */
CMS_API cms_status cms_merge(const float* const* parts, int32_t count, int32_t d,
                     int64_t b, float* c_out, void* stream);

/*
 * cms_selftest_wait - self-test of the failure detection.  Every wait a
 * kernel of this library makes on another agent (a TMA copy completing an
 * mbarrier phase) gives up after a fixed limit (2 s of %globaltimer), records
 * that in a device word and lets the kernel finish, so that the host gets
 * CMS_ERR_TIMEOUT instead of a hung device.  This call runs that bounded wait
 * on a phase nothing completes (one thread, one block) on the given stream and
 * synchronises it: it returns CMS_ERR_TIMEOUT when the wait gave up (the
 * designed outcome, after about 2 s), CMS_ERR_DEVICE if the wait completed,
 * CMS_ERR_CUDA if a CUDA call failed.  The device stays usable afterwards.
 */
CMS_API cms_status cms_selftest_wait(void* stream);

/* Surface asynchronous device errors for work queued on `stream`:
 * synchronises the stream, then reads and clears the device error word. */
CMS_API cms_status cms_check_async(void* stream);

/*
 * Tracing (no counterpart in the paper).  The compute entry points (hash
 * draws, the sketch calls, batches, decodes, post-steps, estimators,
 * FINDSIGNIFICANTENTRIES, merge) each open an NVTX range named after the
 * entry point, visible in a profiler's timeline; without an attached tool
 * the ranges cost a function call.
 *
 * cms_profile_enable - per-kernel device timing (no counterpart in the
 * paper).  While on, every kernel the library launches is bracketed by CUDA
 * events recorded on the stream it runs on.  Switching on or off clears the
 * records (waiting for pending events).  Not for use during graph capture.
 */
CMS_API cms_status cms_profile_enable(int32_t on);

/*
 * cms_profile_summary - the records so far as a JSON object
 * {"kernel": {"launches": L, "ms": T}, ...} in the host buffer buf[len]
 * (waits for the recorded events).  *needed (if not NULL) receives the
 * size including the terminating NUL.  Errors: CMS_ERR_INVALID_ARG when
 * the buffer is too small, CMS_ERR_CUDA.
 */
CMS_API cms_status cms_profile_summary(char* buf, size_t len, size_t* needed);

CMS_API const char* cms_status_string(cms_status s);
CMS_API const char* cms_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CMS_H */
