/*
 * gbid.h -- C ABI of the GB300 interpolative-decomposition (ID) library.
 *
 * The library computes the rank-k interpolative decomposition of
 * Advani & O'Hagan, "Efficient Algorithms for Constructing an Interpolative
 * Decomposition" (arXiv 2105.07076):
 *
 *   Definition 1 (Sec. 1.2)  A ~= C Z, C = k columns of A (the skeleton J),
 *                            Z (k x n) holds a k x k identity at columns J.
 *   Sec. 2.1                 A P = Q R by column-pivoted Householder QR, J =
 *                            the first k pivots, Z from the least-squares
 *                            problem min ||A - C Z||_F; with Q_k^T A P =
 *                            [R11 R12] its solution is Z P = [I  T],
 *                            T = R11^{-1} R12 (back substitution).
 *   Sec. 4.1                 the QR stops after k pivots.
 *   Sec. 2 (footnote)        if m > n the method runs on A^T and returns a
 *                            row ID: A ~= Z^T A[J, :].
 *
 * Conventions shared by every entry point:
 *   - All array pointers are DEVICE pointers owned by the caller, except the
 *     optional `id_info*` which is a HOST pointer. The library never allocates
 *     device memory: scratch comes from the caller's workspace, sized by
 *     id_workspace_size().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on it in order; nothing synchronises the host
 *     unless `info` is non-NULL (then the call copies the status back and
 *     waits for the stream).
 *   - Matrices handed in by the user are row-major with a leading dimension
 *     (element (i, j) at A[i*lda + j]), the PyTorch default. The internal
 *     working matrix of id_cpqr / id_solve is column-major (element (i, j) at
 *     X[j*ldx + i]).
 *   - Argument errors return a negative status BEFORE anything is enqueued.
 *     Conditions found on the device (non-finite input, numerical rank below
 *     k) are returned through id_info (and as the return value when `info`
 *     is non-NULL). No entry point aborts or traps.
 *   - Precision: ID_F64 computes in FP64 throughout. ID_F32 stores and
 *     updates the matrix in FP32, keeps the residual column norms and their
 *     downdate in FP64, and solves T = R11^{-1} R12 in FP64.
 */
#ifndef GBID_H
#define GBID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ID_OK = 0,
    ID_RANK_DEFICIENT = 1,   /* |R_jj| <= sqrt(max(m,n)) * eps * |R_00| for some j < k */
    ID_EINVAL = -1,          /* bad size, leading dimension, pointer or option        */
    ID_ENOMEM = -2,          /* workspace smaller than id_workspace_size()            */
    ID_ECUDA = -3,           /* a CUDA launch or copy failed                          */
    ID_ENONFINITE = -4,      /* the input holds Inf or NaN                            */
    ID_ETIMEOUT = -5         /* a bounded device-side wait expired                    */
} id_status;

typedef enum { ID_F64 = 0, ID_F32 = 1 } id_dtype;

typedef struct {
    /* Panel width: number of pivot steps between compact-WY trailing updates.
     * 0 = choose from the shape; nb >= k = left-looking (the trailing matrix is
     * never rewritten; every step corrects its product through the stored
     * reflectors). */
    int32_t nb;
    int32_t reserved[7];
} id_opts;

typedef struct {
    int32_t status;       /* id_status of the device-side checks                 */
    int32_t rank;         /* numerical rank found within the k steps (k if full)  */
    int32_t transposed;   /* 1 when m > n and a row ID was computed               */
    int32_t n_recompute;  /* residual norms recomputed after cancellation         */
    int64_t n_gt2;        /* number of entries with |Z_ij| > 2 (Definition 1)     */
    double  max_abs_z;    /* largest |Z_ij|                                       */
    double  r00;          /* |R_00|, the largest column norm                      */
    int32_t nb;           /* panel width actually used                            */
    int32_t reserved[5];
} id_info;

/* Bytes of device workspace id_decompose needs for this problem (k <= 16384).
 * m, n are the user's matrix dimensions (the m > n route is accounted for).
 * Returns 0 for invalid sizes (k < 1 or k > min(m, n)). */
size_t id_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);

/* id_decompose -- rank-k ID of A (Sec. 2.1; m > n route of the Sec. 2 footnote).
 *
 *   A      [in]  m x n, row-major, leading dimension lda >= n, dtype. Not modified.
 *   k      [in]  target rank, 1 <= k <= min(m, n).
 *   opts   [in]  may be NULL (defaults).
 *   J      [out] k int32: skeleton indices in pivot order (columns of A if
 *                m <= n, rows of A if m > n).
 *   Z      [out] k x nz row-major (nz = n if m <= n, m if m > n), leading
 *                dimension ldz >= nz, dtype. Z[i, J[i]] = 1, Z[i, J[i']] = 0.
 *   work   [in]  device workspace of at least id_workspace_size() bytes,
 *                256-byte aligned; contents are scratch.
 *   info   [out] HOST pointer or NULL. Non-NULL: the call waits for the stream
 *                and returns the device status (ID_OK, ID_RANK_DEFICIENT,
 *                ID_ENONFINITE). NULL: fully asynchronous; read the status later
 *                with id_info_read(work, ...).
 * Returns ID_OK or an id_status. */
int id_decompose(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                 const id_opts* opts, int32_t* J, void* Z, int64_t ldz,
                 void* work, size_t work_bytes, id_info* info, void* stream);

/* id_decompose_host -- the same decomposition for HOST buffers: copies A to
 * the device, runs id_decompose, copies J and Z back and waits. Uses the
 * caller's device workspace `work`, which must also hold the device copies of
 * A, J and Z: size it with id_decompose_host_workspace_size(). */
size_t id_decompose_host_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);
int id_decompose_host(const void* A_host, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                      const id_opts* opts, int32_t* J_host, void* Z_host, int64_t ldz,
                      void* work, size_t work_bytes, id_info* info, void* stream);

/* id_decompose_noalloc -- id_decompose for callers that cannot allocate
 * device memory (for example code running while a global-mode stream capture
 * is active, plug-ins whose host framework owns all device memory, real-time
 * loops that must not take allocator locks). It takes no workspace: the
 * scratch is a fixed array of ID_NOALLOC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library keeps until the process exits. The
 * paper has no counterpart; this is a deployment convenience.
 *
 *   Arguments as for id_decompose, minus work/work_bytes.
 *   Returns ID_ENOMEM, before enqueuing anything, when
 *   id_workspace_size(dtype, m, n, k, opts) > ID_NOALLOC_SCRATCH_BYTES.
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   All calls share the one array: calls that may overlap on the GPU (other
 *   streams, other host threads) race on it and must be serialised by the
 *   caller. Each call re-initialises the state it needs, so the contents left
 *   by an earlier call do not matter. Calls no allocating routine. */
#define ID_NOALLOC_SCRATCH_BYTES (32u << 20)
int id_decompose_noalloc(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                         const id_opts* opts, int32_t* J, void* Z, int64_t ldz, id_info* info, void* stream);

/* Bytes of device workspace id_cpqr needs (its X, perm and tau belong to the
 * caller and are not counted). Returns 0 for invalid arguments. */
size_t id_cpqr_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k, const id_opts* opts);

/* id_cpqr -- k steps of column-pivoted Householder QR of X (Sec. 2.1, stopped
 * after k pivots as proposed in Sec. 4.1), in place.
 *
 *   X     [in/out] m x n COLUMN-major (X[j*ldx + i]), ldx >= m and ldx a
 *                  multiple of 8, with m <= n. On exit: R in the upper triangle
 *                  of rows 0..k-1 (R11 in columns 0..k-1, R12 in columns k..n-1),
 *                  Householder vectors below the diagonal of columns 0..k-1
 *                  (v_0 = 1 implicit). Rows m..ldx-1 are set to zero.
 *   perm  [out] n int32: perm[i] = original index of the column at position i.
 *   tau   [out] k doubles: reflector scalars, H_j = I - tau_j v_j v_j^T.
 *   work  [in]  at least id_cpqr_workspace_size() bytes, 256-byte aligned.
 *   info, stream as for id_decompose.
 * Pivot rule: largest residual 2-norm, ties to the smallest original index. */
int id_cpqr(void* X, id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k,
            const id_opts* opts, int32_t* perm, double* tau,
            void* work, size_t work_bytes, id_info* info, void* stream);

/* id_solve -- T = R11^{-1} R12 by blocked back substitution (Sec. 2.1,
 * equivalent to the normal equations R_k^T R_k Z = C^T A of Eq. final_eq).
 *
 *   X     [in]  factored matrix from id_cpqr (column-major, ldx), n columns.
 *   T     [out] k x (n-k) row-major FP64, leading dimension ldt >= n-k.
 * Computed in FP64 for both dtypes. Returns ID_EINVAL for bad sizes. */
int id_solve(const void* X, id_dtype dtype, int64_t n, int64_t ldx, int64_t k,
             double* T, int64_t ldt, void* stream);

/* id_sketch -- Gaussian row sketch Y = Omega A for the randomized ID.
 *
 * The sketch replaces A by a short matrix with the same column space
 * relations (the randomized route to the skeleton set; Sec. 2.2 takes the
 * randomized step by sampling columns instead). Computed on the tensor cores:
 * A's FP32 values are rounded to BF16 (nearest even) in shared memory,
 * products are accumulated in FP32.
 *
 *   A      [in]  m x n FP32 row-major, lda >= n, lda a multiple of 4, 16-byte aligned.
 *   Omega  [in]  l x m BF16 row-major (uint16 bit patterns), ldo >= m, ldo a
 *                multiple of 8, 16-byte aligned; 1 <= l <= 640.
 *   Y      [out] l x n FP32 row-major, ldy >= n.
 *   work   [in]  id_sketch_workspace_size() bytes of device scratch, 256-byte aligned.
 *   dtype must be ID_F32. info / stream as for id_decompose.
 * Returns ID_OK, ID_EINVAL (sizes, strides, alignment), ID_ENOMEM, ID_ECUDA,
 * or ID_ETIMEOUT (through info) if a bounded device wait expired. */
size_t id_sketch_workspace_size(void);
int id_sketch(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, const uint16_t* Omega_bf16, int64_t l,
              int64_t ldo, float* Y, int64_t ldy, void* work, size_t work_bytes, id_info* info, void* stream);

/* id_decompose_randomized -- randomized rank-k ID of A (m x n, m <= n) from a
 * Gaussian sketch: Y = Omega A (id_sketch, tensor cores), k steps of column-
 * pivoted QR of Y (FP32 matrix, FP64 residual norms), T = R11^{-1} R12 of Y's R
 * in FP64, Z = [I T] P^T. The skeleton J indexes columns of A; Z is the
 * sketched interpolation matrix (Sec. 2.2 computes Z by least squares on A
 * instead; here the sketch's R supplies it).
 *
 *   A      [in]  m x n FP32 row-major, lda >= n, lda a multiple of 4, 16-byte aligned.
 *   Omega  [in]  l x m BF16 row-major, ldo >= m, ldo a multiple of 8, 16-byte
 *                aligned; k <= l <= min(m, 640).
 *   J, Z   [out] as for id_decompose (Z: k x n FP32, ldz >= n).
 *   work   [in]  id_rid_workspace_size(m, n, l, k, opts) bytes, 256-byte aligned.
 *   dtype must be ID_F32. info / stream as for id_decompose. */
size_t id_rid_workspace_size(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts);
int id_decompose_randomized(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda,
                            const uint16_t* Omega_bf16, int64_t l, int64_t ldo, int64_t k, const id_opts* opts,
                            int32_t* J, void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info,
                            void* stream);

/* id_info_read -- copy the device-side status of the last call that used
 * `work` to *info (host) and wait for `stream`. Returns info->status. */
int id_info_read(const void* work, id_info* info, void* stream);

/* Number of kernel launches one id_decompose call enqueues for this problem
 * (memsets excluded). Returns -1 for invalid arguments. */
int64_t id_launch_count(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);

/* Kernel-class tracing. id_trace_enable(capacity > 0) creates `capacity`
 * CUDA event pairs; while enabled, every launch of the traced kernel classes
 * (until the pairs are used up) is bracketed by an event pair recorded on the
 * call's stream. id_trace_enable(0) disables tracing and frees the events.
 * id_trace_read waits for the recorded events, writes per class the summed
 * milliseconds and launch counts into ms[0..nkinds) and launches[0..nkinds)
 * (classes: 0 persistent CPQR, 1 back substitution, 2 sketch, 3 copy-in,
 * 4 Z scatter), clears the records and returns how many were read.
 * Process-wide state; not thread-safe. */
int id_trace_enable(int capacity);
int id_trace_read(double* ms, int64_t* launches, int nkinds);

/* Library version string. */
const char* id_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBID_H */
