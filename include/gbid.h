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
 *     downdate in FP64, and solves T = R11^{-1} R12 in FP64, except where an
 *     entry point states otherwise (the batched form's double-float solve,
 *     the randomized ID's FP32 solve that only seeds its refinement).
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
    /* id_decompose_randomized only: 0 (default) = one least-squares
     * refinement of T against A_J after the sketch (see id_refine); -1 = none
     * (T stays the sketch's R11^{-1} R12). */
    int32_t refine;
    /* id_decompose only: 0 (default) = choose; 1 = the persistent grid-wide
     * CPQR; 2 = one thread-block cluster holding the matrix in distributed
     * shared memory (small problems: k <= 64, min(m, n) <= 1024, the matrix
     * within 8 CTAs' shared memory; ID_EINVAL if it does not fit). */
    int32_t engine;
    /* id_decompose only: how Z is formed from the k pivots. 0 (default) =
     * Z P = [I  R11^{-1} R12], the back substitution with the CPQR's R;
     * 1 = the paper's own route (Sec. 2.1, Eq. final_eq): the normal equations
     * R_k^T R_k Z = C^T A with C = A[:, J], solved in FP64 (as
     * id_decompose_sampled does). Equal in exact arithmetic; the normal
     * equations carry cond(C)^2 instead of cond(C). Column IDs only (m <= n;
     * ID_EINVAL otherwise) and the grid engine (engine 2 is ID_EINVAL). */
    int32_t zsolve;
    int32_t reserved[4];
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
    int32_t refined;      /* 1 when a least-squares refinement was applied to Z   */
    int32_t engine;       /* 1 persistent grid CPQR, 2 cluster, 3 batched kernel  */
    int32_t reserved0;
    /* ||A - C Z||_F / ||A||_F of a deterministic ID, from the CPQR's residual
     * column norms: with Z P = [I R11^{-1} R12] the residual is Q2 R22
     * (Sec. 2.1), whose Frobenius norm is that of the columns left after k
     * steps. Filled by id_decompose on the grid engine and by id_decompose_csr
     * (relative accuracy about that of the norm downdate, ~1e-6); 0 for an ID
     * of a k x k matrix; -1 where it is not computed. */
    double  err_est;
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
 *   Arguments as for id_decompose, minus work/work_bytes. `info` must be
 *   NULL when the call is enqueued into a stream that is being captured (a
 *   non-NULL info makes the call wait for the stream, which capture forbids).
 *   Returns ID_ENOMEM, before enqueuing anything, when
 *   id_workspace_size(dtype, m, n, k, opts) > ID_NOALLOC_SCRATCH_BYTES.
 *   Every option of id_decompose is taken (the normal-equation route's
 *   products are the library's own kernels and allocate nothing).
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

/* id_cpqr_residual_norms -- after id_cpqr with the same arguments and work:
 * out[i] (n doubles, device) = the residual 2-norm of the column at position
 * i >= k after the k steps, ||X(k:m, i)|| of the updated matrix (the norms the
 * pivot rule compares, kept in FP64 by the CPQR's downdate with exact
 * recomputes); out[i] for i < k is the residual norm column i had when step i
 * chose it (|R_ii| in exact arithmetic). The root sum of squares over i >= k
 * is ||R22||_F, the ID's residual (Sec. 2.1). One stream-ordered kernel (the
 * workspace keeps the squared norms; out gets their square roots); returns
 * ID_EINVAL for bad arguments. */
int id_cpqr_residual_norms(const void* work, id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k,
                           const id_opts* opts, double* out, void* stream);

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
 *   work   [in]  id_sketch_workspace_size() bytes of device scratch, 256-byte aligned;
 *                with id_sketch_scratch_size(n, l) bytes more, a short last wave of
 *                column tiles is split along m (the sum of the slices taken in slice
 *                order), as id_decompose_randomized does: then Y is bit-identical to
 *                the sketch inside id_decompose_randomized on the same device.
 *   dtype must be ID_F32. info / stream as for id_decompose.
 * Returns ID_OK, ID_EINVAL (sizes, strides, alignment), ID_ENOMEM, ID_ECUDA,
 * or ID_ETIMEOUT (through info) if a bounded device wait expired. */
size_t id_sketch_workspace_size(void);
/* Extra workspace bytes for the split of the last wave (0: no split for these sizes
 * on the current device; the library must have been initialised on it, e.g. by an
 * earlier call, for the device's SM count to be known). */
size_t id_sketch_scratch_size(int64_t n, int64_t l);
int id_sketch(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, const uint16_t* Omega_bf16, int64_t l,
              int64_t ldo, float* Y, int64_t ldy, void* work, size_t work_bytes, id_info* info, void* stream);

/* id_decompose_randomized -- randomized rank-k ID of A (m x n, m <= n) from a
 * Gaussian sketch: Y = Omega A (id_sketch, tensor cores), k steps of column-
 * pivoted QR of Y (FP32 matrix, FP64 residual norms), T = R11^{-1} R12 of Y's R,
 * Z = [I T] P^T. The skeleton J indexes columns of A. By default
 * (opts->refine = 0) T is solved in FP32 and Z is then refined once against A
 * (id_refine): the least-squares Z for J that Sec. 2.2 asks for.
 * opts->refine = -1 keeps the sketch's Z, with T solved in FP64.
 *
 *   A      [in]  m x n FP32 row-major, n <= lda < 2^31, lda a multiple of 4, 16-byte aligned.
 *   Omega  [in]  l x m BF16 row-major, ldo >= m, ldo a multiple of 8, 16-byte
 *                aligned; k <= l <= min(m, 640).
 *   J, Z   [out] as for id_decompose (Z: k x n FP32, n <= ldz < 2^31).
 *   work   [in]  id_rid_workspace_size(m, n, l, k, opts) bytes, 256-byte aligned.
 *   dtype must be ID_F32. info / stream as for id_decompose. */
size_t id_rid_workspace_size(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts);
int id_decompose_randomized(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda,
                            const uint16_t* Omega_bf16, int64_t l, int64_t ldo, int64_t k, const id_opts* opts,
                            int32_t* J, void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info,
                            void* stream);

/* id_rid_pipe -- randomized IDs (Sec. 2.2) of a stream of HOST matrices of one
 * size, for serving: consecutive IDs overlap, so that the host-to-device copy of
 * ID i+1's inputs and the device-to-host copy of ID i-1's outputs run while ID i
 * runs on the caller's stream. Each submitted ID is id_decompose_randomized on
 * device copies of its inputs: the same J, Z and id_info, bit for bit.
 *
 * The pipe keeps two device slots (A, Omega, J, Z and the status of one ID each)
 * and one randomized workspace, all carved from the caller's DEVICE buffer; it
 * creates two streams (one per copy direction) and six events on the current
 * device, its only resources. The copy into a slot waits for the compute of the
 * ID that last used it; the compute of an ID waits for its inputs and for the
 * copy-out of that slot's previous outputs.
 *
 * id_rid_pipe_workspace_size(m, n, l, k, opts): bytes of `work` (0 for sizes
 *   id_decompose_randomized rejects).
 * id_rid_pipe_create(&pipe, m, n, l, k, opts, work, work_bytes): work 256-byte
 *   aligned, at least the size above; opts (may be NULL) is copied. Returns
 *   ID_OK, ID_EINVAL, ID_ENOMEM (work too small) or ID_ECUDA.
 * id_rid_pipe_submit(pipe, A_host, lda, Omega_host, ldo, J_host, Z_host, ldz,
 *   info_host, stream): enqueues one ID and returns without waiting. A_host: m x n
 *   FP32 row-major, lda >= n; Omega_host: l x m BF16 row-major, ldo >= m; J_host:
 *   k int32; Z_host: k x n FP32 row-major, ldz >= n; info_host: an id_info that
 *   receives the ID's status, or NULL. All host buffers should be pinned
 *   (pageable ones make the copies synchronous); inputs must stay unchanged and
 *   outputs unread until id_rid_pipe_sync returns. Consecutive submits must use
 *   the same stream. Returns ID_OK, ID_EINVAL or ID_ECUDA (the ID's own status
 *   arrives in *info_host).
 * id_rid_pipe_sync(pipe): waits until every submitted ID's outputs are on the
 *   host. Returns ID_OK or ID_ECUDA.
 * id_rid_pipe_destroy(pipe): waits as id_rid_pipe_sync, then releases the
 *   streams and events (the caller frees `work`). NULL is ignored. */
typedef struct id_rid_pipe id_rid_pipe;
size_t id_rid_pipe_workspace_size(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts);
int id_rid_pipe_create(id_rid_pipe** pipe, int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts,
                       void* work, size_t work_bytes);
int id_rid_pipe_submit(id_rid_pipe* pipe, const float* A_host, int64_t lda, const uint16_t* Omega_host, int64_t ldo,
                       int32_t* J_host, float* Z_host, int64_t ldz, id_info* info_host, void* stream);
int id_rid_pipe_sync(id_rid_pipe* pipe);
void id_rid_pipe_destroy(id_rid_pipe* pipe);

/* id_decompose_sampled -- the paper's randomized algorithm, Optim RID
 * (Sec. 2.2): sample p columns of A without replacement (the sample is an
 * input: the caller draws it; the paper takes p = k + floor(0.2 k)), run the
 * column-pivoted QR on A_S = A[:, idx] for k steps, take J = idx[P_k] and
 * C = A[:, J], and solve the normal equations R_k^T R_k Z = C^T A
 * (Eq. final_eq) for Z against ALL of A, in FP64.
 *   A    [in]  m x n row-major, n <= lda < 2^31, dtype (not modified).
 *   idx  [in]  HOST array of p distinct column indices in [0, n); k <= p <= n.
 *   J    [out] k skeleton columns of A in pivot order; Z [out] k x n
 *              (n <= ldz < 2^31).
 *   work [in]  id_sampled_workspace_size() bytes, 256-byte aligned.
 * FP64 data solve with the CPQR's own R_k (the paper's route). FP32 data: the
 * CPQR runs in FP32, whose R_k the normal equations would square, so the
 * factor is rebuilt from C (C^T C from exact products with double-float sums,
 * FP64 Cholesky) -- the same matrix in exact arithmetic. Z[:, J] = I exactly.
 * When R_k is numerically singular (the paper switches to a
 * symmetric-indefinite solve there) the status is ID_RANK_DEFICIENT, `rank`
 * is the CPQR's numerical rank and Z is not reliable: call again with
 * k <= rank. Returns as id_decompose. */
size_t id_sampled_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t p, int64_t k, const id_opts* opts);
int id_decompose_sampled(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, const int32_t* idx,
                         int64_t p, int64_t k, const id_opts* opts, int32_t* J, void* Z, int64_t ldz, void* work,
                         size_t work_bytes, id_info* info, void* stream);

/* id_refine -- one least-squares refinement of an ID's interpolation matrix
 * against A (the LS problem of Sec. 2.1, min ||A - C Z||_F with C = A[:, J]):
 *     Z <- Z + (C^T C)^{-1} C^T (A - C Z),   Z[:, J] kept = I.
 * For the randomized ID the skeleton J and the first Z come from the sketch;
 * one step lands on the least-squares Z for that J up to rounding (the
 * problem is linear), which is the Z Sec. 2.2 asks for.
 * Arithmetic: C^T C in FP64 (products of FP32 values are exact in FP64) and
 * its Cholesky factor U in FP64; U^{-1} in FP64, applied in FP32; the
 * residual A - C Z and C^T times it as FP32-accurate 3xTF32 products on the
 * tensor cores (the library's own tcgen05 kernel, see id_gemm), by column
 * blocks of A whose residual stays in L2.
 *   A     [in]     m x n FP32 row-major, n <= lda < 2^31, m <= n (a column ID).
 *   J     [in]     k skeleton columns (distinct, in [0, n)).
 *   Z     [in,out] k x n FP32 row-major, n <= ldz < 2^31; Z[:, J] = I on entry.
 *   work  [in]     id_refine_workspace_size() bytes, 256-byte aligned.
 *   info  [out]    HOST pointer or NULL (as for id_decompose): status ID_OK,
 *                  refined = 1, and the Z statistics after the update. If
 *                  C^T C is not numerically positive definite (rank(C) < k)
 *                  Z is left unchanged and refined = 0.
 * dtype must be ID_F32 (an FP64 ID's T = R11^{-1} R12 already solves the LS
 * problem to FP64 accuracy). */
size_t id_refine_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k);
int id_refine(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J,
              void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info, void* stream);

/* id_backward -- gradient of a scalar loss L(Z) through the ID with the
 * skeleton J held fixed (the differentiable form of Sec. 2.1's least-squares
 * Z; the paper itself differentiates nothing):
 *   Z[:, J] = I is constant, Z[:, rest] = T = C^+ B, C = A[:, J], B = A[:, rest];
 *   with W = (C^T C)^{-1} dZ[:, rest]:
 *   dA[:, rest] = C W,   dA[:, J] = (B - C T) W^T - C W T^T.
 *   A   [in]  m x n FP32 row-major (m <= n), n <= lda < 2^31 (ldz, lddz, ldda too).
 *   J   [in]  k skeleton columns; Z [in] k x n FP32 (ldz >= n), the ID's Z for J.
 *   dZ  [in]  k x n FP32 (lddz >= n): dL/dZ (its columns at J are ignored).
 *   dA  [out] m x n FP32 (ldda >= n): dL/dA.
 *   work [in] id_backward_workspace_size() bytes, 256-byte aligned.
 * W is formed in FP64 (C^T C by exact products and double-float sums, its
 * FP64 Cholesky factor applied twice), the products with C, A - C Z and Z as
 * FP32-accurate GEMMs. info (HOST or NULL): ID_OK, ID_RANK_DEFICIENT if C^T C
 * is not numerically positive definite (dA is then meaningless), ID_EINVAL
 * for a J entry outside [0, n). dtype must be ID_F32. */
size_t id_backward_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k);
int id_backward(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J,
                const void* Z, int64_t ldz, const void* dZ, int64_t lddz, void* dA, int64_t ldda, void* work,
                size_t work_bytes, id_info* info, void* stream);

/* ---------------------------------------------------------------- batched --
 * id_decompose_batched -- rank-k IDs of many independent small matrices, of
 * uneven sizes, in ONE persistent launch (Sec. 2.1 for each matrix, with the
 * m > n route of the Sec. 2 footnote per matrix). The paper's use case of
 * many small IDs (a hierarchical compression) has no batched form in the
 * paper itself; the arithmetic per matrix is that of id_decompose:
 * Householder CPQR stopped after k pivots (residual norms taken exactly every
 * step, ties to the smallest original index), T = R11^{-1} R12 by back
 * substitution in FP64 (FP64 data) or in double-float arithmetic of about 48
 * significant bits (FP32 data).
 *
 *   problems   [in]  DEVICE array of `count` id_problem descriptors, read by
 *                    the kernel (so the call can be captured in a CUDA graph
 *                    and replayed with the same descriptors).
 *   dtype      [in]  element type of every A and Z.
 *   batch_work [in]  DEVICE scratch of ID_BATCHED_WORK_BYTES (the work queue).
 *   infos      [out] DEVICE array of `count` id_info, one per problem. A
 *                    descriptor that breaks a rule below gets status ID_EINVAL
 *                    there; the other problems are still decomposed.
 * Per problem: 1 <= k <= min(m, n), k <= ID_BATCHED_MAX_K,
 * min(m, n) <= ID_BATCHED_MAX_MIN_DIM, lda >= n, ldz >= max(m, n), and `work`
 * 256-byte aligned with id_batched_problem_workspace_size() bytes. A is read
 * only; J (k int32) and Z (k x max(m, n), row-major) are as for id_decompose.
 * Nothing is waited for; the call returns after enqueuing a 4-byte memset and
 * one kernel. Returns ID_OK, ID_EINVAL (bad dtype, count < 0, NULL pointer),
 * ID_ENOMEM (batch_work too small) or ID_ECUDA. count == 0 enqueues nothing.
 * The paper has no batched entry point; this one is the library's own. */
#define ID_BATCHED_MAX_K 64
#define ID_BATCHED_MAX_MIN_DIM 1024
#define ID_BATCHED_WORK_BYTES 256
typedef struct {
    const void* A;   /* m x n, row-major, leading dimension lda            */
    int64_t m, n, lda, k;
    int32_t* J;      /* k                                                   */
    void* Z;         /* k x max(m, n), row-major, leading dimension ldz     */
    int64_t ldz;
    void* work;      /* id_batched_problem_workspace_size() bytes, scratch  */
} id_problem;
size_t id_batched_problem_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k);
int id_decompose_batched(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                         size_t batch_work_bytes, id_info* infos, void* stream);

/* Tile shapes of the batched kernel and their tuner. The kernel is built in
 * several instances; each performs the same floating-point operations in the
 * same order on every element, so all of them return bit-identical J, Z and
 * id_info (up to the sign of zero entries) and differ only in speed.
 *
 * id_batched_config_count -- number of instances for dtype (0: bad dtype).
 * id_batched_config_get   -- *out = instance `index` (0 is the default that
 *                            id_decompose_batched uses); ID_EINVAL for a bad
 *                            dtype, index or NULL out.
 * id_decompose_batched_with -- id_decompose_batched with instance `config`
 *                            (same arguments and rules; ID_EINVAL for a bad
 *                            config index). Enqueues only; graph-capturable.
 * id_batched_autotune     -- times every instance on this batch: per instance
 *                            one untimed launch, then `reps` (1..1000) launches
 *                            between two events on `stream`; ms_out (HOST,
 *                            config_count floats, or NULL) receives the mean
 *                            ms per launch and *best (HOST) the fastest index.
 *                            WAITS for the stream (not capturable). J, Z and
 *                            infos then hold the batch's results (any
 *                            instance's: they are identical). Returns ID_OK,
 *                            ID_EINVAL (as above, or best NULL, reps out of
 *                            range), ID_ENOMEM or ID_ECUDA. count == 0: *best
 *                            = 0, nothing launched. */
typedef struct {
    int32_t threads;        /* threads per CTA                                      */
    int32_t cols_per_warp;  /* trailing columns a warp updates per pass             */
    int32_t rows_per_lane;  /* rows a lane holds per pass: column segments of up to
                               32 x this rows stay in registers (64 x this with half
                               the columns), longer ones take two passes             */
    int32_t ctas_per_sm;    /* resident CTAs per SM the register budget is cut for  */
} id_batched_config;
int id_batched_config_count(id_dtype dtype);
int id_batched_config_get(id_dtype dtype, int index, id_batched_config* out);
int id_decompose_batched_with(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                              size_t batch_work_bytes, id_info* infos, int config, void* stream);
int id_batched_autotune(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                        size_t batch_work_bytes, id_info* infos, int reps, float* ms_out, int* best, void* stream);

/* id_info_read -- copy the device-side status of the last call that used
 * `work` to *info (host) and wait for `stream`. Returns info->status. */
int id_info_read(const void* work, id_info* info, void* stream);

/* id_selftest_bounded_wait -- runs the library's bounded device wait (the
 * primitive behind every grid barrier of the CPQR kernel) on a counter that
 * nothing increments: the wait must give up after its poll limit (2^22
 * polls, a few seconds) and report a timeout instead of hanging, leaving the
 * context usable. work: DEVICE scratch of ID_SELFTEST_WORK_BYTES, 256-byte
 * aligned. *status (HOST) receives ID_ETIMEOUT when the wait gave up as
 * designed (ID_OK would mean it did not). WAITS for the stream. Returns
 * ID_OK, ID_EINVAL (NULL pointer, small or misaligned work) or ID_ECUDA.
 * Failure detection of the library's own making; the paper has none. */
/* id_cpqr_timeline -- a diagnostic of the persistent CPQR kernel: while set
 * (steps > 0), every CPQR launch has its first CTA stamp the GPU's nanosecond
 * timer at the phase boundaries of each pivot step j < steps into
 * buf[8 j + q] (DEVICE memory the caller owns, 8 * steps int64):
 *   q = 0 step start, 1 pivot known, 2 pivot column and its norm formed,
 *   3 reflector and aux ready (the trailing product starts), 4 trailing
 *   product done, 5 after the step's last grid barrier; 6 and 7 unused.
 * id_cpqr_timeline(NULL, 0) switches it off. Not thread-safe; the paper has
 * no counterpart. Returns ID_OK or ID_EINVAL. */
int id_cpqr_timeline(long long* buf, int steps);

#define ID_SELFTEST_WORK_BYTES 4096
int id_selftest_bounded_wait(void* work, size_t work_bytes, int* status, void* stream);

/* Number of kernel launches one id_decompose call enqueues for this problem
 * (memsets excluded). Returns -1 for invalid arguments. */
int64_t id_launch_count(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);
/* The same for one id_decompose_randomized call (sketch, CPQR of the l x n
 * sketch, solve, Z, and the refinement unless opts->refine < 0). */
int64_t id_rid_launch_count(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts);

/* id_reconstruct -- the ID's approximation of A (the `approx = C @ Z` that
 * the paper's listings return with the skeleton and Z, Sec. 2.1):
 *   transposed = 0 (column ID, Z k x n): Out = A[:, J] Z   (m x n);
 *   transposed = 1 (row ID of an m > n matrix, Z k x m): Out = Z^T A[J, :].
 *   A    [in]  m x n row-major, n <= lda < 2^31, dtype (not modified).
 *   J    [in]  k indices (columns of A, or rows when transposed).
 *   Z    [in]  k x n (k x m when transposed) row-major, ldz >= that width, < 2^31.
 *   Out  [out] m x n row-major, n <= ldo < 2^31.
 *   work [in]  id_reconstruct_workspace_size() bytes, 256-byte aligned.
 * The skeleton is gathered, then one product (id_gemm's): FP64 data in
 * FP64, FP32 data in FP32-accurate 3xTF32 products on the tensor cores. info (HOST or NULL): status ID_EINVAL if a J entry is out of range
 * (Out is then unspecified), else ID_OK. */
size_t id_reconstruct_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, int32_t transposed);
int id_reconstruct(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J,
                   const void* Z, int64_t ldz, int32_t transposed, void* Out, int64_t ldo, void* work,
                   size_t work_bytes, id_info* info, void* stream);

/* id_gemm -- C = alpha op(A) op(B) + beta C for row-major DEVICE matrices,
 * op(X) = X (flag 0) or X^T (flag 1): the matrix product behind the
 * refinement (the least-squares Z of Sec. 2.2), the gradient and
 * id_reconstruct (Listing 1's approx = C @ Z), exposed for callers and tests.
 *   ID_F64: FP64 arithmetic on the FP64 pipe.
 *   ID_F32: FP32-accurate products on the tensor cores by the 3xTF32 split
 *           (x = hi + lo, hi rounded to TF32; lo_a hi_b + hi_a lo_b +
 *           hi_a hi_b accumulated in FP32 in tensor memory): an entry's
 *           error is about 2^-21 of sum_k |a_ik| |b_kj| (FP32 itself: 2^-24
 *           per operation).
 *   M, N, K in [1, 2^31); lda, ldb, ldc at least the row widths they hold
 *   (op(A) is M x K, op(B) K x N, C M x N). beta = 0: C is not read.
 *   work [in] id_gemm_workspace_size() bytes, 256-byte aligned.
 *   info (HOST or NULL): non-NULL waits and returns ID_ETIMEOUT if a bounded
 *   device wait of the tensor-core kernel expired, else ID_OK. */
size_t id_gemm_workspace_size(id_dtype dtype, int64_t M, int64_t N, int64_t K);
int id_gemm(id_dtype dtype, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K, double alpha, const void* A,
            int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, void* work, size_t work_bytes,
            id_info* info, void* stream);

/* id_decompose_csr -- rank-k ID (as id_decompose) of a sparse A given in CSR
 * form, for inputs such as the sparse matrices of the paper's experiments
 * (Sec. 3): the skeleton C = A[:, J] keeps A's sparsity (Sec. 1.2). A is
 * formed directly in the dense working layout (no dense copy of A), then the
 * same CPQR, back substitution and Z assembly run on the grid engine.
 *   rowptr [in] m + 1 int64 offsets (device), nondecreasing, rowptr[m] <= nnz.
 *   colind [in] nnz int32 column indices in [0, n) (device); values [in] nnz
 *               entries of dtype (device). Duplicate (row, column) entries
 *               are summed, in an unspecified order.
 *   J, Z   [out] as for id_decompose (m > n gives a row ID).
 *   work   [in]  id_csr_workspace_size() bytes, 256-byte aligned.
 *   opts   nb as for id_decompose; engine 2 or zsolve != 0 is ID_EINVAL.
 * A malformed rowptr or column index is found on the device: the status
 * (through info) is ID_EINVAL and J, Z are unspecified. */
size_t id_csr_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);
int id_decompose_csr(const int64_t* rowptr, const int32_t* colind, const void* values, id_dtype dtype, int64_t m,
                     int64_t n, int64_t nnz, int64_t k, const id_opts* opts, int32_t* J, void* Z, int64_t ldz,
                     void* work, size_t work_bytes, id_info* info, void* stream);

/* id_decompose_two_sided -- rank-k two-sided ID A ~= X^T A[I, J] Z, the
 * variant (Cheng et al.) that the footnote of Sec. 1.2 names. For m <= n:
 * the column ID (J, Z) of A (Sec. 2.1), then the row ID (I, X) of the
 * skeleton C = A[:, J] (the m > n route of the Sec. 2 footnote on an m x k
 * matrix). For m > n the roles swap: the row ID (I, X) of A, then the
 * column ID (J, Z) of R = A[I, :]. A stage on a k x k matrix keeps all rows
 * (columns): the identity. In exact arithmetic the second stage adds no
 * error (X^T C[I, :] = C for a rank-k C).
 *   A    [in]  m x n row-major, lda >= n, dtype (not modified).
 *   I    [out] k row indices; X [out] k x m row-major (ldx >= m), X[:, I] = I.
 *   J    [out] k column indices; Z [out] k x n row-major (ldz >= n), Z[:, J] = I.
 *   opts       stage 1's options (nb, engine; zsolve must be 0); stage 2 uses defaults.
 *   work [in]  id_two_sided_workspace_size() bytes, 256-byte aligned.
 *   info [out] HOST array of TWO id_info (stage 1, then stage 2), or NULL.
 * Returns as id_decompose; with info, the first non-OK stage status. */
size_t id_two_sided_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts);
int id_decompose_two_sided(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                           const id_opts* opts, int32_t* I, int32_t* J, void* X, int64_t ldx, void* Z, int64_t ldz,
                           void* work, size_t work_bytes, id_info* info, void* stream);

/* Kernel-class tracing. id_trace_enable(capacity > 0) creates `capacity`
 * CUDA event pairs; while enabled, every launch of the traced kernel classes
 * (until the pairs are used up) is bracketed by an event pair recorded on the
 * call's stream. id_trace_enable(0) disables tracing and frees the events.
 * id_trace_read waits for the recorded events, writes per class the summed
 * milliseconds and launch counts into ms[0..nkinds) and launches[0..nkinds)
 * (classes: 0 persistent CPQR, 1 back substitution, 2 sketch, 3 copy-in,
 * 4 Z scatter, 5 batched ID, 6 least-squares refinement and gradient, 7 the
 * normal-equation Z of the column-sampling RID), clears the records and
 * returns how many were read.
 * Process-wide state; not thread-safe. */
int id_trace_enable(int capacity);
int id_trace_read(double* ms, int64_t* launches, int nkinds);

/* Library version string. */
const char* id_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBID_H */
