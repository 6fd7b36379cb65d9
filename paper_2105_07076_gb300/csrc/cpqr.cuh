// Internal interface of the CPQR kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbid {

constexpr int kMaxPanel = 512;                  // largest panel width nb

// Device buffers and sizes of one truncated CPQR. The working matrix is
// m x n column-major (m <= n), leading dimension ldw (multiple of 8).
struct CpqrPlan {
    int m, n, ldw, k, nb;
    int64_t m_user, n_user;   // the caller's dimensions (for the rank tolerance)
    void* W;                  // m x n working matrix (T)
    void* F;                  // n x ldf row-major panel factor (T)
    int ldf;
    void* xbuf;               // ldw: pivot column after the lazy update (T)
    double* ssq;              // kMaxParts partial sums of squares
    void* sync;               // sync_bytes(k): barrier counter and per-step aux counters
    double* vn1;              // n: residual norm estimates
    double* vn2;              // n: norms at the last exact computation
    int* perm;                // n
    double* tau;              // k
    ArgMax* part3;            // kMaxParts argmax partials of the previous step
    void* aux;                // kMaxPanel (T)
    State* st;
    void* wy_ws;              // FP32 with nb < k: wy_bytes(m, n, nb) of operand scratch for the
                              // tensor-core compact-WY update between panels (nullptr: in-kernel update)
};

// Operand scratch of the FP32 compact-WY update W_trail -= V F^T (3xTF32 on
// the tensor cores): V and F in split operand form.
size_t wy_bytes(int m, int n, int nb);

// Bytes of the zero-initialised synchronisation area of one CPQR: a 64-byte
// grid-barrier slot and k per-step aux counters.
inline size_t sync_bytes(int k) { return 64 + 4 * (size_t)k; }

template <typename T> cudaError_t cpqr_configure();
template <typename T> cudaError_t copy_in(const void* A, int64_t lda, int trans, const CpqrPlan& P, cudaStream_t s);
template <typename T> cudaError_t zero_pad(const CpqrPlan& P, cudaStream_t s);
// CSR input into the (zeroed) working matrix; bad input sets kStatBadInput in *status.
template <typename T>
cudaError_t csr_in(const int64_t* rowptr, const int32_t* colind, const void* vals, int64_t m, int64_t n, int64_t nnz,
                   int trans, const CpqrPlan& P, int* status, cudaStream_t s);
template <typename T> cudaError_t cpqr_run(const CpqrPlan& P, cudaStream_t s);
template <typename T> int cpqr_grid(int m, int nb);   // CTAs of the cooperative launch (0: cannot launch)
bool cpqr_short_rows(int m);   // FP32 matrices with this many rows (and panels of at most 32) take the short kernel

// Back substitution T = R11^{-1} R12 (FP64) and Z assembly.
// T = R11^{-1} R12 (FP64 arithmetic; FP32 when fp32_arith and T = float, for a
// T that only seeds a least-squares refinement).
template <typename T>
cudaError_t solve_run(const void* W, int ldw, int k, int n, double* Tm, int ldt, cudaStream_t s,
                      bool fp32_arith = false);
template <typename T> cudaError_t scatter_z(const int* perm, const double* Tm, int ldt, int k, int n, void* Z,
                                            int64_t ldz, int32_t* J, DevInfo* info, cudaStream_t s);
cudaError_t solve_configure();

// Y = Omega A on tcgen05 tensor cores (sketch.cu). Returns an id_status.
cudaError_t sketch_configure();
// scratch (optional, 16-byte aligned): room for the K slices of a short last
// wave of column tiles (sketch_scratch_bytes); without it no tile is split.
int sketch_run(const float* A, int64_t m, int64_t n, int64_t lda, const uint16_t* Om, int64_t l, int64_t ldo, float* Y,
               int64_t ldy, int* status, cudaStream_t s, float* scratch = nullptr, size_t scratch_bytes = 0);
size_t sketch_scratch_bytes(int64_t n, int64_t l);
int sketch_launch_count(int64_t n, int64_t l, size_t scratch_bytes);
cudaError_t finalize_info(const State* st, DevInfo* info, int k, int transposed, int nb, cudaStream_t s,
                          const int* extra_status = nullptr);
// info->err_est from the CPQR's residual column norms (after finalize_info).
cudaError_t error_estimate(const double* vn1, int k, int n, const State* st, DevInfo* info, cudaStream_t s);
// out[0:n] = the residual norms from the CPQR workspace's squared norms vn1.
cudaError_t norms_from_squares(const double* vn1, double* out, int n, cudaStream_t s);

// One least-squares refinement of Z against A (refine.cu). Returns an id_status;
// updates info->info.refined and the Z statistics.
size_t refine_bytes(int64_t m, int64_t n, int64_t k);
int64_t refine_launch_count(int64_t m, int64_t n, int64_t k);
cudaError_t refine_info_init(DevInfo* dinfo, int k, cudaStream_t s);   // status ID_OK, rank k, statistics zero
int refine_run(const float* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, float* Z, int64_t ldz,
               void* ws, DevInfo* dinfo, cudaStream_t s);

// Small IDs on one thread-block cluster (cluster.cu): the cluster size a
// problem gets (0 if it does not fit) and the launch (+ statistics kernel).
template <typename T> int cluster_size(int64_t m, int64_t n, int64_t k);
template <typename T>
cudaError_t cluster_run(const void* A, int64_t lda, int trans, int mx, int nx, int k, int32_t* J, void* Z,
                        int64_t ldz, DevInfo* dinfo, cudaStream_t s);

// Column-sampling Optim RID pieces (refine.cu): W <- A[:, idx]; J = idx[perm];
// Z from the normal equations in FP64 (an id_status).
template <typename T>
cudaError_t sample_gather_run(const void* A, int64_t lda, int m, const int32_t* idx, int p, void* W, int ldw,
                              cudaStream_t s);
cudaError_t sample_map_j(const int* perm, const int32_t* idx, int k, int32_t* J, cudaStream_t s);
size_t sampled_z_bytes(int64_t m, int64_t n, int64_t k);
// Two-sided ID pieces (refine.cu): S = A[:, idx] (rows = 0) or A[idx, :]
// (rows = 1); the ID of a k x k matrix (idx = 0..k-1, Z = I).
template <typename T>
cudaError_t gather_skeleton(const void* A, int64_t lda, int64_t m, int64_t n, int k, const int32_t* idx, int rows,
                            void* S, int* flag, cudaStream_t s);
template <typename T>
cudaError_t identity_id(int32_t* idx, void* Zx, int64_t ldz, int k, DevInfo* info, cudaStream_t s);
// The ID's approximation A[:, J] Z (rows = 0) or Z^T A[J, :] (rows = 1), refine.cu.
size_t reconstruct_bytes(int64_t m, int64_t n, int64_t k, int rows, size_t elem);
template <typename T>
int reconstruct_run(const void* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const void* Z,
                    int64_t ldz, int rows, void* Out, int64_t ldo, void* ws, DevInfo* dinfo, cudaStream_t s);
template <typename T>
int sampled_z_run(const void* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const void* W, int ldw,
                  void* Z, int64_t ldz, void* ws, DevInfo* dinfo, cudaStream_t s);

// Gradient through the ID with the skeleton frozen (refine.cu). Returns an id_status.
size_t backward_bytes(int64_t m, int64_t n, int64_t k);
int backward_run(const float* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const float* Z,
                 int64_t ldz, const float* dZ, int64_t lddz, float* dA, int64_t ldda, void* ws, DevInfo* dinfo,
                 cudaStream_t s);

}  // namespace gbid
