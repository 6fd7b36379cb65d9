// Matrix products of the library (gemm.cu), written for sm_103a.
//
// FP32 data: FP32-accurate products on the 5th-generation tensor cores by the
// 3xTF32 split. Every operand x is stored as hi + lo, hi = x rounded to TF32
// (the low 13 mantissa bits cleared) and lo = x - hi (exact in FP32); a
// product is accumulated as lo_a hi_b + hi_a lo_b + hi_a hi_b in FP32 in
// tensor memory (tcgen05.mma kind::tf32), which drops only lo_a lo_b
// (below 2^-22 of |a b|) and the TF32 rounding of the lo parts.
//
// FP64 data: a register-tiled SIMT product on the FP64 pipe.
//
// Operand convention of the tensor-core product: D (M x N) = sum_k A(i, k)
// B(j, k) over k, with A (M x Kp) and B (N x Kp) row-major ("K-major", the
// operand layout the tensor cores read), split into hi/lo arrays with Kp a
// multiple of 16 and zero beyond the true K. split_tf32 builds such operands
// from any row-major matrix or its transpose.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbid {

// One split operand: rows x Kp, element (r, c) at hi[r * ld + c] (and lo).
struct TfOperand {
    const float* hi;
    const float* lo;
    int64_t ld;    // elements, a multiple of 4 (16-byte rows for TMA)
    int rows;      // rows beyond this read as zero
};

// dst(r, c), r < rows, c < Kp: src(r, c) when c < cols, else 0, split into hi/lo.
// trans = 0: src(r, c) = S[r * lds + c]; trans = 1: src(r, c) = S[c * lds + r].
// S is float or double (a double is rounded to FP32 first).
template <typename S>
cudaError_t split_tf32(const S* src, int64_t lds, int trans, int rows, int cols, int Kp, float* hi, float* lo,
                       int64_t ldo, cudaStream_t s);

// Epilogue of the tensor-core product: value(i, j) = alpha acc(i, j) + beta cin(i, j).
struct TfEpilogue {
    float alpha = 1.0f, beta = 0.0f;
    const float* cin = nullptr;   // nullptr: no addend
    int64_t ldc = 0;
    int cin_trans = 0;            // 0: cin[i * ldc + j]; 1: cin[j * ldc + i]
    int cin_cols = 0x7fffffff;    // cin(i, j) read only for j < cin_cols (0 beyond)
    float* d = nullptr;           // value (or its hi part when d_lo is set)
    float* d_lo = nullptr;        // split output: lo part of value
    int64_t ldd = 0;
    int d_trans = 0;              // 0: d[i * ldd + j]; 1: d[j * ldd + i]
    int64_t z_stride = 0;         // split-K: slice z writes at d + z * z_stride (no addend)
    const int* skip = nullptr;    // non-null and *skip != 0: nothing is written
};

// D = epilogue(A B^T) for A (M x Kp), B (N x Kp); the K range [0, K) (K a
// multiple of 16) is split into `splits` slices of whole 16-column blocks.
// status: device word, kStatTimeout is OR-ed in if a bounded wait expires.
// Returns an id_status (ID_EINVAL for unsupported shapes or alignment).
int gemm_tf32x3(const TfOperand& A, const TfOperand& B, int M, int N, int K, int splits, const TfEpilogue& ep,
                int* status, cudaStream_t s);
cudaError_t gemm_configure();

// Row-major FP64 product: C (M x N) = alpha op(A) op(B) + beta C, op(X) = X
// (ta = 0) or X^T (ta = 1), leading dimensions in elements.
cudaError_t dgemm(int ta, int tb, int M, int N, int K, double alpha, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s);

// batch row-major FP64 products C_z = alpha A_z B_z + beta C_z with
// X_z = X + z * sx (no transposes), on 16 x 16 tiles: small products that
// still spread over every SM.
cudaError_t dgemm_batched(int M, int N, int K, double alpha, const double* A, int64_t lda, int64_t sa,
                          const double* B, int64_t ldb, int64_t sb, double beta, double* C, int64_t ldc, int64_t sc,
                          int batch, cudaStream_t s);

// Row-major FP32-accurate product through the tensor cores, same semantics as
// dgemm (FP32 data). ws: scratch of gemm_f32_bytes(M, N, K) bytes.
size_t gemm_f32_bytes(int M, int N, int K);
int gemm_f32(int ta, int tb, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
             int64_t ldb, float beta, float* C, int64_t ldc, void* ws, int* status, cudaStream_t s);
// The same with the addend read from Cin (ldcin) and the result written to D (ldd).
int gemm_f32_ex(int ta, int tb, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                int64_t ldb, float beta, const float* Cin, int64_t ldcin, float* D, int64_t ldd, void* ws, int* status,
                cudaStream_t s);
// Tile width the tensor-core product uses for N output columns.
inline int gemm_bn(int N) { return N <= 64 ? 64 : (N <= 128 ? 128 : 256); }

// info->info.status = ID_ETIMEOUT if *status holds kStatTimeout, else ID_OK.
cudaError_t gemm_status_to_info(const int* status, DevInfo* info, cudaStream_t s);

inline int64_t kpad16(int64_t k) { return (k + 15) / 16 * 16; }

// x rounded to TF32 (10 explicit mantissa bits, ties away from zero), the hi
// part of the split; x itself when it is not finite.
__device__ __forceinline__ float tf32_hi(float x) {
    const unsigned u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    return __uint_as_float((u + 0x1000u) & 0xffffe000u);
}

}  // namespace gbid
