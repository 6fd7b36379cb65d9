// The cuBLAS handle the library shares (one per device, created on first
// use) and its FP32-accurate GEMM. cuBLAS runs only plain GEMMs here; callers
// bind their stream and a workspace slice under cublas_mutex().
#pragma once

#include <cublas_v2.h>

#include <mutex>

namespace gbid {

extern std::mutex g_cb_mu;
cublasHandle_t cublas_handle();
inline std::mutex& cublas_mutex() { return g_cb_mu; }

// C = alpha op(A) op(B) + beta C (column-major arguments, FP32 data), FP32
// compute emulated on the BF16 tensor cores where cuBLAS finds it faster.
bool sgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int M, int N, int K, float alpha,
           const float* A, int lda, const float* B, int ldb, float beta, float* C, int ldc);

}  // namespace gbid
