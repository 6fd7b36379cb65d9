// T = R11^{-1} R12 and the assembly of Z = [I T] P^T (Sec. 2.1, Definition 1).
//
// The paper reaches Z through the normal equations R_k^T R_k Z = C^T A
// (Eq. final_eq). With Q_k^T A P = [R11 R12] the same Z satisfies
// Z P = [I  R11^{-1} R12], so one back substitution with R11 replaces the
// forward + backward pair and never squares cond(R11).
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "cpqr.cuh"
#include "trace.cuh"

namespace gbid {

constexpr int kSolveThreads = 256;
constexpr size_t kSolveSmemMax = 200 * 1024;

// One block owns `tb` right-hand sides (columns of R12) and runs the
// column-oriented back substitution on them in shared memory:
//   for i = k-1 .. 0:  B(i, :) /= R(i, i);  B(0:i, :) -= R(0:i, i) B(i, :)
// R(r, i) = W[i*ldw + r] (column-major, contiguous in r). FP64 arithmetic.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) k_trsm(const T* __restrict__ W, int ldw, int k, int nrhs, int tb,
                                                        double* __restrict__ Tm, int ldt) {
    extern __shared__ double B[];   // k x tb, then k reciprocals of R's diagonal
    double* rinv = B + (size_t)k * tb;
    const int t = threadIdx.x;
    const int c0 = blockIdx.x * tb;
    const int rg_count = kSolveThreads / tb;
    for (int e = t; e < k * tb; e += kSolveThreads) {
        const int c = e / k, i = e % k;
        B[i * tb + c] = (c0 + c < nrhs) ? (double)W[(int64_t)(k + c0 + c) * ldw + i] : 0.0;
    }
    for (int i = t; i < k; i += kSolveThreads) rinv[i] = 1.0 / (double)W[(int64_t)i * ldw + i];
    const int c = t % tb, rg = t / tb;
    for (int i = k - 1; i >= 0; --i) {
        __syncthreads();
        if (t < tb) B[i * tb + t] *= rinv[i];
        __syncthreads();
        const double ti = B[i * tb + c];
        const T* Rcol = W + (int64_t)i * ldw;
#pragma unroll 4
        for (int r = rg; r < i; r += rg_count) B[r * tb + c] = fma(-(double)Rcol[r], ti, B[r * tb + c]);
    }
    __syncthreads();
    for (int e = t; e < k * tb; e += kSolveThreads) {
        const int i = e / tb, cc = e % tb;
        if (c0 + cc < nrhs) Tm[(int64_t)i * ldt + c0 + cc] = B[i * tb + cc];
    }
}

static int solve_tb(int k) {
    int tb = 32;
    while (tb > 1 && (size_t)k * (tb + 1) * sizeof(double) > kSolveSmemMax) tb /= 2;
    return tb;
}

cudaError_t solve_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmemMax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmemMax);
}

template <typename T>
cudaError_t solve_run(const void* W, int ldw, int k, int n, double* Tm, int ldt, cudaStream_t s) {
    const int nrhs = n - k;
    if (nrhs <= 0) return cudaSuccess;
    const int tb = solve_tb(k);
    const size_t smem = (size_t)k * (tb + 1) * sizeof(double);
    const int tr = trace_begin(TraceKind::kSolve, s);
    k_trsm<T><<<ceil_div(nrhs, tb), kSolveThreads, smem, s>>>(static_cast<const T*>(W), ldw, k, nrhs, tb, Tm, ldt);
    trace_end(tr, s);
    return cudaGetLastError();
}

// Z[i, perm[l]] = delta(i, l) for l < k, T[i, l - k] otherwise; every entry of
// Z's k x n block is written exactly once. Also J = perm[0:k], the count of
// |Z_ij| > 2 and max |Z_ij| (Definition 1 bounds the entries by 2).
template <typename T>
__global__ void __launch_bounds__(256) k_scatter_z(const int* __restrict__ perm, const double* __restrict__ Tm, int ldt,
                                                   int k, int n, T* __restrict__ Z, int64_t ldz, int32_t* J,
                                                   DevInfo* info) {
    const int i = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long gt2 = 0;
    double amax = 0.0;
    if (l < n) {
        const int col = perm[l];
        const double val = l < k ? (l == i ? 1.0 : 0.0) : Tm[(int64_t)i * ldt + (l - k)];
        Z[(int64_t)i * ldz + col] = (T)val;
        const double a = fabs(val);
        gt2 = a > 2.0 ? 1ull : 0ull;
        amax = a == a ? a : INFINITY;
        if (i == 0 && l < k) J[l] = col;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gt2 += __shfl_xor_sync(0xffffffffu, gt2, o);
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if (threadIdx.x % kWarp == 0) {
        if (gt2) atomicAdd(&info->n_gt2, gt2);
        atomicMax(&info->max_abs_z_bits, (unsigned long long)__double_as_longlong(amax));
    }
}

template <typename T>
cudaError_t scatter_z(const int* perm, const double* Tm, int ldt, int k, int n, void* Z, int64_t ldz, int32_t* J,
                      DevInfo* info, cudaStream_t s) {
    dim3 grid(ceil_div(n, 256), k);
    k_scatter_z<T><<<grid, 256, 0, s>>>(perm, Tm, ldt, k, n, static_cast<T*>(Z), ldz, J, info);
    return cudaGetLastError();
}

__global__ void k_finalize(const State* st, DevInfo* info, int k, int transposed, int nb) {
    id_info r = info->info;
    r.rank = st->rank;
    r.n_recompute = st->n_recompute;
    r.r00 = st->r00;
    r.transposed = transposed;
    r.nb = nb;
    r.n_gt2 = (int64_t)info->n_gt2;
    r.max_abs_z = __longlong_as_double((long long)info->max_abs_z_bits);
    if (st->status & kStatNonFinite) r.status = ID_ENONFINITE;
    else if (st->status & kStatTimeout) r.status = ID_ETIMEOUT;
    else if (st->rank < k) r.status = ID_RANK_DEFICIENT;
    else r.status = ID_OK;
    info->info = r;
}

cudaError_t finalize_info(const State* st, DevInfo* info, int k, int transposed, int nb, cudaStream_t s) {
    k_finalize<<<1, 1, 0, s>>>(st, info, k, transposed, nb);
    return cudaGetLastError();
}

template cudaError_t solve_run<double>(const void*, int, int, int, double*, int, cudaStream_t);
template cudaError_t solve_run<float>(const void*, int, int, int, double*, int, cudaStream_t);
template cudaError_t scatter_z<double>(const int*, const double*, int, int, int, void*, int64_t, int32_t*, DevInfo*,
                                       cudaStream_t);
template cudaError_t scatter_z<float>(const int*, const double*, int, int, int, void*, int64_t, int32_t*, DevInfo*,
                                      cudaStream_t);

}  // namespace gbid
