// T = R11^{-1} R12 and the assembly of Z = [I T] P^T (Sec. 2.1, Definition 1).
//
// The paper reaches Z through the normal equations R_k^T R_k Z = C^T A
// (Eq. final_eq). With Q_k^T A P = [R11 R12] the same Z satisfies
// Z P = [I  R11^{-1} R12], so one back substitution with R11 replaces the
// forward + backward pair and never squares cond(R11).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cpqr.cuh"
#include "trace.cuh"

namespace gbid {

constexpr int kSolveThreads = 256;
constexpr size_t kSolveSmemMax = 227 * 1024;
constexpr int kTrsmCols = 32;    // right-hand sides per CTA; lane = column in the update phase
constexpr int kTrsmBlk = 32;     // rows of a diagonal block
constexpr int kTrsmChunk = 64;   // rows of the off-diagonal R panel staged per pass
constexpr int kTrsmLdb = 33;     // padded row stride (doubles) of B and of the diagonal block
constexpr int kTrsmPre = kTrsmBlk * kTrsmChunk / kSolveThreads;   // staged R values per thread

static size_t trsm_smem(int k, bool smem_b, size_t acc_bytes = sizeof(double)) {
    return ((size_t)kTrsmBlk * kTrsmChunk + (size_t)kTrsmBlk * kTrsmLdb + (smem_b ? (size_t)k * kTrsmLdb : 0)) *
           acc_bytes;
}

// Blocked back substitution T = R11^{-1} R12, R = W(0:k, :) upper triangular
// (column-major, R(r, i) = W[i*ldw + r]). One CTA owns kTrsmCols right-hand
// sides B (columns of R12), in shared memory when k x 33 doubles fit (kSmemB)
// and in T itself otherwise. Diagonal blocks of 32 rows go bottom-up:
//   1. B(blk) = D^{-1} B(blk) by column substitution: warp w owns columns
//      4w .. 4w+3, lane r holds row r, x_i broadcast by a shuffle;
//   2. B(0:i0) -= R(0:i0, blk) X: lane = column with X (32 values) in
//      registers, R staged through shared memory 64 rows at a time and read
//      as broadcasts; each warp accumulates 8 rows.
// Every B(r, c) receives its updates in decreasing i and each as
// fma(-R(r, i), x_i, B(r, c)), the order of the unblocked column-oriented
// substitution; x_i = B(i, c) * (1 / R(i, i)). Arithmetic in Acc: FP64 (the
// default), or FP32 for a T that only seeds a least-squares refinement.
template <typename T, bool kSmemB, typename Acc = double>
__global__ void __launch_bounds__(kSolveThreads, 2) k_trsm(const T* __restrict__ W, int ldw, int k, int nrhs,
                                                           double* __restrict__ Tm, int ldt) {
    static_assert(kSmemB || sizeof(Acc) == sizeof(double), "B kept in T requires FP64 arithmetic");
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Acc* sm = reinterpret_cast<Acc*>(sm_raw);
    Acc* Ps = sm;                                   // Ps[q * kTrsmChunk + row]
    Acc* Ds = Ps + kTrsmBlk * kTrsmChunk;           // Ds[col * kTrsmLdb + row]
    Acc* Bs = Ds + kTrsmBlk * kTrsmLdb;             // Bs[i * kTrsmLdb + c]
    const int t = threadIdx.x, lane = t & (kWarp - 1), w = t / kWarp;
    const int c0 = blockIdx.x * kTrsmCols;
    const int ncols = min(kTrsmCols, nrhs - c0);
    Acc* B = kSmemB ? Bs : reinterpret_cast<Acc*>(Tm + c0);
    const int64_t ldb = kSmemB ? kTrsmLdb : ldt;

    for (int e = t; e < k * kTrsmCols; e += kSolveThreads) {
        const int c = e / k, i = e - c * k;         // i fastest: coalesced reads of R12's columns
        if (kSmemB) Bs[i * kTrsmLdb + c] = c < ncols ? (Acc)W[(int64_t)(k + c0 + c) * ldw + i] : Acc(0);
        else if (c < ncols) B[i * ldb + c] = (Acc)W[(int64_t)(k + c0 + c) * ldw + i];
    }
    const bool lane_col = kSmemB || lane < ncols;
    const int nblk = (k + kTrsmBlk - 1) / kTrsmBlk;
    for (int ib = nblk - 1; ib >= 0; --ib) {
        const int i0 = ib * kTrsmBlk, bs = min(kTrsmBlk, k - i0);
        __syncthreads();   // B(i0 : i0+bs) has all its updates; Ds is free
        for (int e = t; e < kTrsmBlk * kTrsmBlk; e += kSolveThreads) {
            const int col = e / kTrsmBlk, row = e % kTrsmBlk;
            Ds[col * kTrsmLdb + row] =
                (col < bs && row < bs) ? (Acc)W[(int64_t)(i0 + col) * ldw + i0 + row] : Acc(0);
        }
        __syncthreads();
        {
            const Acc rv = lane < bs ? Acc(1) / Ds[lane * kTrsmLdb + lane] : Acc(0);
            Acc x[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int c = 4 * w + qq;
                x[qq] = (lane < bs && (kSmemB || c < ncols)) ? B[(i0 + lane) * ldb + c] : Acc(0);
            }
            for (int i = bs - 1; i >= 0; --i) {
                const Acc dl = Ds[i * kTrsmLdb + lane];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    if (lane == i) x[qq] *= rv;
                    const Acc xi = __shfl_sync(0xffffffffu, x[qq], i);
                    if (lane < i) x[qq] = fma(-dl, xi, x[qq]);
                }
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int c = 4 * w + qq;
                if (lane < bs && (kSmemB || c < ncols)) B[(i0 + lane) * ldb + c] = x[qq];
            }
        }
        if (i0 == 0) break;
        __syncthreads();
        Acc X[kTrsmBlk];
#pragma unroll
        for (int q = 0; q < kTrsmBlk; ++q) X[q] = (q < bs && lane_col) ? B[(i0 + q) * ldb + lane] : Acc(0);
        const int nch = (i0 + kTrsmChunk - 1) / kTrsmChunk;
        Acc pre[kTrsmPre];
        auto stage = [&](int r0) {
#pragma unroll
            for (int j = 0; j < kTrsmPre; ++j) {
                const int e = t + j * kSolveThreads, q = e / kTrsmChunk, rl = e % kTrsmChunk;
                pre[j] = (q < bs && r0 + rl < i0) ? (Acc)W[(int64_t)(i0 + q) * ldw + r0 + rl] : Acc(0);
            }
        };
        stage(0);
        for (int ch = 0; ch < nch; ++ch) {
            const int r0 = ch * kTrsmChunk;
            __syncthreads();   // the previous pass is done reading Ps
#pragma unroll
            for (int j = 0; j < kTrsmPre; ++j) Ps[t + j * kSolveThreads] = pre[j];
            __syncthreads();
            if (ch + 1 < nch) stage(r0 + kTrsmChunk);
            const int rb = r0 + 8 * w;
            if (rb < i0) {
                Acc acc[8];
#pragma unroll
                for (int jr = 0; jr < 8; ++jr)
                    acc[jr] = (rb + jr < i0 && lane_col) ? B[(rb + jr) * ldb + lane] : Acc(0);
#pragma unroll
                for (int q = kTrsmBlk - 1; q >= 0; --q) {
                    const Acc* pr = Ps + q * kTrsmChunk + 8 * w;   // broadcast reads
#pragma unroll
                    for (int h = 0; h < 8; ++h) acc[h] = fma(-pr[h], X[q], acc[h]);
                }
#pragma unroll
                for (int jr = 0; jr < 8; ++jr)
                    if (rb + jr < i0 && lane_col) B[(rb + jr) * ldb + lane] = acc[jr];
            }
        }
    }
    if (kSmemB) {
        __syncthreads();
        for (int e = t; e < k * kTrsmCols; e += kSolveThreads) {
            const int i = e / kTrsmCols, c = e % kTrsmCols;
            if (c < ncols) Tm[(int64_t)i * ldt + c0 + c] = (double)Bs[i * kTrsmLdb + c];
        }
    }
}

cudaError_t solve_configure() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_trsm<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSolveSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_trsm<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSolveSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_trsm<float, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSolveSmemMax)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

template <typename T>
cudaError_t solve_run(const void* W, int ldw, int k, int n, double* Tm, int ldt, cudaStream_t s, bool fp32_arith) {
    const int nrhs = n - k;
    if (nrhs <= 0) return cudaSuccess;
    const int grid = ceil_div(nrhs, kTrsmCols);
    if (fp32_arith && sizeof(T) == 4 && trsm_smem(k, true, sizeof(float)) <= kSolveSmemMax) {
        const int tr = trace_begin(TraceKind::kSolve, s);
        k_trsm<float, true, float><<<grid, kSolveThreads, trsm_smem(k, true, sizeof(float)), s>>>(
            static_cast<const float*>(W), ldw, k, nrhs, Tm, ldt);
        trace_end(tr, s);
        return cudaGetLastError();
    }
    const bool smem_b = trsm_smem(k, true) <= kSolveSmemMax;
    const size_t smem = trsm_smem(k, smem_b);
    const int tr = trace_begin(TraceKind::kSolve, s);
    if (smem_b)
        k_trsm<T, true><<<grid, kSolveThreads, smem, s>>>(static_cast<const T*>(W), ldw, k, nrhs, Tm, ldt);
    else
        k_trsm<T, false><<<grid, kSolveThreads, smem, s>>>(static_cast<const T*>(W), ldw, k, nrhs, Tm, ldt);
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
    unsigned long long gt2 = 0;
    T amax = T(0);   // statistics of the stored values, in their precision
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int col = perm[l];
        const T val = l < k ? (l == i ? T(1) : T(0)) : (T)Tm[(int64_t)i * ldt + (l - k)];
        Z[(int64_t)i * ldz + col] = val;
        const T a = val < T(0) ? -val : val;
        gt2 += a > T(2) ? 1ull : 0ull;
        amax = a == a ? (a > amax ? a : amax) : T(INFINITY);
        if (i == 0 && l < k) J[l] = col;
    }
    zstats_commit(gt2, (double)amax, info);
}

template <typename T>
cudaError_t scatter_z(const int* perm, const double* Tm, int ldt, int k, int n, void* Z, int64_t ldz, int32_t* J,
                      DevInfo* info, cudaStream_t s) {
    dim3 grid(ceil_div(n, 256 * 8) > 0 ? ceil_div(n, 256 * 8) : 1, k);   // 8 columns per thread
    k_scatter_z<T><<<grid, 256, 0, s>>>(perm, Tm, ldt, k, n, static_cast<T*>(Z), ldz, J, info);
    return cudaGetLastError();
}

__global__ void k_finalize(const State* st, DevInfo* info, int k, int transposed, int nb, const int* extra_status) {
    id_info r = info->info;
    const int status = st->status | (extra_status ? *extra_status : 0);
    r.rank = st->rank;
    r.n_recompute = st->n_recompute;
    r.r00 = st->r00;
    r.transposed = transposed;
    r.nb = nb;
    r.engine = 1;
    r.err_est = -1.0;
    r.n_gt2 = (int64_t)info->n_gt2;
    r.max_abs_z = __longlong_as_double((long long)info->max_abs_z_bits);
    if (status & kStatBadInput) r.status = ID_EINVAL;
    else if (status & kStatNonFinite) r.status = ID_ENONFINITE;
    else if (status & kStatTimeout) r.status = ID_ETIMEOUT;
    else if (st->rank < k) r.status = ID_RANK_DEFICIENT;
    else r.status = ID_OK;
    info->info = r;
}

cudaError_t finalize_info(const State* st, DevInfo* info, int k, int transposed, int nb, cudaStream_t s,
                          const int* extra_status) {
    k_finalize<<<1, 1, 0, s>>>(st, info, k, transposed, nb, extra_status);
    return cudaGetLastError();
}

// err_est = sqrt(sum of the residual column norms^2 over positions k..n-1) / ||X||_F
// (vn1 holds the squared norms).
__global__ void __launch_bounds__(256) k_err_est(const double* __restrict__ vn1, int k, int n, const State* st,
                                                 DevInfo* info) {
    double s = 0.0;
    for (int l = k + threadIdx.x; l < n; l += blockDim.x) s += vn1[l];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        const double f = st->fro2;
        info->info.err_est = f > 0.0 ? sqrt(tot / f) : 0.0;
    }
}

cudaError_t error_estimate(const double* vn1, int k, int n, const State* st, DevInfo* info, cudaStream_t s) {
    k_err_est<<<1, 256, 0, s>>>(vn1, k, n, st, info);
    return cudaGetLastError();
}

// out[l] = sqrt(vn1[l]): the residual norms from the CPQR's squared norms.
__global__ void __launch_bounds__(256) k_norms_from_squares(const double* __restrict__ vn1, double* __restrict__ out,
                                                            int n) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) out[l] = sqrt(vn1[l]);
}

cudaError_t norms_from_squares(const double* vn1, double* out, int n, cudaStream_t s) {
    const int grid = std::min((n + 255) / 256, 1024);
    k_norms_from_squares<<<grid, 256, 0, s>>>(vn1, out, n);
    return cudaGetLastError();
}

template cudaError_t solve_run<double>(const void*, int, int, int, double*, int, cudaStream_t, bool);
template cudaError_t solve_run<float>(const void*, int, int, int, double*, int, cudaStream_t, bool);
template cudaError_t scatter_z<double>(const int*, const double*, int, int, int, void*, int64_t, int32_t*, DevInfo*,
                                       cudaStream_t);
template cudaError_t scatter_z<float>(const int*, const double*, int, int, int, void*, int64_t, int32_t*, DevInfo*,
                                      cudaStream_t);

}  // namespace gbid
