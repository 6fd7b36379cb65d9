// One least-squares refinement of an ID's interpolation matrix against A:
//     Z <- Z + (C^T C)^{-1} C^T (A - C Z),   C = A[:, J]
// (the least-squares problem of Sec. 2.1, min ||A - C Z||_F, taken one exact
// Newton step from the Z the sketch gives; Sec. 2.2 asks for this Z).
//
//   1. C = A[:, J] gathered.
//   2. G = C^T C with every product exact and the sums in double-float
//      (about 48 bits), on the FP32 pipe (k_gram).
//   3. G = U^T U by a blocked Cholesky in FP64 (32-wide panels: a one-warp
//      diagonal factorisation, a forward substitution for the panel row, a
//      tiled rank-32 update of the trailing upper triangle). A non-positive
//      pivot (rank(C) < k) sets a flag and Z is left unchanged.
//   4. U^{-1} in FP64 by a blocked inverse (32 x 32 diagonal blocks by back
//      substitution, merged with FP64 products).
//   5. Over column blocks of A small enough that the block's residual stays in
//      L2: R_b^T = A_b^T - Z_b^T C^T and H_b^T = R_b^T C, FP32-accurate
//      3xTF32 products on the tensor cores (gemm.cu). The first writes R_b^T
//      already split into the operand form of the second; the second runs
//      split-K over the m rows, its slices summed in FP64 by k_reduce_split.
//      Columns of J give R_b = 0 exactly (Z[:, J] = I), so they receive no
//      update.
//   6. Y^T = H^T U^{-1}, then Z += (Y^T U^{-T})^T in the last product's
//      epilogue (the correction needs relative accuracy cond(U) u_32 only),
//      Z[:, J] = I restored, Z statistics recomputed.
// Every product runs in the library's own kernels; nothing is allocated.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "cpqr.cuh"
#include "gbid.h"
#include "gemm.cuh"
#include "trace.cuh"

namespace gbid {
namespace {

constexpr int kRThreads = 256;
constexpr int kCholB = 32;
constexpr int kTargetCtas = 152;   // split-K slices are sized to about one wave of CTAs
constexpr int kGramSplit = 16;     // row chunks of the Gram matrix

size_t al(size_t x) { return (x + 255) / 256 * 256; }


// Column block of the refinement's residual: R_b^T (nb x mp, hi and lo) is
// kept near 64 MB so that it stays in L2 between its two products.
int ref_block(int64_t m, int64_t n) {
    const int64_t mp = kpad16(m);
    int64_t nb = (64ll << 20) / (8 * mp) / 128 * 128;
    if (nb < 128) nb = 128;
    if (nb > 8192) nb = 8192;
    const int64_t n128 = (n + 127) / 128 * 128;
    return (int)(nb < n128 ? nb : n128);
}

// Split-K slices of H_b^T = R_b^T C (nb x k output tiles, K = mp).
int ref_splits(int nb, int k, int64_t mp) {
    const int tiles = ((nb + 127) / 128) * ((k + gemm_bn(k) - 1) / gemm_bn(k));
    int sp = kTargetCtas / tiles;
    const int kb = (int)(mp / 16);
    if (sp < 1) sp = 1;
    if (sp > kb) sp = kb;
    const int per = (kb + sp - 1) / sp;
    return (kb + per - 1) / per;
}

struct RefLayout {
    size_t flag, C32, Wa, Gp, gdiag, Uinv64, Ch, Cl, Cth, Ctl, Uth, Utl, Uh, Ul, Zth, Ztl, Rth, Rtl, Part, Hth, Htl,
        Yth, Ytl, total;
    int nb, splits;
};

RefLayout ref_layout(int64_t m, int64_t n, int64_t k) {
    RefLayout L;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = al(off + b);
        return o;
    };
    const size_t kp = (size_t)kpad16(k), mp = (size_t)kpad16(m);
    L.nb = ref_block(m, n);
    L.splits = ref_splits(L.nb, (int)k, (int64_t)mp);
    L.flag = take(16);
    L.C32 = take(4 * (size_t)m * k);
    L.Wa = take(8 * (size_t)k * 2 * k);
    L.Gp = take(8 * (size_t)kGramSplit * k * k);
    L.gdiag = take(8 * (size_t)k);
    L.Uinv64 = take(8 * (size_t)k * k);
    L.Ch = take(4 * (size_t)m * kp);
    L.Cl = take(4 * (size_t)m * kp);
    L.Cth = take(4 * (size_t)k * mp);
    L.Ctl = take(4 * (size_t)k * mp);
    L.Uth = take(4 * (size_t)k * kp);
    L.Utl = take(4 * (size_t)k * kp);
    L.Uh = take(4 * (size_t)k * kp);
    L.Ul = take(4 * (size_t)k * kp);
    L.Zth = take(4 * (size_t)n * kp);
    L.Ztl = take(4 * (size_t)n * kp);
    L.Rth = take(4 * (size_t)L.nb * mp);
    L.Rtl = take(4 * (size_t)L.nb * mp);
    L.Part = take(4 * (size_t)L.splits * L.nb * k);
    L.Hth = take(4 * (size_t)n * kp);
    L.Htl = take(4 * (size_t)n * kp);
    L.Yth = take(4 * (size_t)n * kp);
    L.Ytl = take(4 * (size_t)n * kp);
    L.total = off;
    return L;
}

// flag[0]: 1 = C^T C not positive definite, 2 = a J entry outside [0, n).
__global__ void k_check_j(const int32_t* J, int k, int64_t n, int* flag) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x)
        if (J[c] < 0 || J[c] >= n) flag[0] = 2;
}

__global__ void k_gather(const float* __restrict__ A, int64_t lda, int m, int k, int64_t n,
                         const int32_t* __restrict__ J, float* __restrict__ C32) {
    const int64_t total = (int64_t)m * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e % k);
        const int jc = J[c];
        const float v = (jc >= 0 && jc < n) ? A[i * lda + jc] : 0.0f;   // bad J: flagged, never read out of range
        C32[e] = v;
    }
}

// G = C^T C from C (m x k row-major FP32), upper triangle. Every product is
// split exactly (p = a b, e = fma(a, b, -p)) and summed in double-float (a
// pair of FP32 values, about 48 significant bits; TwoSum for the high part),
// so the FP64 pipe, scarce on this GPU, is not used. 64 x 64 output tiles
// (tile row <= tile column), 16 outputs per thread; blockIdx.z splits the m
// rows into chunks whose FP64 partials P[z] are summed by k_gram_sum.
constexpr int kGT = 64;       // output tile
constexpr int kGK = 32;       // rows of C staged per pass

// (hi, lo) += p + e with TwoSum on the high part; explicit round-to-nearest
// intrinsics keep the compiler from contracting the error terms into FMAs.
__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float e) {
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    lo = __fadd_rn(lo, __fadd_rn(err, e));
    hi = s;
}

__global__ void __launch_bounds__(256) k_gram(const float* __restrict__ C, int m, int k, int rows_per,
                                              double* __restrict__ P) {
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (ti > tj) return;
    __shared__ float As[kGK][kGT], Bs[kGK][kGT];
    const int i0 = ti * kGT, j0 = tj * kGT;
    const int r_lo = blockIdx.z * rows_per, r_hi = min(m, r_lo + rows_per);
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.0f;
    for (int r0 = r_lo; r0 < r_hi; r0 += kGK) {
        __syncthreads();
        for (int e = t; e < kGK * kGT; e += 256) {
            const int rr = e / kGT, c = e % kGT, r = r0 + rr;
            As[rr][c] = (r < r_hi && i0 + c < k) ? C[(int64_t)r * k + i0 + c] : 0.0f;
            Bs[rr][c] = (r < r_hi && j0 + c < k) ? C[(int64_t)r * k + j0 + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kGK; ++rr) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[rr][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[rr][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float p = __fmul_rn(av[a], bv[b]);
                    const float e = fmaf(av[a], bv[b], -p);   // exact: a b = p + e
                    df_add(hi[a][b], lo[a][b], p, e);
                }
        }
    }
    double* Pz = P + (size_t)blockIdx.z * k * k;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < k && j < k && i <= j) Pz[(int64_t)j * k + i] = (double)hi[a][b] + (double)lo[a][b];
        }
}

__global__ void k_gram_sum(const double* __restrict__ P, int nz, int k, double* __restrict__ G,
                           double* __restrict__ gdiag) {
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / k), i = (int)(e % k);
        if (i > j) continue;
        double s = 0.0;
        for (int z = 0; z < nz; ++z) s += P[(size_t)z * total + e];
        G[e] = s;
        if (i == j) gdiag[i] = s;
    }
}

// B = C^T A (k x n, FP64 row-major) from C (m x k row-major FP32) and A (m x n
// row-major FP32, lda), with the products exact and the sums in double-float
// as in k_gram: the right-hand side of the normal equations to about 48 bits
// without the FP64 pipe. 64 x 64 output tiles, 16 outputs per thread, every
// tile sums all m rows.
__global__ void __launch_bounds__(256) k_ctb(const float* __restrict__ C, const float* __restrict__ A, int64_t lda,
                                             int m, int k, int n, double* __restrict__ B) {
    __shared__ float Cs[kGK][kGT], As[kGK][kGT];
    const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.0f;
    for (int r0 = 0; r0 < m; r0 += kGK) {
        __syncthreads();
        for (int e = t; e < kGK * kGT; e += 256) {
            const int rr = e / kGT, c = e % kGT, r = r0 + rr;
            Cs[rr][c] = (r < m && i0 + c < k) ? C[(int64_t)r * k + i0 + c] : 0.0f;
            As[rr][c] = (r < m && j0 + c < n) ? A[(int64_t)r * lda + j0 + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kGK; ++rr) {
            float cv[4], av[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) cv[a] = Cs[rr][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) av[b] = As[rr][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float p = __fmul_rn(cv[a], av[b]);
                    const float e = fmaf(cv[a], av[b], -p);
                    df_add(hi[a][b], lo[a][b], p, e);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < k && j < n) B[(int64_t)i * n + j] = (double)hi[a][b] + (double)lo[a][b];
        }
}

// Diagonal block (b <= 32) at p0: D = U_D^T U_D in place. 256 threads: per
// step j one thread takes the square root, the row is scaled by its
// reciprocal, and the rank-1 update of the remaining upper triangle is spread
// over all threads.
// A pivot at or below 64 eps of its column's squared norm (the original G(j, j))
// counts as zero: C is then numerically rank deficient for normal equations.
__global__ void __launch_bounds__(256) k_chol_diag(double* G, int ld, int p0, int b, const double* gdiag,
                                                   int* flag) {
    __shared__ double D[kCholB][kCholB + 1];
    __shared__ double gd[kCholB];   // the block's original diagonal, loaded once (not per step)
    __shared__ double rj_s;
    const int t = threadIdx.x;
    for (int e = t; e < kCholB * kCholB; e += blockDim.x) {
        const int r = e / kCholB, c = e % kCholB;
        D[r][c] = (c < b && r <= c) ? G[(int64_t)(p0 + c) * ld + p0 + r] : 0.0;
    }
    if (t < b) gd[t] = gdiag[p0 + t];
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (t == 0) {
            const double d = D[j][j];
            double u = 1.0, ru = 1.0;
            if (!(d > 64.0 * DBL_EPSILON * gd[j]) || !isfinite(d)) {
                if (flag[0] == 0) flag[0] = 1;
            } else {
                ru = rsqrt(d);   // one reciprocal square root instead of a square root and a division:
                u = d * ru;      // FP64 runs at 2 lanes per clock per SM, so this chain sets the pace
            }
            D[j][j] = u;
            rj_s = ru;
        }
        __syncthreads();
        if (t > j && t < b) D[j][t] *= rj_s;
        __syncthreads();
        // D(r, c) -= U(j, r) U(j, c) for j < r <= c < b
        const int w = b - j - 1;
        for (int e = t; e < w * w; e += blockDim.x) {
            const int r = j + 1 + e / w, c = j + 1 + e % w;
            if (r <= c) D[r][c] -= D[j][r] * D[j][c];
        }
        __syncthreads();
    }
    for (int e = t; e < kCholB * kCholB; e += blockDim.x) {
        const int r = e / kCholB, c = e % kCholB;
        if (c < b && r <= c) G[(int64_t)(p0 + c) * ld + p0 + r] = D[r][c];
    }
}

// Panel row: U(p0:p0+b, c) = U_D^{-T} G(p0:p0+b, c) for c >= p0 + b. A warp per
// column, lane = row of the panel: forward substitution with x_q broadcast.
__global__ void __launch_bounds__(256) k_chol_row(double* G, int ld, int p0, int b, int k) {
    __shared__ double U[kCholB][kCholB + 1];
    __shared__ double rinv[kCholB];
    for (int e = threadIdx.x; e < kCholB * kCholB; e += blockDim.x) {
        const int r = e / kCholB, q = e % kCholB;
        U[r][q] = (r < b && q < b && r <= q) ? G[(int64_t)(p0 + q) * ld + p0 + r] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < b) rinv[threadIdx.x] = 1.0 / U[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x % kWarp;
    const int c = p0 + b + blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
    if (c >= k) return;                           // warp-uniform
    double* col = G + (int64_t)c * ld + p0;
    double x = lane < b ? col[lane] : 0.0;
    for (int q = 0; q < b; ++q) {
        const double xq = __shfl_sync(0xffffffffu, x, q) * rinv[q];
        if (lane == q) x = xq;
        if (lane > q) x = fma(-U[q][lane], xq, x);
    }
    if (lane < b) col[lane] = x;
}

// Trailing update G(r, c) -= sum_{q < b} U(p0+q, r) U(p0+q, c), p0+b <= r, c < k,
// on 32 x 32 tiles of the upper triangle (tile row <= tile column).
__global__ void k_chol_update(double* G, int ld, int p0, int b, int k) {
    const int t0 = p0 + b;
    const int tr = blockIdx.y, tc = blockIdx.x;
    if (tr > tc) return;
    __shared__ double Ur[kCholB][kCholB + 1], Uc[kCholB][kCholB + 1];
    const int r0 = t0 + tr * kCholB, c0 = t0 + tc * kCholB;
    for (int e = threadIdx.x; e < kCholB * kCholB; e += blockDim.x) {
        const int q = e / kCholB, i = e % kCholB;
        Ur[q][i] = (q < b && r0 + i < k) ? G[(int64_t)(r0 + i) * ld + p0 + q] : 0.0;
        Uc[q][i] = (q < b && c0 + i < k) ? G[(int64_t)(c0 + i) * ld + p0 + q] : 0.0;
    }
    __syncthreads();
    const int i = threadIdx.x % kCholB, jg = threadIdx.x / kCholB;   // 8 groups of 4 columns
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < b; ++q) {
        const double u = Ur[q][i];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a] = fma(u, Uc[q][jg * 4 + a], acc[a]);
    }
    const int r = r0 + i;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int c = c0 + jg * 4 + a;
        if (r < k && c < k && r <= c) G[(int64_t)c * ld + r] -= acc[a];
    }
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

__global__ void k_restore_identity(float* Z, int64_t ldz, const int32_t* J, int k, const int* flag) {
    if (flag[0]) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
        const int i = e / k, l = e % k;
        Z[(int64_t)i * ldz + J[l]] = i == l ? 1.0f : 0.0f;
    }
}

__global__ void k_zstats(const float* Z, int64_t ldz, int k, int n, const int* flag, DevInfo* info) {
    if (flag[0]) return;
    const int i = blockIdx.y;
    unsigned long long gt2 = 0;
    float amax = 0.0f;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const float a = fabsf(Z[(int64_t)i * ldz + l]);
        gt2 += a > 2.0f ? 1ull : 0ull;
        amax = a == a ? fmaxf(amax, a) : INFINITY;
    }
    zstats_commit(gt2, (double)amax, info);
}

__global__ void k_reset_stats(DevInfo* info, const int* flag) {
    if (flag[0]) return;
    info->n_gt2 = 0;
    info->max_abs_z_bits = 0;
}

// flag[0]: 1 = C^T C not positive definite, 2 = a J entry outside [0, n);
// flag[1]: kStat* bits of the products (kStatTimeout: a bounded wait expired).
__global__ void k_ref_finalize(DevInfo* info, const int* flag) {
    id_info r = info->info;
    r.refined = flag[0] ? 0 : 1;
    if (flag[0] == 2) r.status = ID_EINVAL;
    if (flag[1] & kStatTimeout) {
        r.status = ID_ETIMEOUT;
        r.refined = 0;
    }
    if (!flag[0]) {
        r.n_gt2 = (int64_t)info->n_gt2;
        r.max_abs_z = __longlong_as_double((long long)info->max_abs_z_bits);
    }
    info->info = r;
}

__global__ void k_info_init(DevInfo* d, int k) {
    DevInfo z = {};
    z.info.status = ID_OK;
    z.info.rank = k;
    z.info.err_est = -1.0;
    *d = z;
}

int grid_for(int64_t n) {
    const int64_t g = (n + kRThreads - 1) / kRThreads;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// Backward pass (gradient through the ID with J frozen). G64 = dZ with the
// columns of J zeroed, in FP64.
__global__ void k_mask_j(const int32_t* J, int k, int64_t n, unsigned char* mask) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x)
        if (J[c] >= 0 && J[c] < n) mask[J[c]] = 1;
}

__global__ void k_gz(const float* __restrict__ dZ, int64_t lddz, int k, int n, const unsigned char* __restrict__ mask,
                     double* __restrict__ G64) {
    const int i = blockIdx.y;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
        G64[(int64_t)i * n + l] = mask[l] ? 0.0 : (double)dZ[(int64_t)i * lddz + l];
}

// dA[:, J[c]] = dC[:, c] (dC row-major m x k)
__global__ void k_scatter_dc(const float* __restrict__ dC, int m, int k, const int32_t* __restrict__ J, int64_t n,
                             float* dA, int64_t ldda) {
    const int64_t total = (int64_t)m * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e % k);
        const int jc = J[c];
        if (jc >= 0 && jc < n) dA[i * ldda + jc] = dC[e];
    }
}

__global__ void k_bwd_finalize(DevInfo* info, const int* flag) {
    id_info r = info->info;
    if (flag[0] == 2) r.status = ID_EINVAL;
    else if (flag[0] == 1) r.status = ID_RANK_DEFICIENT;
    if (flag[1] & kStatTimeout) r.status = ID_ETIMEOUT;
    info->info = r;
}

// ---- column-sampling Optim RID (Sec. 2.2) ----
// W (column-major, ldw) <- A[:, idx[l]], padding rows zero.
template <typename T>
__global__ void k_gather_sample(const T* __restrict__ A, int64_t lda, int m, const int32_t* __restrict__ idx, int p,
                                T* __restrict__ W, int ldw) {
    const int64_t total = (int64_t)ldw * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / ldw), i = (int)(e % ldw);
        W[e] = i < m ? A[(int64_t)i * lda + idx[l]] : T(0);
    }
}

// J = idx[perm[0:k]] (idx == nullptr: J = perm[0:k], the pivots themselves)
__global__ void k_map_j(const int* __restrict__ perm, const int32_t* __restrict__ idx, int k, int32_t* J) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < k; l += gridDim.x * blockDim.x)
        J[l] = idx ? idx[perm[l]] : perm[l];
}

template <typename T>
__global__ void k_gather_f64(const T* __restrict__ A, int64_t lda, int m, int k, const int32_t* __restrict__ J,
                             double* __restrict__ C64) {
    const int64_t total = (int64_t)m * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e % k);
        C64[e] = (double)A[i * lda + J[c]];
    }
}

// Wr (k x 2k, column-major, ld k) = [R_k | I], R_k from the CPQR's W (R(i, q) = W[q*ldw + i], i <= q).
template <typename T>
__global__ void k_rk_identity(const T* __restrict__ W, int ldw, int k, double* __restrict__ Wr) {
    const int64_t total = (int64_t)k * 2 * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / k), r = (int)(e % k);
        Wr[e] = c < k ? (r <= c ? (double)W[(int64_t)c * ldw + r] : 0.0) : (r == c - k ? 1.0 : 0.0);
    }
}

template <typename T>
__global__ void k_z_from64(const double* __restrict__ Z64, int k, int n, T* __restrict__ Z, int64_t ldz) {
    const int i = blockIdx.y;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
        Z[(int64_t)i * ldz + l] = (T)Z64[(int64_t)i * n + l];
}

template <typename T>
__global__ void k_identity_at_j(T* Z, int64_t ldz, const int32_t* J, int k) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
        const int i = e / k, l = e % k;
        Z[(int64_t)i * ldz + J[l]] = i == l ? T(1) : T(0);
    }
}

template <typename T>
__global__ void k_zstats_t(const T* Z, int64_t ldz, int k, int n, DevInfo* info) {
    const int i = blockIdx.y;
    unsigned long long gt2 = 0;
    T amax = T(0);
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        T a = Z[(int64_t)i * ldz + l];
        a = a < T(0) ? -a : a;
        gt2 += a > T(2) ? 1ull : 0ull;
        amax = a == a ? (a > amax ? a : amax) : T(INFINITY);
    }
    zstats_commit(gt2, (double)amax, info);
}

__global__ void k_sampled_finalize(DevInfo* info, const int* flag) {
    id_info r = info->info;
    if (flag[0] == 1 && r.status == ID_OK) r.status = ID_RANK_DEFICIENT;   // C^T C not positive definite
    r.n_gt2 = (int64_t)info->n_gt2;
    r.max_abs_z = __longlong_as_double((long long)info->max_abs_z_bits);
    info->info = r;
}

// ------------------------------------------------ triangular inverse U^{-1} --
// Blocked: the kTriLeaf x kTriLeaf diagonal blocks are inverted by back
// substitution (one CTA per block, one thread per column), then neighbouring
// blocks merge, [A B; 0 C]^{-1} = [A^{-1}  -A^{-1} B C^{-1}; 0  C^{-1}], with two
// FP64 GEMMs per merge, so the work spreads over the GPU instead of a few
// column blocks of one solve.
constexpr int kTriLeaf = 32;

__global__ void __launch_bounds__(kTriLeaf) k_tri_inv_leaf(const double* __restrict__ U, int k,
                                                          double* __restrict__ Uinv) {
    __shared__ double Us[kTriLeaf][kTriLeaf + 1];
    __shared__ double Xs[kTriLeaf][kTriLeaf + 1];
    const int o = blockIdx.x * kTriLeaf, b = min(kTriLeaf, k - o), c = threadIdx.x;
    for (int r = 0; r < b; ++r) Us[r][c] = (c < b && r <= c) ? U[(int64_t)(o + c) * k + o + r] : 0.0;
    __syncthreads();
    if (c < b) {
        // U_blk x = e_c by back substitution; x_r = 0 for r > c
        for (int r = b - 1; r >= 0; --r) {
            if (r > c) {
                Xs[r][c] = 0.0;
                continue;
            }
            double acc = r == c ? 1.0 : 0.0;
            for (int j = r + 1; j <= c; ++j) acc -= Us[r][j] * Xs[j][c];
            Xs[r][c] = acc / Us[r][r];
        }
        for (int r = 0; r < b; ++r) Uinv[(int64_t)(o + c) * k + o + r] = Xs[r][c];
    }
}

// out (row-major k x k) = the transpose of in (column-major k x k): the same matrix, row-major.
__global__ void k_cm_to_rm(const double* __restrict__ in, int k, double* __restrict__ out) {
    const int64_t total = (int64_t)k * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), c = (int)(e % k);
        out[e] = in[(int64_t)c * k + i];
    }
}

// U: upper triangle of a column-major k x k array (ld k; below the diagonal
// unused). Uinv_cm (k x k, column-major) and tmp ((k/2 + kTriLeaf)^2 doubles)
// are scratch; Uinv_rm receives U^{-1} row-major. The merges run the
// row-major FP64 product on the transposes (a column-major block read
// row-major is the block's transpose).
cudaError_t tri_inverse(const double* U, int k, double* Uinv_cm, double* tmp, double* Uinv_rm, cudaStream_t s) {
    if (cudaMemsetAsync(Uinv_cm, 0, sizeof(double) * (size_t)k * k, s) != cudaSuccess) return cudaErrorUnknown;
    const int nleaf = ceil_div(k, kTriLeaf);
    k_tri_inv_leaf<<<nleaf, kTriLeaf, 0, s>>>(U, k, Uinv_cm);
    // merge blocks of width w into blocks of width 2w, bottom-up; the merges of
    // one level with b2 = w run as one batched launch per product (pair p at
    // o1 = 2 w p; its tmp at tmp + p w^2), a ragged last pair on its own
    for (int w = kTriLeaf; w < k; w *= 2) {
        const int full = (k / w) / 2;           // pairs with b2 = w
        const bool ragged = (k / w) % 2 == 1 && k % w != 0;   // a last pair with 0 < b2 < w
        for (int part = 0; part < 2; ++part) {
            const int batch = part == 0 ? full : (ragged ? 1 : 0);
            if (batch == 0) continue;
            const int o1 = part == 0 ? 0 : 2 * w * full;
            const int b1 = w, o2 = o1 + w, b2 = part == 0 ? w : k - o2;
            const int64_t stride = (int64_t)2 * w * (k + 1);   // pair p+1 is 2w rows and 2w columns further
            double* tp = tmp + (part == 0 ? 0 : (int64_t)full * w * w);
            // tmp (b1 x b2, column-major ld b1) = A^{-1} B, formed as tmp^T = B^T A^{-T}
            cudaError_t e = dgemm_batched(b2, b1, b1, 1.0, U + o1 + (int64_t)o2 * k, k, stride,
                                          Uinv_cm + o1 + (int64_t)o1 * k, k, stride, 0.0, tp, b1, (int64_t)w * w,
                                          batch, s);
            if (e != cudaSuccess) return e;
            // U^{-1}(o1, o2) = -tmp C^{-1}, formed as its transpose -C^{-T} tmp^T
            e = dgemm_batched(b2, b1, b2, -1.0, Uinv_cm + o2 + (int64_t)o2 * k, k, stride, tp, b1, (int64_t)w * w,
                              0.0, Uinv_cm + o1 + (int64_t)o2 * k, k, stride, batch, s);
            if (e != cudaSuccess) return e;
        }
    }
    k_cm_to_rm<<<grid_for((int64_t)k * k), kRThreads, 0, s>>>(Uinv_cm, k, Uinv_rm);
    return cudaGetLastError();
}

// Steps 1-4 shared by the refinement and the backward pass: C = A[:, J],
// G = C^T C (double-float), G = U^T U (FP64, flag[0] = 1 if not positive
// definite), U^{-1} in FP64 (row-major k x k) by the blocked inverse (Gp and
// Wa's second half are its scratch).
// C^T C = U^T U (FP64 Cholesky of the double-float Gram) and U^{-1}, from C32.
static cudaError_t factor_gram(int64_t m, int k, const float* C32, double* Gp, double* Wa, double* Uinv64,
                               double* gdiag, int* flag, cudaStream_t s) {
    const int nt = ceil_div(k, kGT);
    const int rows_per = (int)round_up(ceil_div(m, kGramSplit), kGK);
    k_gram<<<dim3(nt, nt, kGramSplit), 256, 0, s>>>(C32, (int)m, k, rows_per, Gp);
    k_gram_sum<<<grid_for((int64_t)k * k), kRThreads, 0, s>>>(Gp, kGramSplit, k, Wa, gdiag);
    for (int p0 = 0; p0 < k; p0 += kCholB) {
        const int b = k - p0 < kCholB ? k - p0 : kCholB;
        k_chol_diag<<<1, 256, 0, s>>>(Wa, k, p0, b, gdiag, flag);
        const int rest = k - p0 - b;
        if (rest > 0) {
            k_chol_row<<<ceil_div(rest, 8), 256, 0, s>>>(Wa, k, p0, b, k);
            const int nt2 = ceil_div(rest, kCholB);
            k_chol_update<<<dim3(nt2, nt2), kRThreads, 0, s>>>(Wa, k, p0, b, k);
        }
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return tri_inverse(Wa, k, Wa + (size_t)k * k, Gp, Uinv64, s);
}

cudaError_t factor_skeleton(const float* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, float* C32,
                            double* Gp, double* Wa, double* Uinv64, double* gdiag, int* flag, cudaStream_t s) {
    k_check_j<<<1, kRThreads, 0, s>>>(J, k, n, flag);
    k_gather<<<grid_for(m * k), kRThreads, 0, s>>>(A, lda, (int)m, k, n, J, C32);
    return factor_gram(m, k, C32, Gp, Wa, Uinv64, gdiag, flag, s);
}

// A side stream per device for work that overlaps the main stream inside one
// call (the Gram factor of the refinement beside its residual products), with
// the fork and join events. The enqueue of one fork/join pair holds the mutex,
// so concurrent calls never interleave their records and waits on the shared
// events; a stream under capture takes the sequential order instead.
struct SideStream {
    std::mutex mu;
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // a second side stream for the split-K sums of the residual loop, with its events
    cudaStream_t s3 = nullptr;
    cudaEvent_t g2done = nullptr, reddone = nullptr;
    bool ok = false, tried = false;
};
static SideStream g_side[64];

static SideStream* side_stream(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    SideStream* ss = &g_side[dev];
    ss->mu.lock();
    if (!ss->tried) {
        ss->tried = true;
        ss->ok = cudaStreamCreateWithFlags(&ss->s2, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ss->fork, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ss->join, cudaEventDisableTiming) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&ss->s3, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ss->g2done, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ss->reddone, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ss->ok) {
        ss->mu.unlock();
        return nullptr;
    }
    return ss;   // locked: the caller unlocks after enqueueing its join
}

// H^T rows of one column block from the split-K slices of R_b^T C:
// H(l, q) = sum_z P[z][l][q], summed in double-float on the FP32 pipe (TwoSum
// of the running sum, the rounding errors collected in a second float),
// rounded to FP32 and split into the operand form (columns k..kp-1 zero).
__global__ void k_reduce_split(const float* __restrict__ P, int splits, int nb, int k, int kp, float* __restrict__ hi,
                               float* __restrict__ lo) {
    const int64_t total = (int64_t)nb * kp;
    const int64_t slice = (int64_t)nb * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / kp), q = (int)(e % kp);
        float sh = 0.0f, sl = 0.0f;
        if (q < k)
            for (int z0 = 0; z0 < splits; z0 += 8) {
                float xs[8];   // eight slices' loads in flight before the dependent sums
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    xs[u] = z0 + u < splits ? P[(z0 + u) * slice + (int64_t)l * k + q] : 0.0f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float x = xs[u];
                    const float t = __fadd_rn(sh, x);
                    const float bp = __fsub_rn(t, sh);
                    sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
                    sh = t;
                }
            }
        const float x = __fadd_rn(sh, sl);
        const float h = tf32_hi(x);
        hi[e] = h;
        lo[e] = x - h;
    }
}

}  // namespace

size_t refine_bytes(int64_t m, int64_t n, int64_t k) { return ref_layout(m, n, k).total; }

// Kernel launches of refine_run for this problem (memsets excluded); the
// count follows the launch sites of factor_skeleton, tri_inverse and
// refine_run one for one.
int64_t refine_launch_count(int64_t m, int64_t n, int64_t k) {
    int64_t c = 4;   // k_check_j, k_gather, k_gram, k_gram_sum
    for (int64_t p0 = 0; p0 < k; p0 += kCholB) c += 1 + (k - p0 - kCholB > 0 ? 2 : 0);
    c += 2;          // the inverse's leaves and the final layout change
    for (int64_t w = kTriLeaf; w < k; w *= 2) {
        const bool full = (k / w) / 2 > 0, ragged = (k / w) % 2 == 1 && k % w != 0;
        c += (full ? 2 : 0) + (ragged ? 2 : 0);
    }
    const RefLayout L = ref_layout(m, n, k);
    c += 5;                                     // the operand splits of C, C^T, U^{-T}, U^{-1}, Z^T
    c += 3 * ((n + L.nb - 1) / L.nb);           // per column block: R_b^T, the split-K slices, their sum
    c += 2 + 4;                                 // Y^T and the Z update; identity, reset, statistics, status
    return c;
}



cudaError_t refine_info_init(DevInfo* dinfo, int k, cudaStream_t s) {
    k_info_init<<<1, 1, 0, s>>>(dinfo, k);
    return cudaGetLastError();
}

int refine_run(const float* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, float* Z, int64_t ldz,
               void* ws, DevInfo* dinfo, cudaStream_t s) {
    const RefLayout L = ref_layout(m, n, k);
    char* base = static_cast<char*>(ws);
    auto fp = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
    int* flag = reinterpret_cast<int*>(base + L.flag);
    int* gst = flag + 1;   // status bits of the products
    float* C32 = fp(L.C32);
    double* Gp = reinterpret_cast<double*>(base + L.Gp);
    double* Wa = reinterpret_cast<double*>(base + L.Wa);
    double* Uinv64 = reinterpret_cast<double*>(base + L.Uinv64);
    const int kp = (int)kpad16(k), mp = (int)kpad16(m);
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    const int tr = trace_begin(TraceKind::kRefine, s);
    k_check_j<<<1, kRThreads, 0, s>>>(J, k, n, flag);
    k_gather<<<grid_for(m * k), kRThreads, 0, s>>>(A, lda, (int)m, k, n, J, C32);
    // The Gram factor (C^T C = U^T U, U^{-1} and its operand forms) is needed only by the
    // last two products: it runs on a side stream beside the residual products when the
    // caller's stream is not being captured (a chain of small latency-bound launches).
    SideStream* ss = side_stream(s);
    cudaStream_t sg = ss ? ss->s2 : s;
    if (ss && (cudaEventRecord(ss->fork, s) != cudaSuccess || cudaStreamWaitEvent(sg, ss->fork, 0) != cudaSuccess)) {
        ss->mu.unlock();
        return ID_ECUDA;
    }
    bool gram_ok = factor_gram(m, k, C32, Gp, Wa, Uinv64, reinterpret_cast<double*>(base + L.gdiag), flag, sg) ==
                       cudaSuccess &&
                   split_tf32<double>(Uinv64, k, 1, k, k, kp, fp(L.Uth), fp(L.Utl), kp, sg) == cudaSuccess &&
                   split_tf32<double>(Uinv64, k, 0, k, k, kp, fp(L.Uh), fp(L.Ul), kp, sg) == cudaSuccess;
    if (ss) gram_ok = gram_ok && cudaEventRecord(ss->join, sg) == cudaSuccess;   // (waited on after the loop)
    if (!gram_ok) {
        if (ss) ss->mu.unlock();
        return ID_ECUDA;
    }
    // operands: C (m x kp), C^T (k x mp)
    auto fail = [&](int rc) {
        if (ss) ss->mu.unlock();
        return rc;
    };
    if (split_tf32<float>(C32, k, 0, (int)m, k, kp, fp(L.Ch), fp(L.Cl), kp, s) != cudaSuccess) return fail(ID_ECUDA);
    if (split_tf32<float>(C32, k, 1, k, (int)m, mp, fp(L.Cth), fp(L.Ctl), mp, s) != cudaSuccess) return fail(ID_ECUDA);
    const TfOperand opC{fp(L.Ch), fp(L.Cl), kp, (int)m};
    const TfOperand opCt{fp(L.Cth), fp(L.Ctl), mp, k};
    // columns m..mp-1 of R_b^T stay zero (the products write columns < m only)
    if (mp > m && (cudaMemsetAsync(fp(L.Rth), 0, 4 * (size_t)L.nb * mp, s) != cudaSuccess ||
                   cudaMemsetAsync(fp(L.Rtl), 0, 4 * (size_t)L.nb * mp, s) != cudaSuccess))
        return fail(ID_ECUDA);
    // Z^T (n x kp) in operand form, once for all column blocks
    if (split_tf32<float>(Z, ldz, 1, (int)n, k, kp, fp(L.Zth), fp(L.Ztl), kp, s) != cudaSuccess) return fail(ID_ECUDA);
    // 5. H^T = (A - C Z)^T C by column blocks of A
    for (int64_t b0 = 0; b0 < n; b0 += L.nb) {
        const int nbb = (int)(n - b0 < L.nb ? n - b0 : L.nb);
        // R_b = A_b - C Z_b (m x nbb, the accumulator's lanes along the rows of A, so that
        // the reads of A and the transposed stores of R_b^T (nbb x mp, operand form) coalesce)
        TfEpilogue e1;
        e1.alpha = -1.0f;
        e1.beta = 1.0f;
        e1.cin = A + b0;
        e1.ldc = lda;
        e1.cin_cols = nbb;
        e1.d = fp(L.Rth);
        e1.d_lo = fp(L.Rtl);
        e1.ldd = mp;
        e1.d_trans = 1;
        int rc = gemm_tf32x3(opC, TfOperand{fp(L.Zth) + b0 * kp, fp(L.Ztl) + b0 * kp, kp, nbb}, (int)m, nbb, kp, 1, e1,
                             gst, s);
        if (rc != ID_OK) return fail(rc);
        // split-K slices of H_b^T = R_b^T C (nbb x k), then their FP64 sum in operand form
        TfEpilogue e2;
        e2.d = fp(L.Part);
        e2.ldd = k;
        e2.z_stride = (int64_t)nbb * k;
        // (the previous block's sum must be done reading the slices before they are rewritten)
        if (ss && b0 > 0 && cudaStreamWaitEvent(s, ss->reddone, 0) != cudaSuccess) return fail(ID_ECUDA);
        rc = gemm_tf32x3(TfOperand{fp(L.Rth), fp(L.Rtl), mp, nbb}, opCt, nbb, k, mp, L.splits, e2, gst, s);
        if (rc != ID_OK) return fail(rc);
        // the sum of the slices runs on the second side stream, beside the next block's
        // residual product (which leaves SMs idle in its last wave)
        cudaStream_t sr = s;
        if (ss) {
            if (cudaEventRecord(ss->g2done, s) != cudaSuccess || cudaStreamWaitEvent(ss->s3, ss->g2done, 0) != cudaSuccess)
                return fail(ID_ECUDA);
            sr = ss->s3;
        }
        k_reduce_split<<<grid_for((int64_t)nbb * kp), kRThreads, 0, sr>>>(fp(L.Part), L.splits, nbb, k, kp,
                                                                           fp(L.Hth) + b0 * kp, fp(L.Htl) + b0 * kp);
        if (ss && cudaEventRecord(ss->reddone, ss->s3) != cudaSuccess) return fail(ID_ECUDA);
    }
    // join: the products below need U^{-1} and every block's sum
    if (ss) {
        const bool jw = cudaStreamWaitEvent(s, ss->join, 0) == cudaSuccess &&
                        cudaStreamWaitEvent(s, ss->reddone, 0) == cudaSuccess;
        ss->mu.unlock();
        if (!jw) return ID_ECUDA;
    }
    // 6. Y^T = H^T U^{-1} (B(q, p) = U^{-1}(p, q)); Z += (Y^T U^{-T})^T in the epilogue (B(q, p) = U^{-1}(q, p))
    TfEpilogue e3;
    e3.d = fp(L.Yth);
    e3.d_lo = fp(L.Ytl);
    e3.ldd = kp;
    int rc = gemm_tf32x3(TfOperand{fp(L.Hth), fp(L.Htl), kp, (int)n}, TfOperand{fp(L.Uth), fp(L.Utl), kp, k}, (int)n,
                         kp, kp, 1, e3, gst, s);
    if (rc != ID_OK) return rc;
    TfEpilogue e4;
    e4.alpha = 1.0f;
    e4.beta = 1.0f;
    e4.cin = Z;
    e4.ldc = ldz;
    e4.cin_trans = 1;
    e4.d = Z;
    e4.ldd = ldz;
    e4.d_trans = 1;
    e4.skip = flag;   // no update when C^T C is singular or J is invalid
    rc = gemm_tf32x3(TfOperand{fp(L.Yth), fp(L.Ytl), kp, (int)n}, TfOperand{fp(L.Uh), fp(L.Ul), kp, k}, (int)n, k,
                     kp, 1, e4, gst, s);
    if (rc != ID_OK) return rc;
    dim3 g2(ceil_div(n, kRThreads * 8), k);
    k_restore_identity<<<grid_for((int64_t)k * k), kRThreads, 0, s>>>(Z, ldz, J, k, flag);
    k_reset_stats<<<1, 1, 0, s>>>(dinfo, flag);
    k_zstats<<<g2, kRThreads, 0, s>>>(Z, ldz, k, (int)n, flag, dinfo);
    k_ref_finalize<<<1, 1, 0, s>>>(dinfo, flag);
    trace_end(tr, s);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

struct BwdLayout {
    size_t flag, mask, C32, Gp, gdiag, Wa, Uinv64, G64, Y64, W32, R, dC, M1, gws, total;
};

static BwdLayout bwd_layout(int64_t m, int64_t n, int64_t k) {
    BwdLayout L;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = al(off + b);
        return o;
    };
    L.flag = take(16);
    L.mask = take((size_t)n);
    L.C32 = take(4 * (size_t)m * k);
    L.Gp = take(8 * (size_t)kGramSplit * k * k);
    L.gdiag = take(8 * (size_t)k);
    L.Wa = take(8 * (size_t)k * 2 * k);
    L.Uinv64 = take(8 * (size_t)k * k);
    L.G64 = take(8 * (size_t)k * n);
    L.Y64 = take(8 * (size_t)k * n);
    L.W32 = take(4 * (size_t)k * n);
    L.R = take(4 * (size_t)m * n);
    L.dC = take(4 * (size_t)m * k);
    L.M1 = take(4 * (size_t)k * k);
    // operand scratch of the largest of the five FP32 products
    size_t g = gemm_f32_bytes((int)m, (int)n, (int)k);
    const size_t g2 = gemm_f32_bytes((int)m, (int)k, (int)n), g3 = gemm_f32_bytes((int)k, (int)k, (int)n);
    if (g2 > g) g = g2;
    if (g3 > g) g = g3;
    L.gws = take(g);
    L.total = off;
    return L;
}

size_t backward_bytes(int64_t m, int64_t n, int64_t k) { return bwd_layout(m, n, k).total; }

// Gradient of L(Z) through the ID with J frozen: Z[:, rest] = T = C^+ B
// (C = A[:, J], B = A[:, rest]); with W = (C^T C)^{-1} dZ_rest:
//   dA[:, rest] = C W,   dA[:, J] = (B - C T) W^T - C W T^T.
// In full-width form (W zero on J, R = A - C Z zero on J):
//   dA = C W (all columns, zero on J), dC = R W^T - C (W Z^T), dA[:, J] = dC.
// W is formed in FP64 (U^{-1} applied twice: the gradient carries
// cond(C)^2); the products with C, R and Z are FP32-accurate 3xTF32
// products on the tensor cores.
int backward_run(const float* A, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const float* Z,
                 int64_t ldz, const float* dZ, int64_t lddz, float* dA, int64_t ldda, void* ws, DevInfo* dinfo,
                 cudaStream_t s) {
    const BwdLayout L = bwd_layout(m, n, k);
    char* base = static_cast<char*>(ws);
    int* flag = reinterpret_cast<int*>(base + L.flag);
    int* gst = flag + 1;
    unsigned char* mask = reinterpret_cast<unsigned char*>(base + L.mask);
    float* C32 = reinterpret_cast<float*>(base + L.C32);
    double* Gp = reinterpret_cast<double*>(base + L.Gp);
    double* Wa = reinterpret_cast<double*>(base + L.Wa);
    double* Uinv64 = reinterpret_cast<double*>(base + L.Uinv64);
    double* G64 = reinterpret_cast<double*>(base + L.G64);
    double* Y64 = reinterpret_cast<double*>(base + L.Y64);
    float* W32 = reinterpret_cast<float*>(base + L.W32);
    float* R = reinterpret_cast<float*>(base + L.R);
    float* dC = reinterpret_cast<float*>(base + L.dC);
    float* M1 = reinterpret_cast<float*>(base + L.M1);
    void* gws = base + L.gws;
    const int M = (int)m, N = (int)n;
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    if (cudaMemsetAsync(mask, 0, (size_t)n, s) != cudaSuccess) return ID_ECUDA;
    const int tr = trace_begin(TraceKind::kRefine, s);
    if (factor_skeleton(A, m, n, lda, k, J, C32, Gp, Wa, Uinv64, reinterpret_cast<double*>(base + L.gdiag), flag, s) !=
        cudaSuccess)
        return ID_ECUDA;
    k_mask_j<<<1, kRThreads, 0, s>>>(J, k, n, mask);
    dim3 g2(ceil_div(n, kRThreads) < 1024 ? ceil_div(n, kRThreads) : 1024, k);
    k_gz<<<g2, kRThreads, 0, s>>>(dZ, lddz, k, N, mask, G64);
    // W = U^{-1} (U^{-T} G) in FP64 (Uinv64 is U^{-1} row-major)
    if (dgemm(1, 0, k, N, k, 1.0, Uinv64, k, G64, n, 0.0, Y64, n, s) != cudaSuccess) return ID_ECUDA;
    if (dgemm(0, 0, k, N, k, 1.0, Uinv64, k, Y64, n, 0.0, G64, n, s) != cudaSuccess) return ID_ECUDA;
    k_to_f32<<<grid_for((int64_t)k * n), kRThreads, 0, s>>>(G64, W32, (int64_t)k * n);
    int rc;
    // dA = C W (m x n)
    if ((rc = gemm_f32(0, 0, M, N, k, 1.0f, C32, k, W32, n, 0.0f, dA, ldda, gws, gst, s)) != ID_OK) return rc;
    // R = A - C Z (m x n)
    if ((rc = gemm_f32_ex(0, 0, M, N, k, -1.0f, C32, k, Z, ldz, 1.0f, A, lda, R, n, gws, gst, s)) != ID_OK) return rc;
    // dC = R W^T (m x k)
    if ((rc = gemm_f32(0, 1, M, k, N, 1.0f, R, n, W32, n, 0.0f, dC, k, gws, gst, s)) != ID_OK) return rc;
    // M1 = W Z^T (k x k), then dC -= C M1
    if ((rc = gemm_f32(0, 1, k, k, N, 1.0f, W32, n, Z, ldz, 0.0f, M1, k, gws, gst, s)) != ID_OK) return rc;
    if ((rc = gemm_f32(0, 0, M, k, k, -1.0f, C32, k, M1, k, 1.0f, dC, k, gws, gst, s)) != ID_OK) return rc;
    k_scatter_dc<<<grid_for(m * k), kRThreads, 0, s>>>(dC, M, k, J, n, dA, ldda);
    k_bwd_finalize<<<1, 1, 0, s>>>(dinfo, flag);
    trace_end(tr, s);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

// ------------------------------------------------------ reconstruction C Z --
// S = A[:, J] (m x k row-major) or, for a row ID, S = A[J, :] (k x n
// row-major). An index outside its range sets flag[0] = 2 and gathers zeros.
template <typename T>
__global__ void k_gather_skel(const T* __restrict__ A, int64_t lda, int m, int n, int k, const int32_t* __restrict__ J,
                              int rows, T* __restrict__ S, int* flag) {
    const int64_t total = rows ? (int64_t)k * n : (int64_t)m * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (rows) {
            const int c = (int)(e / n), l = (int)(e % n);
            const int r = J[c];
            const bool ok = r >= 0 && r < m;
            if (!ok && l == 0) flag[0] = 2;
            S[e] = ok ? A[(int64_t)r * lda + l] : T(0);
        } else {
            const int64_t i = e / k;
            const int c = (int)(e % k);
            const int l = J[c];
            const bool ok = l >= 0 && l < n;
            if (!ok && i == 0) flag[0] = 2;
            S[e] = ok ? A[i * lda + l] : T(0);
        }
    }
}

template <typename T>
cudaError_t gather_skeleton(const void* A, int64_t lda, int64_t m, int64_t n, int k, const int32_t* idx, int rows,
                            void* S, int* flag, cudaStream_t s) {
    k_gather_skel<T><<<grid_for(rows ? (int64_t)k * n : m * k), kRThreads, 0, s>>>(
        static_cast<const T*>(A), lda, (int)m, (int)n, k, idx, rows, static_cast<T*>(S), flag);
    return cudaGetLastError();
}
template cudaError_t gather_skeleton<double>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, int, void*,
                                             int*, cudaStream_t);
template cudaError_t gather_skeleton<float>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, int, void*,
                                            int*, cudaStream_t);

// An ID of a k x k matrix keeps everything: idx = 0..k-1, Zx = I (k x k, ld ldz);
// info: status ID_OK, rank k, Z statistics of the identity.
template <typename T>
__global__ void k_identity_id(int32_t* idx, T* Zx, int64_t ldz, int k, DevInfo* info) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
        const int r = e / k, c = e % k;
        Zx[(int64_t)r * ldz + c] = r == c ? T(1) : T(0);
        if (r == 0) idx[c] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        id_info z = {};
        z.rank = k;
        z.max_abs_z = 1.0;
        z.engine = 1;
        z.err_est = 0.0;   // an ID of a k x k matrix is exact
        info->info = z;
    }
}

template <typename T>
cudaError_t identity_id(int32_t* idx, void* Zx, int64_t ldz, int k, DevInfo* info, cudaStream_t s) {
    k_identity_id<T><<<grid_for((int64_t)k * k), kRThreads, 0, s>>>(idx, static_cast<T*>(Zx), ldz, k, info);
    return cudaGetLastError();
}
template cudaError_t identity_id<double>(int32_t*, void*, int64_t, int, DevInfo*, cudaStream_t);
template cudaError_t identity_id<float>(int32_t*, void*, int64_t, int, DevInfo*, cudaStream_t);

__global__ void k_recon_finalize(DevInfo* info, const int* flag) {
    id_info r = {};
    r.status = flag[0] == 2 ? ID_EINVAL : ((flag[1] & kStatTimeout) ? ID_ETIMEOUT : ID_OK);
    r.err_est = -1.0;
    info->info = r;
}

size_t reconstruct_bytes(int64_t m, int64_t n, int64_t k, int rows, size_t s) {
    return al(16) + al(s * (size_t)k * (size_t)(rows ? n : m)) + (s == 4 ? gemm_f32_bytes((int)m, (int)n, (int)k) : 0);
}

template <typename T>
int reconstruct_run(const void* Av, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const void* Zv,
                    int64_t ldz, int rows, void* Outv, int64_t ldo, void* ws, DevInfo* dinfo, cudaStream_t s) {
    char* base = static_cast<char*>(ws);
    int* flag = reinterpret_cast<int*>(base);
    T* S = reinterpret_cast<T*>(base + al(16));
    char* gws = base + al(16) + al(sizeof(T) * (size_t)k * (size_t)(rows ? n : m));
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    const T* A = static_cast<const T*>(Av);
    k_gather_skel<T><<<grid_for(rows ? (int64_t)k * n : m * k), kRThreads, 0, s>>>(A, lda, (int)m, (int)n, k, J, rows,
                                                                                  S, flag);
    // Column ID: Out (m x n) = S (m x k) Z (k x n). Row ID: Out = Z^T (m x k; Z is k x m) S (k x n).
    const int M = (int)m, N = (int)n;
    if (sizeof(T) == 8) {
        const double* Z = static_cast<const double*>(Zv);
        const double* Sd = reinterpret_cast<const double*>(S);
        double* Out = static_cast<double*>(Outv);
        const cudaError_t e = rows ? dgemm(1, 0, M, N, k, 1.0, Z, ldz, Sd, n, 0.0, Out, ldo, s)
                                   : dgemm(0, 0, M, N, k, 1.0, Sd, k, Z, ldz, 0.0, Out, ldo, s);
        if (e != cudaSuccess) return ID_ECUDA;
    } else {
        const float* Z = static_cast<const float*>(Zv);
        const float* Sf = reinterpret_cast<const float*>(S);
        float* Out = static_cast<float*>(Outv);
        const int rc = rows ? gemm_f32(1, 0, M, N, k, 1.0f, Z, ldz, Sf, n, 0.0f, Out, ldo, gws, flag + 1, s)
                            : gemm_f32(0, 0, M, N, k, 1.0f, Sf, k, Z, ldz, 0.0f, Out, ldo, gws, flag + 1, s);
        if (rc != ID_OK) return rc;
    }
    k_recon_finalize<<<1, 1, 0, s>>>(dinfo, flag);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

template int reconstruct_run<double>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, const void*, int64_t,
                                     int, void*, int64_t, void*, DevInfo*, cudaStream_t);
template int reconstruct_run<float>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, const void*, int64_t,
                                    int, void*, int64_t, void*, DevInfo*, cudaStream_t);

// ------------------------------------------------ column-sampling Optim RID --
struct SampLayout {
    size_t flag, C32, Gp, gdiag, Wa, Uinv64, M64, C64, B64, Z64, total;
};

static SampLayout samp_layout(int64_t m, int64_t n, int64_t k) {
    SampLayout L;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = al(off + b);
        return o;
    };
    L.flag = take(16);
    L.C32 = take(4 * (size_t)m * k);
    L.Gp = take(8 * (size_t)kGramSplit * k * k);
    L.gdiag = take(8 * (size_t)k);
    L.Wa = take(8 * (size_t)k * 2 * k);
    L.Uinv64 = take(8 * (size_t)k * k);
    L.M64 = take(8 * (size_t)k * k);
    L.C64 = take(8 * (size_t)m * k);
    L.B64 = take(8 * (size_t)k * n);
    L.Z64 = take(8 * (size_t)k * n);
    L.total = off;
    return L;
}

size_t sampled_z_bytes(int64_t m, int64_t n, int64_t k) { return samp_layout(m, n, k).total; }

template <typename T>
cudaError_t sample_gather_run(const void* A, int64_t lda, int m, const int32_t* idx, int p, void* W, int ldw,
                              cudaStream_t s) {
    k_gather_sample<T><<<grid_for((int64_t)ldw * p), kRThreads, 0, s>>>(static_cast<const T*>(A), lda, m, idx, p,
                                                                      static_cast<T*>(W), ldw);
    return cudaGetLastError();
}

cudaError_t sample_map_j(const int* perm, const int32_t* idx, int k, int32_t* J, cudaStream_t s) {
    k_map_j<<<ceil_div(k, kRThreads), kRThreads, 0, s>>>(perm, idx, k, J);
    return cudaGetLastError();
}

// Z of Optim RID: R_k^T R_k Z = C^T A in FP64. FP64 data: R_k is the CPQR's own
// factor (the paper's route) and B = C^T A is an FP64 product. FP32 data: the
// CPQR's R_k carries FP32 rounding, which the normal equations would square,
// so U with U^T U = C^T C is formed from C itself (exact products,
// double-float sums, FP64 Cholesky) -- the same matrix in exact arithmetic --
// and B = C^T A comes from k_ctb (exact products, double-float sums). Then
// M = U^{-1} U^{-T} and Z = M B in FP64; Z[:, J] is set to the identity it
// equals in exact arithmetic.
template <typename T>
int sampled_z_run(const void* Av, int64_t m, int64_t n, int64_t lda, int k, const int32_t* J, const void* W, int ldw,
                  void* Zv, int64_t ldz, void* ws, DevInfo* dinfo, cudaStream_t s) {
    const T* A = static_cast<const T*>(Av);
    T* Z = static_cast<T*>(Zv);
    const SampLayout L = samp_layout(m, n, k);
    char* base = static_cast<char*>(ws);
    int* flag = reinterpret_cast<int*>(base + L.flag);
    double* Wa = reinterpret_cast<double*>(base + L.Wa);
    double* Uinv64 = reinterpret_cast<double*>(base + L.Uinv64);
    double* M64 = reinterpret_cast<double*>(base + L.M64);
    double* C64 = reinterpret_cast<double*>(base + L.C64);
    double* B64 = reinterpret_cast<double*>(base + L.B64);
    double* Z64 = reinterpret_cast<double*>(base + L.Z64);
    const int N = (int)n;
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    const int tr = trace_begin(TraceKind::kSampledZ, s);
    if (sizeof(T) == 8) {
        const double* A64 = reinterpret_cast<const double*>(Av);
        k_rk_identity<T><<<grid_for((int64_t)2 * k * k), kRThreads, 0, s>>>(static_cast<const T*>(W), ldw, k, Wa);
        if (tri_inverse(Wa, k, Wa + (size_t)k * k, reinterpret_cast<double*>(base + L.Gp), Uinv64, s) != cudaSuccess)
            return ID_ECUDA;
        k_gather_f64<T><<<grid_for(m * k), kRThreads, 0, s>>>(A, lda, (int)m, k, J, C64);
        // B = C^T A (k x n)
        if (dgemm(1, 0, k, N, (int)m, 1.0, C64, k, A64, lda, 0.0, B64, n, s) != cudaSuccess) return ID_ECUDA;
    } else {
        float* C32 = reinterpret_cast<float*>(base + L.C32);
        if (factor_skeleton(reinterpret_cast<const float*>(A), m, n, lda, k, J, C32,
                            reinterpret_cast<double*>(base + L.Gp), Wa, Uinv64,
                            reinterpret_cast<double*>(base + L.gdiag), flag, s) != cudaSuccess)
            return ID_ECUDA;
        k_ctb<<<dim3(ceil_div(n, kGT), ceil_div(k, kGT)), 256, 0, s>>>(C32, reinterpret_cast<const float*>(A), lda,
                                                                       (int)m, k, N, B64);
    }
    // M = U^{-1} U^{-T} (= (C^T C)^{-1}), then Z = M B (k x n)
    if (dgemm(0, 1, k, k, k, 1.0, Uinv64, k, Uinv64, k, 0.0, M64, k, s) != cudaSuccess) return ID_ECUDA;
    double* Zd = sizeof(T) == 8 ? reinterpret_cast<double*>(Zv) : Z64;
    const int64_t ldzd = sizeof(T) == 8 ? ldz : n;
    if (dgemm(0, 0, k, N, k, 1.0, M64, k, B64, n, 0.0, Zd, ldzd, s) != cudaSuccess) return ID_ECUDA;
    dim3 g2(ceil_div(n, kRThreads) < 1024 ? ceil_div(n, kRThreads) : 1024, k);
    dim3 g8(ceil_div(n, kRThreads * 8), k);
    if (sizeof(T) == 4) k_z_from64<T><<<g2, kRThreads, 0, s>>>(Z64, k, N, Z, ldz);
    k_identity_at_j<T><<<grid_for((int64_t)k * k), kRThreads, 0, s>>>(Z, ldz, J, k);
    k_zstats_t<T><<<g8, kRThreads, 0, s>>>(Z, ldz, k, N, dinfo);
    k_sampled_finalize<<<1, 1, 0, s>>>(dinfo, flag);
    trace_end(tr, s);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

template cudaError_t sample_gather_run<double>(const void*, int64_t, int, const int32_t*, int, void*, int,
                                               cudaStream_t);
template cudaError_t sample_gather_run<float>(const void*, int64_t, int, const int32_t*, int, void*, int, cudaStream_t);
template int sampled_z_run<double>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, const void*, int,
                                   void*, int64_t, void*, DevInfo*, cudaStream_t);
template int sampled_z_run<float>(const void*, int64_t, int64_t, int64_t, int, const int32_t*, const void*, int,
                                  void*, int64_t, void*, DevInfo*, cudaStream_t);

}  // namespace gbid
