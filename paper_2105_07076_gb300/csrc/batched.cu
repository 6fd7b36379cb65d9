// Batched ID: many small, unevenly sized matrices in one persistent launch
// (Sec. 2.1 applied to every matrix of the batch independently).
//
// The grid is sized to the resident capacity of the GPU; each CTA takes
// problems from an atomic queue and runs the whole ID of one matrix:
//   1. X (A, or A^T when m > n: the Sec. 2 footnote) is copied column-major
//      into the problem's scratch W; column norms give the first pivot.
//   2. k Householder steps, right-looking and unblocked. Columns are never
//      moved: perm maps positions to columns of W. Warp 0 forms the
//      reflector of the pivot column (beta = -sign(x_j) ||x||, v_j = 1,
//      tau = (beta - x_j) / beta); then every warp updates a group of
//      trailing columns held in registers, W(j:m, l) -= tau v (v^T W(j:m, l)),
//      and takes the EXACT squared residual norm ||W(j+1:m, l)||^2 of the
//      updated column (the data are already in registers, so this costs what
//      a downdate would; squares of y / 2^e, 2^e near the largest column
//      norm, summed in the working precision) for the next pivot's argmax
//      (ties: smallest original column index).
//   3. T = R11^{-1} R12 by back substitution (R11 staged in shared memory;
//      a warp solves four right-hand sides at a time, lane = row), in FP64
//      for FP64 data and in double-float arithmetic (about 48 bits, on the
//      FP32 pipe) for FP32 data, written straight into Z through perm;
//      Z[:, J] = I, J = perm[0:k].
// Per-problem status (argument check, non-finite input, numerical rank) goes
// to that problem's id_info. Nothing waits on another CTA: the only shared
// state is the queue counter.
//
// The kernel is instantiated for several tile shapes (threads per CTA,
// trailing columns per warp, rows a lane holds per pass, resident CTAs per
// SM). Every instance performs the same operations in the same order on
// every element: a lane always sums its rows j + lane + 32q in increasing q,
// the warp and block reductions are fixed butterflies or exact comparisons,
// and one warp solves each column of T. So all instances give bit-identical
// J, Z and id_info, and id_batched_autotune may time them on the caller's
// batch and keep the fastest.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "cpqr.cuh"
#include "gbid.h"
#include "trace.cuh"

namespace gbid {
namespace {

constexpr int kBMaxWarps = 16;               // up to 512 threads per CTA
constexpr int kBRows = 8;                    // rows per lane per pass of the reflector (256-row chunks)
constexpr int kBCopy = 16;                   // loads in flight per thread in the copy-in
constexpr int kBMaxK = ID_BATCHED_MAX_K;
constexpr int kBMaxM = ID_BATCHED_MAX_MIN_DIM;

__host__ __device__ inline size_t b_align(size_t x) { return (x + 255) & ~size_t(255); }

// R11 (upper triangular, k <= kBMaxK) packed by columns in shared memory:
// entry (r, i), r <= i, at i (i + 1) / 2 + r. Lanes reading one column take
// consecutive words.
constexpr int kBR11 = kBMaxK * (kBMaxK + 1) / 2;
__device__ __forceinline__ int rp(int r, int i) { return i * (i + 1) / 2 + r; }

// x <- x - r b on unevaluated float pairs (hi + lo), about 48 significant
// bits: r b by Dekker's product (the FMA gives hi's rounding error exactly),
// the difference by Knuth's TwoSum, renormalised by Dekker's FastTwoSum. The
// _rn intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void df_sub_mul(float& xh, float& xl, float rh, float rl, float bh, float bl) {
    const float p = __fmul_rn(rh, bh);
    float pe = __fmaf_rn(rh, bh, -p);
    pe = __fmaf_rn(rh, bl, pe);
    pe = __fmaf_rn(rl, bh, pe);
    const float s = __fsub_rn(xh, p);
    const float v = __fsub_rn(s, xh);
    float e = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, v)), __fsub_rn(-p, v));
    e = __fadd_rn(e, __fsub_rn(xl, pe));
    const float nh = __fadd_rn(s, e);
    xl = __fsub_rn(e, __fsub_rn(nh, s));
    xh = nh;
}

struct BLayout {
    size_t perm, total;
    int ldw;
};

__host__ __device__ inline BLayout b_layout(int s, int64_t mx, int64_t nx) {
    BLayout L;
    L.ldw = (int)((mx + 3) / 4 * 4);
    L.perm = b_align((size_t)s * L.ldw * nx);
    L.total = L.perm + b_align(4 * (size_t)nx);
    return L;
}

template <int NW>
__device__ ArgMax b_block_argmax(ArgMax a, ArgMax* red) {
    a = warp_argmax(a);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    __syncthreads();
    if (lane == 0) red[w] = a;
    __syncthreads();
    a = lane < NW ? red[lane] : empty_argmax();
    return warp_argmax(a);
}

template <int NW>
__device__ double b_block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < NW ? red[lane] : 0.0;
    return warp_sum(v);
}

template <int NW>
__device__ double b_block_max(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < NW ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Pivot candidate in the working precision: the SQUARED residual norm (same
// order as the norm, no square root), ties to the smaller original index.
// Comparing in T keeps the per-column epilogue off the FP64 pipe, which on
// this GPU runs one warp instruction per 16 clocks per SM.
template <typename T>
struct Cand {
    T val;
    int orig, pos;
};

template <typename T>
__device__ __forceinline__ Cand<T> cand_empty() {
    Cand<T> c;
    c.val = T(-1);
    c.orig = 0x7fffffff;
    c.pos = -1;
    return c;
}

template <typename T>
__device__ __forceinline__ bool cand_better(const Cand<T>& a, const Cand<T>& b) {
    return a.val > b.val || (a.val == b.val && a.orig < b.orig);
}

template <typename T>
__device__ __forceinline__ ArgMax cand_to_argmax(const Cand<T>& c) {
    ArgMax a;
    a.val = (double)c.val;
    a.orig = c.orig;
    a.pos = c.pos;
    return a;
}

// Trailing update of the CG columns at positions pos0 .. pos0+CG-1 (those
// below nx) by one warp, and their exact squared residual norms on rows
// j+1..mx-1.
// The squares are taken of y * ysc, ysc a power of two near 1 / max column
// norm, so they neither overflow nor underflow in the working precision.
template <typename T, int CG, int R>
__device__ void b_update_group(T* W, int ldw, const int* perm, int mx, int nx, int j, int pos0, T tauT, T ysc,
                               const T* v_s, Cand<T>& best) {
    const int lane = threadIdx.x % kWarp;
    int col[CG];
    bool ok[CG];
#pragma unroll
    for (int g = 0; g < CG; ++g) {
        ok[g] = pos0 + g < nx;
        col[g] = ok[g] ? perm[pos0 + g] : 0;
    }
    T d[CG];
    T ss[CG];   // sums of squares in the working precision (at most 8 terms per lane per chunk)
#pragma unroll
    for (int g = 0; g < CG; ++g) {
        d[g] = T(0);
        ss[g] = T(0);
    }
    if (mx - j <= kWarp * R) {
        // the whole column segment fits in registers: one read, one write
        T x[CG][R];
#pragma unroll
        for (int g = 0; g < CG; ++g)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = j + lane + kWarp * q;
                x[g][q] = (ok[g] && i < mx) ? W[(int64_t)col[g] * ldw + i] : T(0);
            }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = j + lane + kWarp * q;
            const T vi = i < mx ? v_s[i] : T(0);
#pragma unroll
            for (int g = 0; g < CG; ++g) d[g] += vi * x[g][q];
        }
#pragma unroll
        for (int g = 0; g < CG; ++g) d[g] = warp_sum(d[g]);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = j + lane + kWarp * q;
            if (i < mx) {
                const T vi = v_s[i];
#pragma unroll
                for (int g = 0; g < CG; ++g) {
                    const T y = x[g][q] - (tauT * d[g]) * vi;
                    if (ok[g]) W[(int64_t)col[g] * ldw + i] = y;
                    if (i > j) ss[g] += (y * ysc) * (y * ysc);
                }
            }
        }
    } else {
        for (int i0 = j; i0 < mx; i0 += kWarp * R) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = i0 + lane + kWarp * q;
                if (i < mx) {
                    const T vi = v_s[i];
#pragma unroll
                    for (int g = 0; g < CG; ++g)
                        if (ok[g]) d[g] += vi * W[(int64_t)col[g] * ldw + i];
                }
            }
        }
#pragma unroll
        for (int g = 0; g < CG; ++g) d[g] = warp_sum(d[g]);
        for (int i0 = j; i0 < mx; i0 += kWarp * R) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = i0 + lane + kWarp * q;
                if (i < mx) {
                    const T vi = v_s[i];
#pragma unroll
                    for (int g = 0; g < CG; ++g) {
                        if (!ok[g]) continue;
                        T* p = W + (int64_t)col[g] * ldw + i;
                        const T y = *p - (tauT * d[g]) * vi;
                        *p = y;
                        if (i > j) ss[g] += (y * ysc) * (y * ysc);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < CG; ++g) {
        const T s = warp_sum(ss[g]);
        if (ok[g]) {
            Cand<T> c;
            c.val = isfinite(s) ? s : T(-1);
            c.orig = col[g];
            c.pos = pos0 + g;
            if (cand_better(c, best)) best = c;
        }
    }
}

// TH threads per CTA, CG trailing columns per warp and pass, R rows per lane
// per pass (column segments of up to 32 R rows stay in registers), MINB the
// resident CTAs per SM the register budget is cut for.
template <typename T, int TH, int CG, int R, int MINB>
__global__ void __launch_bounds__(TH, MINB) k_id_batched(const id_problem* __restrict__ probs, int count,
                                                      unsigned* queue, id_info* __restrict__ infos) {
    constexpr int kBThreads = TH;
    constexpr int kBWarps = TH / kWarp;
    static_assert(TH % kWarp == 0 && kBWarps <= kBMaxWarps, "threads per CTA");
    const double eps = sizeof(T) == 8 ? DBL_EPSILON : (double)FLT_EPSILON;
    __shared__ T v_s[kBMaxM];
    __shared__ double r11[kBR11];
    __shared__ double rinv[kBMaxK];
    __shared__ ArgMax red_a[kBMaxWarps];
    __shared__ double red_d[kBMaxWarps];
    __shared__ double sc[2];
    __shared__ int s_b;
    const int t = threadIdx.x, lane = t % kWarp, w = t / kWarp;

    for (;;) {
        __syncthreads();
        if (t == 0) s_b = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int b = s_b;
        if (b >= count) break;
        const id_problem pr = probs[b];
        const int64_t mn = pr.m < pr.n ? pr.m : pr.n;
        const bool valid = pr.A && pr.J && pr.Z && pr.work && pr.m >= 1 && pr.n >= 1 && pr.k >= 1 && pr.k <= mn &&
                           pr.k <= kBMaxK && mn <= kBMaxM && pr.lda >= pr.n &&
                           pr.ldz >= (pr.m > pr.n ? pr.m : pr.n) && (reinterpret_cast<uintptr_t>(pr.work) & 255) == 0;
        if (!valid) {
            if (t == 0) {
                id_info r = {};
                r.status = ID_EINVAL;
                r.err_est = -1.0;
                infos[b] = r;
            }
            continue;
        }
        const bool trans = pr.m > pr.n;
        const int mx = (int)mn, nx = (int)(trans ? pr.m : pr.n), k = (int)pr.k;
        const BLayout L = b_layout(sizeof(T), mx, nx);
        const int ldw = L.ldw;
        T* W = static_cast<T*>(pr.work);
        int* perm = reinterpret_cast<int*>(static_cast<char*>(pr.work) + L.perm);
        const T* A = static_cast<const T*>(pr.A);

        // 1. X -> W (column-major) with the column norms and the first pivot;
        //    kBCopy loads in flight per thread
        ArgMax best = empty_argmax();
        int nonfinite = 0;
        if (!trans) {
            // thread per column: the rows of A are read coalesced across the warp
            for (int l = t; l < nx; l += kBThreads) {
                double s = 0.0;
                for (int i0 = 0; i0 < mx; i0 += kBCopy) {
                    T v[kBCopy];
#pragma unroll
                    for (int q = 0; q < kBCopy; ++q)
                        v[q] = i0 + q < mx ? A[(int64_t)(i0 + q) * pr.lda + l] : T(0);
#pragma unroll
                    for (int q = 0; q < kBCopy; ++q) {
                        if (i0 + q < mx) W[(int64_t)l * ldw + i0 + q] = v[q];
                        s = fma((double)v[q], (double)v[q], s);
                    }
                }
                perm[l] = l;
                if (!isfinite(s)) nonfinite = 1;
                ArgMax c;
                c.val = isfinite(s) ? s : -1.0;
                c.orig = l;
                c.pos = l;
                if (better(c, best)) best = c;
            }
        } else {
            // warp per column of X = row of A (contiguous)
            for (int l = w; l < nx; l += kBWarps) {
                double s = 0.0;
                for (int i0 = lane; i0 < mx; i0 += kWarp * kBCopy) {
                    T v[kBCopy];
#pragma unroll
                    for (int q = 0; q < kBCopy; ++q) {
                        const int i = i0 + kWarp * q;
                        v[q] = i < mx ? A[(int64_t)l * pr.lda + i] : T(0);
                    }
#pragma unroll
                    for (int q = 0; q < kBCopy; ++q) {
                        const int i = i0 + kWarp * q;
                        if (i < mx) W[(int64_t)l * ldw + i] = v[q];
                        s = fma((double)v[q], (double)v[q], s);
                    }
                }
                s = warp_sum(s);
                if (lane == 0) {
                    perm[l] = l;
                    if (!isfinite(s)) nonfinite = 1;
                    ArgMax c;
                    c.val = isfinite(s) ? s : -1.0;
                    c.orig = l;
                    c.pos = l;
                    if (better(c, best)) best = c;
                }
            }
        }
        nonfinite = __syncthreads_or(nonfinite);
        best = b_block_argmax<kBWarps>(best, red_a);
        T ysc = T(1);
        if (best.val > 0.0) {
            int e2;
            frexp(sqrt(best.val), &e2);
            ysc = (T)ldexp(1.0, -e2);
        }

        // 2. k Householder steps
        double r00 = 0.0;
        int rank = k;
        const double rank_tol = sqrt((double)nx) * eps;   // |R_jj| <= sqrt(max(m, n)) eps |R_00|
        for (int j = 0; j < k; ++j) {
            const int p = best.pos >= j ? best.pos : j;
            if (t == 0 && p != j) {
                const int a = perm[j];
                perm[j] = perm[p];
                perm[p] = a;
            }
            __syncthreads();
            T* xj = W + (int64_t)perm[j] * ldw;
            if (w == 0) {
                double ss = 0.0;
                for (int i0 = j + 1 + lane; i0 < mx; i0 += kWarp * kBRows) {
                    T v[kBRows];
#pragma unroll
                    for (int q = 0; q < kBRows; ++q) v[q] = i0 + kWarp * q < mx ? xj[i0 + kWarp * q] : T(0);
#pragma unroll
                    for (int q = 0; q < kBRows; ++q) ss = fma((double)v[q], (double)v[q], ss);
                }
                ss = warp_sum(ss);
                const double x0 = (double)xj[j];
                const double alpha = sqrt(fma(x0, x0, ss));
                double beta = 0.0, tau = 0.0, scale = 0.0;
                if (alpha != 0.0) {
                    beta = x0 >= 0.0 ? -alpha : alpha;
                    tau = (beta - x0) / beta;
                    scale = 1.0 / (x0 - beta);
                }
                const T scaleT = (T)scale;
                for (int i0 = j + 1 + lane; i0 < mx; i0 += kWarp * kBRows) {
                    T v[kBRows];
#pragma unroll
                    for (int q = 0; q < kBRows; ++q) v[q] = i0 + kWarp * q < mx ? xj[i0 + kWarp * q] : T(0);
#pragma unroll
                    for (int q = 0; q < kBRows; ++q) {
                        const int i = i0 + kWarp * q;
                        if (i < mx) {
                            xj[i] = v[q] * scaleT;
                            v_s[i] = v[q] * scaleT;
                        }
                    }
                }
                if (lane == 0) {
                    xj[j] = (T)beta;
                    v_s[j] = T(1);
                    sc[0] = beta;
                    sc[1] = tau;
                }
            }
            __syncthreads();
            const double beta = sc[0];
            if (j == 0) r00 = fabs(beta);
            if (rank == k && (r00 == 0.0 || fabs(beta) <= rank_tol * r00)) rank = j;
            const T tauT = (T)sc[1];
            // the last step still updates: it writes row k-1 of R12. Column segments
            // of up to 32 R rows stay in registers CG columns at a time, up to 64 R
            // rows CG / 2 columns at a time; longer ones take two passes.
            Cand<T> bw = cand_empty<T>();
            if (mx - j > kWarp * R && mx - j <= 2 * kWarp * R) {
                constexpr int CG2 = CG > 1 ? CG / 2 : 1;
                for (int pos0 = j + 1 + w * CG2; pos0 < nx; pos0 += kBWarps * CG2)
                    b_update_group<T, CG2, 2 * R>(W, ldw, perm, mx, nx, j, pos0, tauT, ysc, v_s, bw);
            } else {
                for (int pos0 = j + 1 + w * CG; pos0 < nx; pos0 += kBWarps * CG)
                    b_update_group<T, CG, R>(W, ldw, perm, mx, nx, j, pos0, tauT, ysc, v_s, bw);
            }
            best = b_block_argmax<kBWarps>(cand_to_argmax(bw), red_a);   // its barriers also order this step's writes
        }

        // 3. T = R11^{-1} R12 (FP64), Z, J
        for (int e0 = t; e0 < k * k; e0 += 4 * kBThreads) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kBThreads, i = e / k, q = e % k;
                v[u] = (e < k * k && i <= q) ? (double)W[(int64_t)perm[q] * ldw + i] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * kBThreads;
                if (e < k * k && e / k <= e % k) r11[rp(e / k, e % k)] = v[u];
            }
        }
        __syncthreads();
        for (int i = t; i < k; i += kBThreads) rinv[i] = 1.0 / r11[rp(i, i)];
        __syncthreads();
        // R(r, i) / R(i, i) above the diagonal: the substitution then needs one
        // FMA per step, b_r -= (R(r,i) / R(i,i)) b_i, and one scaling at the end.
        // FP32 data: the ratio is kept as a float pair in the same slot, and the
        // substitution runs in double-float arithmetic on the FP32 pipe (about
        // 48 bits, far below the FP32 data's own rounding; the FP64 pipe does
        // one warp instruction per 16 clocks per SM on this GPU).
        for (int e = t; e < k * k; e += kBThreads) {
            const int r = e / k, i = e % k;
            if (r < i) {
                const double d = r11[rp(r, i)] * rinv[i];
                if constexpr (sizeof(T) == 4) {
                    const float hi = (float)d;
                    reinterpret_cast<float2*>(r11)[rp(r, i)] = make_float2(hi, (float)(d - (double)hi));
                } else {
                    r11[rp(r, i)] = d;
                }
            }
        }
        __syncthreads();
        T* Z = static_cast<T*>(pr.Z);
        const int64_t ldz = pr.ldz;
        T zmax = T(1);                  // the identity block holds ones
        float gt2 = 0.0f;
        for (int l0 = k + 4 * w; l0 < nx; l0 += 4 * kBWarps) {
            T xv[4][2];
            int colq[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int l = l0 + qq;
                colq[qq] = l < nx ? perm[l] : -1;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int i = lane + kWarp * s;
                    xv[qq][s] = (colq[qq] >= 0 && i < k) ? W[(int64_t)colq[qq] * ldw + i] : T(0);
                }
            }
            // b_i (final once rows > i are applied) is broadcast; rows below 32
            // only when k > 32; x = b / diag(R) at the end
            const bool two = k > kWarp;
            double x[4][2];
            if constexpr (sizeof(T) == 4) {
                float xl[4][2];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) xl[qq][0] = xl[qq][1] = 0.0f;
                const float2* r11f = reinterpret_cast<const float2*>(r11);
                for (int i = k - 1; i >= 0; --i) {
                    const int own = i % kWarp, sl = i / kWarp;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const float bh = __shfl_sync(0xffffffffu, sl ? xv[qq][1] : xv[qq][0], own);
                        const float bl = __shfl_sync(0xffffffffu, sl ? xl[qq][1] : xl[qq][0], own);
                        if (lane < i) {
                            const float2 r = r11f[rp(lane, i)];
                            df_sub_mul(xv[qq][0], xl[qq][0], r.x, r.y, bh, bl);
                        }
                        if (two && lane + kWarp < i) {
                            const float2 r = r11f[rp(lane + kWarp, i)];
                            df_sub_mul(xv[qq][1], xl[qq][1], r.x, r.y, bh, bl);
                        }
                    }
                }
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
#pragma unroll
                    for (int s = 0; s < 2; ++s) x[qq][s] = (double)xv[qq][s] + (double)xl[qq][s];
            } else {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
#pragma unroll
                    for (int s = 0; s < 2; ++s) x[qq][s] = (double)xv[qq][s];
                for (int i = k - 1; i >= 0; --i) {
                    const int own = i % kWarp, sl = i / kWarp;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const double bi = __shfl_sync(0xffffffffu, sl ? x[qq][1] : x[qq][0], own);
                        if (lane < i) x[qq][0] = fma(-r11[rp(lane, i)], bi, x[qq][0]);
                        if (two && lane + kWarp < i) x[qq][1] = fma(-r11[rp(lane + kWarp, i)], bi, x[qq][1]);
                    }
                }
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                x[qq][0] *= lane < k ? rinv[lane] : 0.0;
                if (two) x[qq][1] *= lane + kWarp < k ? rinv[lane + kWarp] : 0.0;
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                if (colq[qq] < 0) continue;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int i = lane + kWarp * s;
                    if (i < k) {
                        const T z = (T)x[qq][s];
                        Z[(int64_t)i * ldz + colq[qq]] = z;
                        const T a = fabs(z);
                        zmax = a == a ? fmax(zmax, a) : T(INFINITY);
                        if (a > T(2)) gt2 += 1.0f;
                    }
                }
            }
        }
        for (int e = t; e < k * k; e += kBThreads) {
            const int i = e / k, l = e % k;
            Z[(int64_t)i * ldz + perm[l]] = i == l ? T(1) : T(0);
        }
        for (int l = t; l < k; l += kBThreads) pr.J[l] = perm[l];
        const double zmax_b = b_block_max<kBWarps>((double)zmax, red_d);
        const double gt2_b = b_block_sum<kBWarps>((double)gt2, red_d);
        if (t == 0) {
            id_info r = {};
            r.status = nonfinite ? ID_ENONFINITE : (rank < k ? ID_RANK_DEFICIENT : ID_OK);
            r.rank = rank;
            r.transposed = trans ? 1 : 0;
            r.n_recompute = 0;
            r.n_gt2 = (int64_t)gt2_b;
            r.max_abs_z = zmax_b;
            r.r00 = r00;
            r.nb = 1;
            r.engine = 3;
            r.err_est = -1.0;
            infos[b] = r;
        }
    }
}

// The instances the tuner chooses from, one table per element type: {threads,
// columns per warp, rows per lane, CTAs per SM}. Entry 0 is the default.
using BatchedFn = void (*)(const id_problem*, int, unsigned*, id_info*);
struct BConfig {
    id_batched_config c;
    BatchedFn fn;
};

#define GBID_BCFG(T, TH, CG, R, MB) {{TH, CG, R, MB}, &k_id_batched<T, TH, CG, R, MB>}
const BConfig kBCfg32[] = {
    GBID_BCFG(float, 256, 4, 8, 3), GBID_BCFG(float, 256, 2, 8, 3), GBID_BCFG(float, 256, 8, 4, 3),
    GBID_BCFG(float, 256, 4, 4, 3), GBID_BCFG(float, 128, 4, 8, 5), GBID_BCFG(float, 256, 4, 8, 2),
    GBID_BCFG(float, 512, 4, 8, 1), GBID_BCFG(float, 128, 4, 8, 6), GBID_BCFG(float, 128, 2, 8, 8),
};
const BConfig kBCfg64[] = {
    GBID_BCFG(double, 256, 2, 8, 3), GBID_BCFG(double, 256, 1, 8, 3), GBID_BCFG(double, 256, 4, 4, 3),
    GBID_BCFG(double, 256, 2, 4, 3), GBID_BCFG(double, 128, 2, 8, 5), GBID_BCFG(double, 256, 2, 8, 2),
    GBID_BCFG(double, 512, 2, 8, 1), GBID_BCFG(double, 128, 2, 8, 6), GBID_BCFG(double, 128, 1, 8, 8),
};
#undef GBID_BCFG
constexpr int kBNumCfg = (int)(sizeof(kBCfg32) / sizeof(kBCfg32[0]));
static_assert(kBNumCfg == (int)(sizeof(kBCfg64) / sizeof(kBCfg64[0])), "one table size");

inline const BConfig* b_table(id_dtype dtype) {
    return dtype == ID_F64 ? kBCfg64 : dtype == ID_F32 ? kBCfg32 : nullptr;
}

int g_bnsm = 0;
int g_bocc[2][kBNumCfg] = {};
std::mutex g_bmu;

// Grid of one instance: the resident capacity (SMs x CTAs per SM that the
// occupancy calculator gives for it), or the problem count if smaller.
int batched_grid(id_dtype dtype, int cfg, int count) {
    const int slot = dtype == ID_F64 ? 0 : 1;
    const BConfig& b = b_table(dtype)[cfg];
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        if (g_bnsm == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&g_bnsm, cudaDevAttrMultiProcessorCount, dev);
        }
        if (g_bocc[slot][cfg] == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_bocc[slot][cfg], b.fn, b.c.threads, 0);
    }
    const int cap = g_bnsm * (g_bocc[slot][cfg] > 0 ? g_bocc[slot][cfg] : 1);
    return count < cap ? count : cap;
}

int check_batched(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                  size_t batch_work_bytes, id_info* infos, int config) {
    if (!b_table(dtype)) return ID_EINVAL;
    if (count < 0 || count > INT32_MAX) return ID_EINVAL;
    if (config < 0 || config >= kBNumCfg) return ID_EINVAL;
    if (count == 0) return ID_OK;
    if (!problems || !batch_work || !infos) return ID_EINVAL;
    if (batch_work_bytes < ID_BATCHED_WORK_BYTES) return ID_ENOMEM;
    return ID_OK;
}

// One memset (the queue counter) and one launch; arguments already checked.
int launch_batched(const id_problem* problems, int count, id_dtype dtype, unsigned* queue, id_info* infos,
                   int config, cudaStream_t s) {
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned), s) != cudaSuccess) return ID_ECUDA;
    const BConfig& b = b_table(dtype)[config];
    const int g = batched_grid(dtype, config, count);
    const int tr = trace_begin(TraceKind::kBatched, s);
    b.fn<<<g, b.c.threads, 0, s>>>(problems, count, queue, infos);
    trace_end(tr, s);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

}  // namespace
}  // namespace gbid

using namespace gbid;

extern "C" size_t id_batched_problem_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k) {
    if (dtype != ID_F64 && dtype != ID_F32) return 0;
    const int64_t mn = m < n ? m : n, mx = m < n ? n : m;
    if (m < 1 || n < 1 || k < 1 || k > mn || k > kBMaxK || mn > kBMaxM || mx > (int64_t)1 << 24) return 0;
    return b_layout(dtype == ID_F64 ? 8 : 4, mn, mx).total;
}

extern "C" int id_batched_config_count(id_dtype dtype) { return b_table(dtype) ? kBNumCfg : 0; }

extern "C" int id_batched_config_get(id_dtype dtype, int index, id_batched_config* out) {
    if (!b_table(dtype) || !out || index < 0 || index >= kBNumCfg) return ID_EINVAL;
    *out = b_table(dtype)[index].c;
    return ID_OK;
}

extern "C" int id_decompose_batched_with(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                                         size_t batch_work_bytes, id_info* infos, int config, void* stream) {
    const int rc = check_batched(problems, count, dtype, batch_work, batch_work_bytes, infos, config);
    if (rc != ID_OK || count == 0) return rc;
    return launch_batched(problems, (int)count, dtype, static_cast<unsigned*>(batch_work), infos, config,
                          static_cast<cudaStream_t>(stream));
}

extern "C" int id_decompose_batched(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                                    size_t batch_work_bytes, id_info* infos, void* stream) {
    return id_decompose_batched_with(problems, count, dtype, batch_work, batch_work_bytes, infos, 0, stream);
}

extern "C" int id_batched_autotune(const id_problem* problems, int64_t count, id_dtype dtype, void* batch_work,
                                   size_t batch_work_bytes, id_info* infos, int reps, float* ms_out, int* best,
                                   void* stream) {
    if (!best || reps < 1 || reps > 1000) return ID_EINVAL;
    const int rc = check_batched(problems, count, dtype, batch_work, batch_work_bytes, infos, 0);
    if (rc != ID_OK) return rc;
    if (count == 0) {
        *best = 0;
        if (ms_out)
            for (int c = 0; c < kBNumCfg; ++c) ms_out[c] = 0.0f;
        return ID_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned* queue = static_cast<unsigned*>(batch_work);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return ID_ECUDA;
    }
    int status = ID_OK, arg = 0;
    float best_ms = 0.0f;
    for (int c = 0; c < kBNumCfg && status == ID_OK; ++c) {
        // one untimed launch (first-use costs, the problems' scratch paged in), then reps timed back to back
        status = launch_batched(problems, (int)count, dtype, queue, infos, c, s);
        if (status == ID_OK && cudaEventRecord(e0, s) != cudaSuccess) status = ID_ECUDA;
        for (int r = 0; r < reps && status == ID_OK; ++r)
            status = launch_batched(problems, (int)count, dtype, queue, infos, c, s);
        if (status == ID_OK && cudaEventRecord(e1, s) != cudaSuccess) status = ID_ECUDA;
        float ms = 0.0f;
        if (status == ID_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            status = ID_ECUDA;
        if (status != ID_OK) break;
        ms /= (float)reps;
        if (ms_out) ms_out[c] = ms;
        if (c == 0 || ms < best_ms) {
            best_ms = ms;
            arg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status == ID_OK) *best = arg;
    return status;
}
