// Column-pivoted Householder QR, truncated after k pivots (Sec. 2.1; the early
// stop proposed in Sec. 4.1), for sm_103a.
//
// Working matrix W is column-major (column l at W + l*ldw), m <= n, ldw a
// multiple of 8, rows m..ldw-1 kept at zero so 16-byte vector loads may run
// over them.
//
// All k pivot steps run in one persistent cooperative kernel (k_cpqr); its
// phases are described above the kernel. The left-looking form (nb = k) never
// rewrites the trailing matrix: each step corrects its product through the
// panel factor F. With nb < k a compact-WY update W_trail -= V F^T runs every
// nb steps and F restarts.
//
// The norm downdate follows Drmac & Bujanovic (LAPACK Working Note 176): the
// downdated estimate nu_l * sqrt(1 - (r_l / nu_l)^2) is replaced by an exact
// recompute once (nu_new / nu_last_exact)^2 falls below sqrt(eps_64).
// The residual norms are kept SQUARED in FP64 (vn1: the current estimate,
// vn2: the recompute threshold sqrt(eps) times the last exact value): the
// downdate is then nu^2 <- nu^2 - r^2 (one FMA), the argmax over squared norms
// picks the same column as over norms, and no square root, division or
// threshold product is taken on the step's critical path.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cpqr.cuh"
#include "cpqr_dev.cuh"
#include "gemm.cuh"
#include "trace.cuh"

namespace gbid {

constexpr int kThreads = 256;              // threads per CTA of the persistent CPQR kernel
constexpr size_t kCpqrSmemMax = 200 * 1024;  // dynamic shared memory (v cached when it fits)

// ------------------------------------------------------------------ copy-in --
// X (m x n, m <= n) into column-major W. trans == 0: X(i,l) = A[i*lda + l]
// (A is m x n row-major). trans == 1: X(i,l) = A[l*lda + i] (A is the user's
// n x m row-major matrix with more rows than columns; X = A^T). Rows m..ldw-1
// of W are zeroed.
template <typename T>
__global__ void __launch_bounds__(256) k_copy_in(const T* __restrict__ A, int64_t lda, int trans, int m, int n,
                                                 T* __restrict__ W, int ldw) {
    __shared__ T tile[32][33];
    const int i0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    if (!trans) {
        for (int q = ty; q < 32; q += 8) {
            const int i = i0 + q, l = l0 + tx;
            tile[q][tx] = (i < m && l < n) ? A[(int64_t)i * lda + l] : T(0);
        }
        __syncthreads();
        for (int q = ty; q < 32; q += 8) {
            const int l = l0 + q, i = i0 + tx;
            if (l < n && i < ldw) W[(int64_t)l * ldw + i] = tile[tx][q];
        }
    } else {
        for (int q = ty; q < 32; q += 8) {
            const int l = l0 + q, i = i0 + tx;
            if (l < n && i < ldw) W[(int64_t)l * ldw + i] = (i < m) ? A[(int64_t)l * lda + i] : T(0);
        }
    }
}

// CSR A (m x n: rowptr[m + 1], colind, values) into the working matrix,
// X = A (trans = 0: W[l * ldw + i]) or X = A^T (trans = 1: W[i * ldw + l]).
// W is zero on entry. One warp per row; duplicate entries are summed (in an
// unspecified order). A decreasing or out-of-range rowptr, or a column index
// outside [0, n), sets kStatBadInput and the entry is skipped.
template <typename T>
__global__ void __launch_bounds__(256) k_csr_in(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                                const T* __restrict__ vals, int m, int n, int64_t nnz, int trans,
                                                T* W, int ldw, int* status) {
    const int lane = threadIdx.x % kWarp;
    for (int i = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp; i < m; i += gridDim.x * (blockDim.x / kWarp)) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicOr(status, kStatBadInput);
            continue;
        }
        for (int64_t q = b + lane; q < e; q += kWarp) {
            const int l = colind[q];
            if (l < 0 || l >= n) {
                atomicOr(status, kStatBadInput);
                continue;
            }
            atomicAdd(trans ? W + (int64_t)i * ldw + l : W + (int64_t)l * ldw + i, vals[q]);
        }
    }
}

// Zero rows m..ldw-1 of every column (id_cpqr path, user-provided X).
template <typename T>
__global__ void k_zero_pad(T* W, int ldw, int m, int n) {
    const int64_t pad = ldw - m;
    const int64_t total = pad * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = e / pad, i = m + e % pad;
        W[l * ldw + i] = T(0);
    }
}

// Self-test of the bounded wait: thread 0 waits on a counter that nothing
// increments, so the wait gives up after kSpinLimit polls and records
// kStatTimeout, the path every barrier of k_cpqr takes when a CTA never
// arrives. One CTA, no other waiter: the kernel always ends.
__global__ void k_selftest_wait(const unsigned* counter, State* st) {
    if (threadIdx.x == 0) wait_geq(counter, 1u, st);
}

// WY tile: W(i, l) -= sum_{c < nbw} V(i, c) F(l, c), 64 x 64 tile at (i0, l0).
template <typename T>
__device__ void wy_tile(T* W, int ldw, int m, int n, int i0, int l0, int j0, int nbw, const T* F, int ldf,
                        T* Vs, T* Fs) {
    constexpr int TM = 64, TN = 64, TK = 16;
    const int t = threadIdx.x;
    const bool act = t < 256;   // 16 x 16 threads own the 64 x 64 tile
    const int tx = t % 16, ty = (t / 16) % 16;
    T acc[4][4], wv[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    // FP32: the tile of W goes out first, its loads overlapping the staging of
    // V and F (FP64 keeps the registers for the rest of the kernel)
    constexpr bool kPreW = sizeof(T) == 4;
#pragma unroll
    for (int b = 0; b < 4 && kPreW; ++b) {
        const int l = l0 + ty * 4 + b;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx * 4 + a;
            wv[a][b] = (act && l < n && i < m) ? ld(W + (int64_t)l * ldw + i) : T(0);
        }
    }
    for (int c0 = 0; c0 < nbw; c0 += TK) {
        __syncthreads();
        for (int e = t; e < TK * TM; e += kThreads) {
            const int c = e / TM, i = e % TM;
            Vs[c * TM + i] = (c0 + c < nbw && i0 + i < m) ? ld(W + (int64_t)(j0 + c0 + c) * ldw + i0 + i) : T(0);
        }
        for (int e = t; e < TK * TN; e += kThreads) {
            const int l = e / TK, c = e % TK;
            Fs[c * (TN + 1) + l] = (c0 + c < nbw && l0 + l < n) ? ld(F + (int64_t)(l0 + l) * ldf + c0 + c) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < TK; ++c) {
            T va[4], fb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) va[a] = Vs[c * TM + tx * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) fb[b] = Fs[c * (TN + 1) + ty * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += va[a] * fb[b];
        }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int l = l0 + ty * 4 + b;
        if (!act || l >= n) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx * 4 + a;
            if (i < m) W[(int64_t)l * ldw + i] = (kPreW ? wv[a][b] : ld(W + (int64_t)l * ldw + i)) - acc[a][b];
        }
    }
    __syncthreads();
}

constexpr int kFRegs = 8;   // panel entries per lane held in registers (panels up to 256 wide)
// reflector entries per thread prefetched ahead of the pivot argmax (panels up to 8 * kPre wide)
template <typename T> constexpr int pre_entries() { return sizeof(T) == 4 ? 32 : 16; }

// Shared-memory plan of k_cpqr (dynamic part): vrow_s | fco | v_s.
struct SmemPlan {
    bool smem_v;    // v cached in shared memory
    size_t bytes;   // dynamic shared memory
};

// ------------------------------------------------------- persistent CPQR --
// One cooperative launch runs all k pivot steps. Per step j (panel start j0,
// jj = j - j0):
//  A. pivot p = argmax over the CTAs' partials (ties: smallest original
//     index); swap columns j <-> p; x = W(:, p) - V F(p, :)^T on rows >= j
//     (the pivot column brought up to date with the panel's reflectors), each
//     CTA on its row chunk; partial ||x(j+1:m)||^2.            -- grid barrier
//  B. beta = -sign(x_j) ||x||, tau = (beta - x_j) / beta, v = x / (x_j - beta)
//     with v_j = 1, written to W(:, j); aux = -tau V^T v (CTA c owns entry c,
//     published through a counter); then the trailing product over the CTA's
//     contiguous column range, one warp per column, sweep direction reversed
//     on odd steps (the tail of one sweep is still in L2 when the next starts):
//       g = W(j:m, l)^T v,  F(l, jj) = tau g + F(l, 0:jj) aux,
//       R(j, l) = W(j, l) - F(l, 0:jj) V(j, 0:jj)^T - F(l, jj),
//     and the FP64 norm downdate nu_l^2 <- nu_l^2 - R(j,l)^2,
//     replaced by an exact recompute when (nu_new / nu_exact)^2 <= sqrt(eps)
//     of the working precision (Drmac & Bujanovic, LAPACK Working Note 176);
//     at a panel's first step the norms are reset exactly from the product's
//     sum of squares; partial argmax.                          -- grid barrier
//     In FP64 (outside a panel's first step) the product takes a row-slab
//     form instead: every warp covers one row slab of every column of the
//     CTA, so the warps finish together (no tail of whole columns), and the
//     epilogue runs a lane per column (FP64 arithmetic on full warps).
//  C. every nb steps (nb < k): compact-WY update W_trail -= V F^T. -- barrier
// Every wait (grid barrier, aux counter) is bounded and ends the kernel early
// with kStatTimeout instead of hanging.
// (Short FP32 matrices with panels of at most 32 run on k_cpqr_short instead.)
template <typename T, bool kSmemV>
__global__ void __launch_bounds__(kThreads, 2) k_cpqr(KParams P) {
    using V = typename Vec<T>::type;
    constexpr int VN = Vec<T>::n;
    constexpr int NW = kThreads / kWarp;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* vrow_s = reinterpret_cast<T*>(smem_raw);
    T* fco = vrow_s + kMaxPanel + 4;
    T* v_s = fco + kMaxPanel + 4;                      // 16-byte aligned
    __shared__ T wy_s[16 * 64 + 16 * 65];              // WY-update tiles
    __shared__ T red[NW][kWarp];
    __shared__ double sc[4];
    __shared__ float scf[4];       // beta, tau, scale rounded to FP32
    __shared__ double red2[NW];
    __shared__ int qctr;   // column queue of this CTA
    __shared__ double nu_s[2][kWarp], nu2_s[2][kWarp];   // slab-form epilogue operands
    __shared__ int orig_s[2][kWarp];
    __shared__ int abort_s;

    T* W = static_cast<T*>(P.W);
    T* F = static_cast<T*>(P.F);
    T* xbuf = static_cast<T*>(P.xbuf);
    T* aux = static_cast<T*>(P.aux);
    State* st = P.st;
    const int m = P.m, n = P.n, ldw = P.ldw, ldf = P.ldf;
    const int t = threadIdx.x, lane = t % kWarp, w = t / kWarp;
    const int G = gridDim.x;
    // Recompute threshold of the norm downdate: sqrt(eps) of the precision the
    // R entries carry (FP32 R entries drift like u_32 (nu_exact / nu)^2).
    const double tol3z = sqrt(sizeof(T) == 8 ? DBL_EPSILON : (double)FLT_EPSILON);
    unsigned epoch = 0;
    const uint64_t pol_last = l2_policy(true), pol_first = l2_policy(false);

    // ---- column norms, perm, first argmax partials (the first launch only)
    if (P.j_begin == 0) {
        if (blockIdx.x == 0 && t == 0) {
            st->rank = P.k;
            st->rank_tol = P.rank_tol;
        }
        ArgMax best = empty_argmax();
        double fro = 0.0;   // this thread's share of ||X||_F^2 (lane 0 of each warp)
        for (int l = blockIdx.x * NW + w; l < n; l += G * NW) {
            const T* col = W + (int64_t)l * ldw;
            double s = 0.0;
            for (int i = lane; i < m; i += kWarp) {
                const double x = (double)ld(col + i);
                s = fma(x, x, s);
            }
            s = warp_sum(s);
            if (lane == 0) fro += s;
            if (lane == 0) {
                P.vn1[l] = s;   // squared norms
                P.vn2[l] = tol3z * s;
                P.perm[l] = l;
                if (!isfinite(s)) atomicOr(&st->status, kStatNonFinite);
                ArgMax c;
                c.val = isfinite(s) ? s : -1.0;
                c.orig = l;
                c.pos = l;
                if (better(c, best)) best = c;
            }
        }
        best = block_argmax(best);
        if (t == 0) P.part[blockIdx.x] = best;
        fro = block_sum(fro);
        if (t == 0) atomicAdd(&st->fro2, fro);
        grid_sync(P.bar, epoch, st);
    }

    const int RC = P.rows_per_cta;
    const int r0 = blockIdx.x * RC;
    const int r1 = min(r0 + RC, m);
    double r00 = P.j_begin > 0 ? ld(&st->r00) : 0.0;   // |R_00| (thread 0; set at step 0)

    for (int j = P.j_begin; j < P.j_end; ++j) {
        if (timed_out(st)) break;
        tl_stamp(P, j, 0);
        const int j0 = j / P.nb * P.nb;
        const int jj = j - j0;

        const int j_al = j & ~(VN - 1);
        const int m_pad = (m + VN - 1) / VN * VN;
        int p = j;
        {
        // ---- A: pivot, swap, lazy update of the pivot column
        // The panel's reflector entries on this CTA's first row tile do not
        // depend on the pivot: their loads are issued before the argmax
        // reduction so that the two latencies overlap.
        constexpr int kPre = pre_entries<T>();
        T vpre[kPre];
        {
            const int r = r0 + lane;
            const bool ok = r < r1 && r >= j;
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                const int c = w + u * NW;
                vpre[u] = (ok && c < jj) ? ld(W + (int64_t)(j0 + c) * ldw + r) : T(0);
            }
        }
        ArgMax best = empty_argmax();
        for (int e = t; e < G; e += kThreads) {
            const ArgMax c = ld_argmax(P.part + e);
            if (better(c, best)) best = c;
        }
        best = block_argmax(best);
        p = best.pos >= j ? best.pos : j;
        tl_stamp(P, j, 1);
        if (blockIdx.x == 0 && p != j) {
            if (t == 0) {
                const double a = ld(P.vn1 + j), b = ld(P.vn1 + p);
                P.vn1[j] = b;
                P.vn1[p] = a;
            } else if (t == 32) {
                const double a = ld(P.vn2 + j), b = ld(P.vn2 + p);
                P.vn2[j] = b;
                P.vn2[p] = a;
            } else if (t == 64) {
                const int a = ld(P.perm + j), b = ld(P.perm + p);
                P.perm[j] = b;
                P.perm[p] = a;
            }
        }
        // W(r, p), W(r, j) of the first row tile go out together with the F-row loads
        T wa = T(0), wb = T(0);
        if (w == 0 && r0 + lane < r1) {
            wa = ld(W + (int64_t)p * ldw + r0 + lane);
            wb = ld(W + (int64_t)j * ldw + r0 + lane);
        }
        for (int c = t; c < jj; c += kThreads) fco[c] = ld(F + (int64_t)p * ldf + c);
        __syncthreads();
        double ssq = 0.0;
        for (int rt = r0; rt < r1; rt += kWarp) {
            const int r = rt + lane;
            if (rt != r0 && w == 0 && r < r1) {   // later row tiles (matrices taller than 32 rows per CTA)
                wa = ld(W + (int64_t)p * ldw + r);
                wb = ld(W + (int64_t)j * ldw + r);
            }
            T acc = T(0);
            if (r < r1 && r >= j) {
                T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
                int cs = w;
                if (rt == r0) {
#pragma unroll
                    for (int u = 0; u < kPre; ++u) {
                        const int c = w + u * NW;
                        const T fv = c < jj ? fco[c] : T(0);
                        if (u % 4 == 0) a0 += vpre[u] * fv;
                        else if (u % 4 == 1) a1 += vpre[u] * fv;
                        else if (u % 4 == 2) a2 += vpre[u] * fv;
                        else a3 += vpre[u] * fv;
                    }
                    cs = w + kPre * NW;
                }
                for (; cs < jj; cs += 8 * NW) {
                    T vv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int c = cs + u * NW;
                        vv[u] = c < jj ? ld(W + (int64_t)(j0 + c) * ldw + r) : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int c = cs + u * NW;
                        const T fv = c < jj ? fco[c] : T(0);
                        if (u % 4 == 0) a0 += vv[u] * fv;
                        else if (u % 4 == 1) a1 += vv[u] * fv;
                        else if (u % 4 == 2) a2 += vv[u] * fv;
                        else a3 += vv[u] * fv;
                    }
                }
                acc = (a0 + a1) + (a2 + a3);
            }
            red[w][lane] = acc;
            __syncthreads();
            if (w == 0 && r < r1) {
                T sr = T(0);
#pragma unroll
                for (int g = 0; g < NW; ++g) sr += red[g][lane];
                const T x = r >= j ? wa - sr : wa;
                W[(int64_t)p * ldw + r] = wb;
                if (r < j) W[(int64_t)j * ldw + r] = x;   // R entries travel with their column
                else xbuf[r] = x;
                if (r > j) ssq = fma((double)x, (double)x, ssq);
                if (r == j) st->x0 = (double)x;
            }
            __syncthreads();
        }
        if (w == 0) {
            ssq = warp_sum(ssq);
            if (lane == 0) P.ssq[blockIdx.x] = ssq;
        }
        grid_sync(P.bar, epoch, st);
        tl_stamp(P, j, 2);

        // ---- B: reflector scalars (same arithmetic in every CTA), this CTA's
        // aux entry and the trailing product's operands, from one round of loads.
        //   aux(c) = -tau V(j:m, c)^T v = -tau (scale V(j+1:m, c)^T x + V(j, c))
        // (the dot needs only x, so it is formed before beta is known).
        const int c_aux = blockIdx.x;
        const bool has_aux = c_aux < jj;
        const T* vca = W + (int64_t)(j0 + (has_aux ? c_aux : 0)) * ldw;
        {
            double sq = t < G ? ld(P.ssq + t) : 0.0;
            const double sq_b = t + kThreads < G ? ld(P.ssq + t + kThreads) : 0.0;
            for (int e = t + 2 * kThreads; e < G; e += kThreads) sq += ld(P.ssq + e);
            sq += sq_b;
            if (t == kThreads - 1) sc[3] = ld(&st->x0);
            for (int c = t; c < jj; c += kThreads) vrow_s[c] = ld(W + (int64_t)(j0 + c) * ldw + j);
            T adot = T(0);
            const int i_lo = kSmemV ? j_al : j + 1, i_hi = kSmemV ? m_pad : m;
            constexpr int kBU = sizeof(T) == 4 ? 16 : 8;   // loads in flight per thread and operand
            for (int i = i_lo + t; (kSmemV || has_aux) && i < i_hi; i += kBU * kThreads) {
                T xs[kBU], vs4[kBU];
#pragma unroll
                for (int u = 0; u < kBU; ++u) {
                    const int ii = i + u * kThreads;
                    const bool in = ii > j && ii < m;
                    xs[u] = in ? ld(xbuf + ii) : T(0);
                    vs4[u] = (in && has_aux) ? ld(vca + ii) : T(0);
                }
#pragma unroll
                for (int u = 0; u < kBU; ++u) {
                    const int ii = i + u * kThreads;
                    if (kSmemV && ii < i_hi) v_s[ii - j_al] = xs[u];
                    if (has_aux) adot += vs4[u] * xs[u];
                }
            }
            sq = warp_sum(sq);
            adot = warp_sum(adot);
            if (lane == 0) {
                red2[w] = sq;
                red[w][0] = adot;
            }
            __syncthreads();
            if (t == 0) {
                double S = 0.0;
                T A = T(0);
#pragma unroll
                for (int g = 0; g < NW; ++g) {
                    S += red2[g];
                    A += red[g][0];
                }
                const double x0 = sc[3];
                const double alpha = sqrt(fma(x0, x0, S));
                double beta = 0.0, tau = 0.0, scale = 0.0;
                if (alpha != 0.0) {
                    beta = x0 >= 0.0 ? -alpha : alpha;
                    tau = (beta - x0) / beta;
                    scale = 1.0 / (x0 - beta);
                }
                sc[0] = beta;
                sc[1] = tau;
                sc[2] = scale;
                scf[0] = (float)beta;
                scf[1] = (float)tau;
                scf[2] = (float)scale;
                if (j == 0) r00 = fabs(beta);     // |R_00|, identical in every CTA
                if (blockIdx.x == 0) {
                    st->beta = beta;
                    st->tau = tau;
                    P.tau[j] = tau;
                    if (j == 0) st->r00 = r00;
                    if (r00 == 0.0 || fabs(beta) <= P.rank_tol * r00) atomicMin(&st->rank, j);
                    if (!isfinite(beta)) atomicOr(&st->status, kStatNonFinite);
                }
                if (has_aux) {
                    aux[c_aux] = -(T)tau * ((T)scale * A + ld(vca + j));
                    __threadfence();
                    red_release_add(P.auxcnt + j, 1u);
                }
                qctr = 0;
            }
            __syncthreads();
        }
        {
            const T scaleT = sizeof(T) == 4 ? (T)scf[2] : (T)sc[2];
            // v on this CTA's rows into W(:, j) (reflector storage, v_j = 1 implicit)
            for (int r = max(r0, j) + t; r < r1; r += kThreads)
                W[(int64_t)j * ldw + r] = r == j ? (T)sc[0] : ld(xbuf + r) * scaleT;
        }

        // aux entries past the first G panel columns (panels wider than the grid)
        for (int c = blockIdx.x + G; c < jj; c += G) {
            const T* vc = W + (int64_t)(j0 + c) * ldw;
            T acc = T(0);
            for (int i = j + 1 + t; i < m; i += kThreads) acc += ld(vc + i) * ld(xbuf + i);
            const T tot = block_sum_t(acc);
            if (t == 0) {
                aux[c] = -(T)sc[1] * ((T)sc[2] * tot + ld(vc + j));
                __threadfence();
                red_release_add(P.auxcnt + j, 1u);
            }
        }
        }   // phases A and B (grid path)
        // v = x * scale (v_j = 1) in the working precision. The stored reflector
        // is formed elementwise; the products with v below use
        // v^T y = scale * x(j+1:m)^T y(j+1:m) + y_j, so no per-element scaling
        // (and no FP64 conversion in FP32) is needed on the hot loops.
        // (FP32 reads the scalars' FP32 copies: no per-thread FP64 conversion)
        const T scaleT = sizeof(T) == 4 ? (T)scf[2] : (T)sc[2];

        // ---- B3: trailing product over this CTA's column range
        tl_stamp(P, j, 3);
        if (j + 1 < n) {
            const T tauT = sizeof(T) == 4 ? (T)scf[1] : (T)sc[1];
            const int ncols = n - j - 1;
            // Each CTA owns a contiguous, balanced range of trailing columns (so
            // every SM gets the same work) and its warps share it through a
            // shared-memory counter. The sweep direction alternates every step:
            // the columns a CTA reads last in step j it reads first in step j+1,
            // while they are still in L2.
            const bool rev = (j & 1) != 0;
            const int per = ncols / G, rem = ncols % G;
            const int c_lo = blockIdx.x * per + min((int)blockIdx.x, rem);
            const int c_cnt = per + ((int)blockIdx.x < rem ? 1 : 0);
            int* ctr = &qctr;
            ArgMax bestc = empty_argmax();
            bool aux_ready = false;
            constexpr int kFR = kFRegs;
            T auxr[kFR];                     // aux[lane + 32 q], loaded once the counter says it is complete
            // Epilogues are batched: lane q owns the q-th finished column of the
            // current batch, so the FP64 downdate of 32 columns is one pass of
            // full-warp FP64 instructions instead of 32 single-lane ones.
            int nbat = 0;                    // columns in the batch (warp-uniform)
            int b_l = -1, b_orig = 0;
            T b_r = T(0), b_f = T(0), b_sq = T(0);
            double b_nu = 0.0, b_nu2 = 1.0;
            // At the first step of a panel W(j:m, l) is up to date, so the
            // trailing product also yields S = ||W(j:m, l)||^2 and the residual
            // norm is reset exactly: nu^2 = S - R(j, l)^2.
            const bool exact_norms = jj == 0;
            auto flush = [&]() {
                int flagged = 0;
                // The downdate on squared norms, without division or square root
                // (long instruction sequences on this GPU's FP64 pipe):
                //   nu_new^2 = nu^2 - r^2 (one FMA), and the recompute test
                //   (nu_new / nu_exact)^2 <= sqrt(eps) multiplied out.
                if (lane < nbat && exact_norms) {
                    ArgMax cnd;
                    cnd.orig = b_orig;
                    cnd.pos = b_l;
                    cnd.val = 0.0;
                    const double S = (double)b_sq;
                    if (S > 0.0) {
                        const double ra = fabs((double)b_r);
                        double t2 = fma(-ra, ra, S);   // ||W(j:m, l)||^2 - R(j, l)^2
                        t2 = t2 > 0.0 ? t2 : 0.0;
                        if (t2 <= tol3z * S) {
                            flagged = 1;
                        } else {
                            cnd.val = t2;
                            P.vn1[b_l] = t2;
                            P.vn2[b_l] = tol3z * t2;
                        }
                    }
                    if (!flagged && better(cnd, bestc)) bestc = cnd;
                } else if (lane < nbat) {
                    ArgMax cnd;
                    cnd.orig = b_orig;
                    cnd.pos = b_l;
                    cnd.val = 0.0;
                    if (__double_as_longlong(b_nu) != 0) {
                        // b_nu: squared norm; b_nu2: its recompute threshold
                        const double ra = (double)b_r;
                        const double t2 = clamp_sq(fma(-ra, ra, b_nu));
                        if (dle(t2, b_nu2)) {
                            flagged = 1;
                        } else {
                            cnd.val = t2;
                            P.vn1[b_l] = t2;
                        }
                    }
                    if (!flagged && better(cnd, bestc)) bestc = cnd;
                }
                unsigned fm = __ballot_sync(0xffffffffu, flagged);
                while (fm) {
                    // cancellation: exact ||W(j+1:m, l) - V F(l, 0:jj+1)^T|| by the whole warp
                    const int src = __ffs(fm) - 1;
                    fm &= fm - 1;
                    const int l = __shfl_sync(0xffffffffu, b_l, src);
                    const T f = __shfl_sync(0xffffffffu, b_f, src);
                    const T* frow = F + (int64_t)((l == p && p != j) ? j : l) * ldf;
                    const T* col = W + (int64_t)l * ldw;
                    double sacc = 0.0;
                    for (int i = j + 1 + lane; i < m; i += kWarp) {
                        T y = ld(col + i);
                        for (int c = 0; c < jj; ++c) y -= ld(W + (int64_t)(j0 + c) * ldw + i) * ld(frow + c);
                        // the current reflector (other CTAs may still be writing it to W(:, j))
                        const T vi = ld(xbuf + i) * scaleT;
                        y -= vi * f;
                        sacc = fma((double)y, (double)y, sacc);
                    }
                    sacc = warp_sum(sacc);
                    if (lane == src) {
                        P.vn1[l] = sacc;
                        P.vn2[l] = tol3z * sacc;
                        ArgMax cnd;
                        cnd.val = sacc;
                        cnd.orig = b_orig;
                        cnd.pos = l;
                        if (better(cnd, bestc)) bestc = cnd;
                        atomicAdd(&st->n_recompute, 1);
                    }
                }
                nbat = 0;
            };
            constexpr int S = kWarp * VN;   // rows per vector load of a warp
            if (sizeof(T) == 8 && !exact_norms) {
                // FP64: balanced row-slab form. Warp w takes the same row slab of every
                // column of a group of GC columns (GC accumulators per lane), so the
                // warps of a CTA finish a group together. Loads run PD columns ahead
                // of the products. The lane partials are reduced across the warp in
                // transposed form (lane q ends with the sum of column q: about one
                // add per column), and the slabs' sums meet in shared memory. The
                // epilogue then runs one lane per column: the panel products
                // F(l, :) aux and F(l, :) V(j, :)^T by all threads (TPC per column),
                // the scalar part (F(l, jj), R(j, l), the norm downdate) by one warp.
                constexpr int GC = 16;                          // columns per group
                constexpr int TPC = kThreads / GC;              // threads per column in the panel products
                constexpr int UR = 4;                           // row units (S rows) of a slab per pass
                constexpr int PD = 1;                           // columns whose loads run ahead
                T* part_s = wy_s;                               // [2][NW][32] slab sums (phase C's tiles are idle)
                T* auxs = part_s + 2 * NW * kWarp;              // [kMaxPanel]
                T* s1_s = auxs + kMaxPanel;                     // [2][32] F(l, :) aux
                T* s2_s = s1_s + 2 * kWarp;                     // [2][32] F(l, :) V(j, :)^T
                T* wj_s = s2_s + 2 * kWarp;                     // [2][32] W(j, l)
                const int nU = (m_pad - j_al + S - 1) / S;
                const int uw0 = w * nU / NW, uw1 = (w + 1) * nU / NW;
                auto col_of = [&](int q) { return j + 1 + c_lo + (rev ? c_cnt - 1 - q : q); };
                for (int g0 = 0, gi = 0; g0 < c_cnt; g0 += GC, ++gi) {
                    const int ncg = min(GC, c_cnt - g0);
                    const int pb = gi & 1;
                    T* part = part_s + pb * NW * kWarp;
                    // the scalar epilogue's operands, loaded now and stored after the products
                    const int pk = t / GC, pq = t % GC;
                    double pre = 0.0;
                    if (pk < 4 && pq < ncg) {
                        const int l = col_of(g0 + pq);
                        if (pk == 0) pre = (double)ld(W + (int64_t)l * ldw + j);
                        else if (pk == 1) pre = ld(P.vn1 + l);
                        else if (pk == 2) pre = ld(P.vn2 + l);
                        else pre = (double)ld(P.perm + l);
                    }
                    T acc[GC];
#pragma unroll
                    for (int cc = 0; cc < GC; ++cc) acc[cc] = T(0);
                    for (int u0 = uw0; u0 < uw1; u0 += UR) {
                        V xv[PD + 1][UR];
                        auto load_col = [&](V(&x)[UR], int cc) {
                            const T* col = W + (int64_t)col_of(g0 + cc) * ldw;
                            const uint64_t pol = 2 * (g0 + cc) >= c_cnt ? pol_last : pol_first;
#pragma unroll
                            for (int ur = 0; ur < UR; ++ur) {
                                const int i = j_al + (u0 + ur) * S + lane * VN;
                                if (u0 + ur < uw1 && i < m_pad) x[ur] = ld_hint(reinterpret_cast<const V*>(col + i), pol);
                            }
                        };
#pragma unroll
                        for (int q = 0; q < PD; ++q)
                            if (q < ncg) load_col(xv[q], q);
#pragma unroll
                        for (int cc = 0; cc < GC; ++cc) {
                            if (cc < ncg) {
                                if (cc + PD < ncg) load_col(xv[(cc + PD) % (PD + 1)], cc + PD);
#pragma unroll
                                for (int ur = 0; ur < UR; ++ur) {
                                    const int i = j_al + (u0 + ur) * S + lane * VN;
                                    if (u0 + ur < uw1 && i < m_pad) {
                                        const V yv = kSmemV ? *reinterpret_cast<const V*>(v_s + (i - j_al))
                                                            : x_at<T, V, VN>(xbuf, i, j, m);
                                        acc[cc] = dot_vec(xv[cc % (PD + 1)][ur], yv, acc[cc]);
                                    }
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int o = GC / 2; o >= 1; o >>= 1) {
                        const bool hi = (lane & o) != 0;
#pragma unroll
                        for (int q = 0; q < o; ++q) {
                            const T send = hi ? acc[q] : acc[q + o];
                            const T keep = hi ? acc[q + o] : acc[q];
                            acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                        }
                    }
                    if (GC < kWarp) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], GC);
                    if (lane < GC) part[w * kWarp + lane] = acc[0];
                    if (pk < 4 && pq < ncg) {
                        if (pk == 0) wj_s[pb * kWarp + pq] = (T)pre;
                        else if (pk == 1) nu_s[pb][pq] = pre;
                        else if (pk == 2) nu2_s[pb][pq] = pre;
                        else orig_s[pb][pq] = (int)pre;
                    }
                    if (gi == 0 && w == 0) {   // the panel's aux entries, complete once the counter reaches jj
                        int ok = 1;
                        if (lane == 0) ok = wait_geq(P.auxcnt + j, (unsigned)jj, st) ? 1 : 0;
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        if (ok)
                            for (int c = lane; c < jj; c += kWarp) auxs[c] = ld(aux + c);
                        if (lane == 0) abort_s = !ok;
                    }
                    __syncthreads();
                    if (abort_s) break;
                    {   // panel products, TPC threads per column, 16 loads in flight per thread
                        const int cc = t / TPC, seg = t % TPC;
                        T s1 = T(0), s2 = T(0);
                        if (cc < ncg) {
                            const int l = col_of(g0 + cc);
                            const bool moved = l == p && p != j;   // column p carries the old column j's F row
                            const T* frow = F + (int64_t)(moved ? j : l) * ldf;
                            for (int c0 = seg; c0 < jj; c0 += 16 * TPC) {
                                T fv[16];
#pragma unroll
                                for (int b = 0; b < 16; ++b) {
                                    const int c = c0 + b * TPC;
                                    fv[b] = c < jj ? ld(frow + c) : T(0);
                                }
#pragma unroll
                                for (int b = 0; b < 16; ++b) {
                                    const int c = c0 + b * TPC;
                                    if (c < jj) {
                                        if (moved) F[(int64_t)p * ldf + c] = fv[b];
                                        s1 += fv[b] * auxs[c];
                                        s2 += fv[b] * vrow_s[c];
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int o = TPC / 2; o >= 1; o >>= 1) {
                            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                        }
                        if (cc < ncg && seg == 0) {
                            s1_s[pb * kWarp + cc] = s1;
                            s2_s[pb * kWarp + cc] = s2;
                        }
                    }
                    __syncthreads();
                    if (w == (gi + (int)blockIdx.x) % NW) {   // scalar epilogue, lane q <-> column q of the group
                        int flagged = 0, l = -1;
                        T f = T(0);
                        if (lane < ncg) {
                            l = col_of(g0 + lane);
                            T gx = T(0);
#pragma unroll
                            for (int w2 = 0; w2 < NW; ++w2) gx += part[w2 * kWarp + lane];
                            const T wjl = wj_s[pb * kWarp + lane];
                            const T g = scaleT * gx + wjl;          // v^T W(j:m, l)
                            f = tauT * g + s1_s[pb * kWarp + lane];
                            const T r = wjl - s2_s[pb * kWarp + lane] - f;   // R(j, l)
                            F[(int64_t)l * ldf + jj] = f;
                            W[(int64_t)l * ldw + j] = r;
                            ArgMax cnd;
                            cnd.orig = orig_s[pb][lane];
                            cnd.pos = l;
                            cnd.val = 0.0;
                            const double nu = nu_s[pb][lane];   // squared norms
                            if (nu != 0.0) {
                                // nu_new^2 = nu^2 - r^2; recompute when it falls to
                                // sqrt(eps) of the last exact squared norm
                                const double ra = (double)r;
                                const double t2 = clamp_sq(fma(-ra, ra, nu));
                                if (dle(t2, nu2_s[pb][lane])) {   // (the recompute threshold)
                                    flagged = 1;
                                } else {
                                    cnd.val = t2;
                                    P.vn1[l] = t2;
                                }
                            }
                            if (!flagged && better(cnd, bestc)) bestc = cnd;
                        }
                        unsigned fm = __ballot_sync(0xffffffffu, flagged);
                        while (fm) {
                            // cancellation: exact ||W(j+1:m, l) - V F(l, 0:jj+1)^T|| by the whole warp
                            const int src = __ffs(fm) - 1;
                            fm &= fm - 1;
                            const int lr = __shfl_sync(0xffffffffu, l, src);
                            const T fr = __shfl_sync(0xffffffffu, f, src);
                            const int origr = orig_s[pb][src];
                            const T* frow = F + (int64_t)((lr == p && p != j) ? j : lr) * ldf;
                            const T* col = W + (int64_t)lr * ldw;
                            double sacc = 0.0;
                            for (int i = j + 1 + lane; i < m; i += kWarp) {
                                T y = ld(col + i);
                                for (int c = 0; c < jj; ++c) y -= ld(W + (int64_t)(j0 + c) * ldw + i) * ld(frow + c);
                                const T vi = ld(xbuf + i) * scaleT;   // the current reflector
                                y -= vi * fr;
                                sacc = fma((double)y, (double)y, sacc);
                            }
                            sacc = warp_sum(sacc);
                            if (lane == src) {
                                P.vn1[lr] = sacc;
                                P.vn2[lr] = tol3z * sacc;
                                ArgMax cnd;
                                cnd.val = sacc;
                                cnd.orig = origr;
                                cnd.pos = lr;
                                if (better(cnd, bestc)) bestc = cnd;
                                atomicAdd(&st->n_recompute, 1);
                            }
                        }
                    }
                }
            } else {
            int idx = 0;
            if (lane == 0) idx = atomicAdd(ctr, 1);
            idx = __shfl_sync(0xffffffffu, idx, 0);
            while (idx < c_cnt) {
                const int l = j + 1 + c_lo + (rev ? c_cnt - 1 - idx : idx);
                int nidx = 0;
                if (lane == 0) nidx = atomicAdd(ctr, 1);   // next column, in flight meanwhile
                const bool moved = l == p && p != j;        // column p carries the old column j's F row
                const T* frow = F + (int64_t)(moved ? j : l) * ldf;
                const int slot = nbat;
                T wjl = T(0);
                if (lane == slot) {                         // this column's epilogue operands
                    b_l = l;
                    wjl = ld(W + (int64_t)l * ldw + j);
                    b_nu = ld(P.vn1 + l);
                    b_nu2 = ld(P.vn2 + l);
                    b_orig = ld(P.perm + l);
                }
                T fr[kFR];
#pragma unroll
                for (int q = 0; q < kFR; ++q) {
                    const int c = lane + q * kWarp;
                    fr[q] = c < jj ? ld(frow + c) : T(0);
                }
                // g = W(j_al:m_pad, l)^T v, eight 16-byte loads per lane in flight
                constexpr int kGU = 8;
                const T* col = W + (int64_t)l * ldw;
                const uint64_t pol = 2 * idx >= c_cnt ? pol_last : pol_first;
                T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0), sq = T(0);
                for (int i0 = j_al + lane * VN; i0 < m_pad; i0 += kGU * S) {
                    V xv[kGU];
#pragma unroll
                    for (int u = 0; u < kGU; ++u) {
                        const int i = i0 + u * S;
                        if (i < m_pad) xv[u] = ld_hint(reinterpret_cast<const V*>(col + i), pol);
                    }
                    if (exact_norms) {
#pragma unroll
                        for (int u = 0; u < kGU; ++u) {
                            const int i = i0 + u * S;
                            if (i < m_pad) {
                                const T* xe = reinterpret_cast<const T*>(&xv[u]);
#pragma unroll
                                for (int q = 0; q < VN; ++q)
                                    if (i + q >= j) sq = fma(xe[q], xe[q], sq);   // rows j..m (padding is zero)
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kGU; ++u) {
                        const int i = i0 + u * S;
                        if (i < m_pad) {
                            const V yv = kSmemV ? *reinterpret_cast<const V*>(v_s + (i - j_al))
                                                : x_at<T, V, VN>(xbuf, i, j, m);
                            if (u % 4 == 0) a0 = dot_vec(xv[u], yv, a0);
                            else if (u % 4 == 1) a1 = dot_vec(xv[u], yv, a1);
                            else if (u % 4 == 2) a2 = dot_vec(xv[u], yv, a2);
                            else a3 = dot_vec(xv[u], yv, a3);
                        }
                    }
                }
                if (!aux_ready) {
                    int ok = 1;
                    if (lane == 0) ok = wait_geq(P.auxcnt + j, (unsigned)jj, st) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) break;
#pragma unroll
                    for (int q = 0; q < kFR; ++q) {
                        const int c = lane + q * kWarp;
                        auxr[q] = c < jj ? ld(aux + c) : T(0);
                    }
                    aux_ready = true;
                }
                T s1 = T(0), s2 = T(0);
#pragma unroll
                for (int q = 0; q < kFR; ++q) {
                    const int c = lane + q * kWarp;
                    if (c < jj) {
                        if (moved) F[(int64_t)p * ldf + c] = fr[q];
                        s1 += fr[q] * auxr[q];
                        s2 += fr[q] * vrow_s[c];
                    }
                }
                for (int c = lane + kFR * kWarp; c < jj; c += kWarp) {   // panels wider than kFR * 32
                    const T fv = ld(frow + c);
                    if (moved) F[(int64_t)p * ldf + c] = fv;
                    s1 += fv * ld(aux + c);
                    s2 += fv * vrow_s[c];
                }
                const T gx = warp_sum((a0 + a1) + (a2 + a3));   // x(j+1:m)^T W(j+1:m, l)
                if (exact_norms) sq = warp_sum(sq);
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                if (lane == slot) {
                    const T g = scaleT * gx + wjl;          // v^T W(j:m, l)
                    const T f = tauT * g + s1;
                    b_f = f;
                    b_r = wjl - s2 - f;                     // R(j, l)
                    b_sq = sq;
                    F[(int64_t)l * ldf + jj] = f;
                    W[(int64_t)l * ldw + j] = b_r;
                }
                ++nbat;
                idx = __shfl_sync(0xffffffffu, nidx, 0);
                if (nbat == kWarp || idx >= c_cnt) flush();
            }
            if (nbat > 0) flush();   // only reached after a timed-out wait
            }
            tl_stamp(P, j, 4);
            bestc = block_argmax(bestc);
            if (t == 0) P.part[blockIdx.x] = bestc;
        }
        grid_sync(P.bar, epoch, st);
        tl_stamp(P, j, 5);

        // ---- C: compact-WY trailing update at the end of a panel
        if (!P.wy_outside && j + 1 < P.k && jj == P.nb - 1 && m > j + 1) {
            const int je = j + 1;
            const int tm = (m - je + 63) / 64, tn = (n - je + 63) / 64;
            for (int tile = blockIdx.x; tile < tm * tn; tile += G)
                wy_tile<T>(W, ldw, m, n, je + (tile % tm) * 64, je + (tile / tm) * 64, j0, P.nb, F, ldf, wy_s,
                           wy_s + 16 * 64);
            grid_sync(P.bar, epoch, st);
        }
    }
}

// ------------------------------------------------------------------- host --
// Short FP32 matrices (at most 640 rows) with panels of at most 32 run on the
// short-matrix kernel (cpqr_short.cu), one launch for all panels. FP32 only: it
// keeps the panel's reflectors and the staged columns in shared memory.
template <typename T>
static bool use_short(int m, int nb) {
    return sizeof(T) == 4 && cpqr_short_rows(m) && nb <= kWarp;
}

// Shared-memory bytes of k_cpqr for m working rows; v is cached in shared
// memory when it fits in kCpqrSmemMax.
template <typename T>
static SmemPlan cpqr_smem(int m, int nb) {
    const int vn = Vec<T>::n;
    const size_t m_pad = (size_t)(m + vn - 1) / vn * vn;
    const size_t fixed = sizeof(T) * 2 * ((size_t)kMaxPanel + 4);
    const size_t vbytes = sizeof(T) * (m_pad + 8);
    SmemPlan pl;
    pl.smem_v = fixed + vbytes <= kCpqrSmemMax;
    pl.bytes = fixed + (pl.smem_v ? vbytes : 0);
    (void)nb;
    return pl;
}

static int g_nsm = 0;
static long long* g_tl = nullptr;   // step timeline of the next CPQR runs (diagnostic)
static int g_tl_steps = 0;


template <typename T>
cudaError_t cpqr_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_cpqr<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCpqrSmemMax);
    if (e != cudaSuccess) return e;
    if (sizeof(T) == 4 && (e = cpqr_short_configure()) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cpqr<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCpqrSmemMax);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
}

template <typename T>
cudaError_t copy_in(const void* A, int64_t lda, int trans, const CpqrPlan& P, cudaStream_t s) {
    dim3 grid(ceil_div(P.ldw, 32), ceil_div(P.n, 32));
    k_copy_in<T><<<grid, 256, 0, s>>>(static_cast<const T*>(A), lda, trans, P.m, P.n, static_cast<T*>(P.W), P.ldw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t csr_in(const int64_t* rowptr, const int32_t* colind, const void* vals, int64_t m, int64_t n, int64_t nnz,
                   int trans, const CpqrPlan& P, int* status, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(P.W, 0, sizeof(T) * (size_t)P.ldw * P.n, s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(ceil_div(m, kThreads / kWarp), 4096);
    k_csr_in<T><<<blocks, kThreads, 0, s>>>(rowptr, colind, static_cast<const T*>(vals), (int)m, (int)n, nnz, trans,
                                            static_cast<T*>(P.W), P.ldw, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t zero_pad(const CpqrPlan& P, cudaStream_t s) {
    if (P.ldw == P.m) return cudaSuccess;
    k_zero_pad<T><<<304, 256, 0, s>>>(static_cast<T*>(P.W), P.ldw, P.m, P.n);
    return cudaGetLastError();
}

template <typename T>
int cpqr_grid(int m, int nb) {
    const SmemPlan pl = cpqr_smem<T>(m, nb);
    if (use_short<T>(m, nb)) return cpqr_short_grid();
    int occ = 0;
    if (pl.smem_v)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cpqr<T, true>, kThreads, pl.bytes);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cpqr<T, false>, kThreads, pl.bytes);
    if (occ < 1) return 0;
    return std::min(kMaxParts, g_nsm * occ);
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

size_t wy_bytes(int m, int n, int nb) {
    const size_t kp = (size_t)kpad16(nb);
    return 2 * al256(4 * (size_t)m * kp) + 2 * al256(4 * (size_t)n * kp);
}

// The compact-WY update after the panel of steps j0..je-1 (FP32 data):
// W(je:m, je:n) -= V F^T with V = W(je:m, j0:je) (the panel's reflectors below
// its diagonal block) and F = F(je:n, 0:je-j0), as a 3xTF32 product on the
// tensor cores whose epilogue updates W in place. The product is formed as
// (W - V F^T)^T = W^T - F V^T: the accumulator's lanes run along the columns of
// the column-major W, so each thread reads and writes 128-byte segments of a
// column with 16-byte accesses.
static int wy_update_f32(const CpqrPlan& P, int j0, int je, cudaStream_t s) {
    const int M = P.m - je, N = P.n - je, nbw = je - j0, kp = (int)kpad16(nbw);
    if (M < 1 || N < 1) return ID_OK;
    char* w = static_cast<char*>(P.wy_ws);
    float* ah = reinterpret_cast<float*>(w);
    float* alo = reinterpret_cast<float*>(w + al256(4 * (size_t)P.m * kp));
    float* bh = reinterpret_cast<float*>(w + 2 * al256(4 * (size_t)P.m * kp));
    float* blo = reinterpret_cast<float*>(w + 2 * al256(4 * (size_t)P.m * kp) + al256(4 * (size_t)P.n * kp));
    float* W = static_cast<float*>(P.W);
    const float* F = static_cast<const float*>(P.F);
    // V (M x nbw): V(r, c) = W[(j0 + c) * ldw + je + r], the transposed read of the panel's columns
    if (split_tf32<float>(W + (int64_t)j0 * P.ldw + je, P.ldw, 1, M, nbw, kp, ah, alo, kp, s) != cudaSuccess)
        return ID_ECUDA;
    // F rows je..n-1 (N x nbw), row-major with leading dimension ldf
    if (split_tf32<float>(F + (int64_t)je * P.ldf, P.ldf, 0, N, nbw, kp, bh, blo, kp, s) != cudaSuccess)
        return ID_ECUDA;
    TfEpilogue ep;
    ep.alpha = -1.0f;
    ep.beta = 1.0f;
    ep.cin = W + (int64_t)je * P.ldw + je;   // (column c, row r) of the block at [c * ldw + r]
    ep.ldc = P.ldw;
    ep.d = W + (int64_t)je * P.ldw + je;
    ep.ldd = P.ldw;
    return gemm_tf32x3(TfOperand{bh, blo, kp, N}, TfOperand{ah, alo, kp, M}, N, M, kp, 1, ep, &P.st->status, s);
}

template <typename T>
cudaError_t cpqr_run(const CpqrPlan& P, cudaStream_t s) {
    const double eps = sizeof(T) == 8 ? DBL_EPSILON : (double)FLT_EPSILON;
    const SmemPlan pl = cpqr_smem<T>(P.m, P.nb);
    // The full resident grid even for small problems: a 16-CTA grid measured
    // slower on a 200 x 400 ID (608 against 504 us), the per-step latencies
    // (L2 round trips, barriers) dominating either way.
    const int G = cpqr_grid<T>(P.m, P.nb);
    if (G < 1) return cudaErrorInvalidConfiguration;

    cudaError_t e = cudaMemsetAsync(P.st, 0, sizeof(State), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(P.sync, 0, sync_bytes(P.k), s);
    if (e != cudaSuccess) return e;

    KParams K;
    K.W = P.W;
    K.ldw = P.ldw;
    K.m = P.m;
    K.n = P.n;
    K.k = P.k;
    K.nb = P.nb;
    K.F = P.F;
    K.ldf = P.ldf;
    K.xbuf = P.xbuf;
    K.vn1 = P.vn1;
    K.vn2 = P.vn2;
    K.perm = P.perm;
    K.tau = P.tau;
    K.part = P.part3;
    K.ssq = P.ssq;
    K.aux = P.aux;
    char* sync = reinterpret_cast<char*>(P.sync);
    K.bar = reinterpret_cast<unsigned*>(sync);
    K.auxcnt = reinterpret_cast<unsigned*>(sync + 64);
    K.st = P.st;
    // numerical rank: |R_jj| <= sqrt(max(m, n)) eps |R_00| (rounding-noise level of a residual)
    K.rank_tol = sqrt((double)(P.m_user > P.n_user ? P.m_user : P.n_user)) * eps;
    K.rows_per_cta = (int)round_up(ceil_div(P.m, G), kWarp);
    K.tl = g_tl;
    K.tl_steps = g_tl_steps;

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = pl.bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    // FP32 panels narrower than k: the WY update runs on the tensor cores
    // between per-panel launches of k_cpqr (which then skips its phase C).
    K.wy_outside = (sizeof(T) == 4 && P.nb < P.k && P.wy_ws != nullptr) ? 1 : 0;
    const int step = K.wy_outside ? P.nb : P.k;
    // the short-matrix kernel runs every panel in one launch (its WY update inside)
    const bool shortk = use_short<T>(P.m, P.nb);
    const int tr = trace_begin(TraceKind::kCpqr, s);
    if (shortk) {
        K.j_begin = 0;
        K.j_end = P.k;
        e = cpqr_short_launch(K, G, s);
        if (e != cudaSuccess) return e;
        trace_end(tr, s);
        return cudaGetLastError();
    }
    for (int j0 = 0; j0 < P.k; j0 += step) {
        K.j_begin = j0;
        K.j_end = j0 + step < P.k ? j0 + step : P.k;
        if (j0 > 0 && (e = cudaMemsetAsync(K.bar, 0, 64, s)) != cudaSuccess) return e;   // fresh barrier epochs
        if (pl.smem_v) e = cudaLaunchKernelEx(&cfg, k_cpqr<T, true>, K);
        else e = cudaLaunchKernelEx(&cfg, k_cpqr<T, false>, K);
        if (e != cudaSuccess) return e;
        if (K.wy_outside && K.j_end < P.k && P.m > K.j_end && wy_update_f32(P, j0, K.j_end, s) != ID_OK)
            return cudaErrorLaunchFailure;
    }
    trace_end(tr, s);
    return cudaGetLastError();
}

template cudaError_t cpqr_configure<double>();
template cudaError_t cpqr_configure<float>();
template int cpqr_grid<double>(int, int);
template int cpqr_grid<float>(int, int);
template cudaError_t copy_in<double>(const void*, int64_t, int, const CpqrPlan&, cudaStream_t);
template cudaError_t copy_in<float>(const void*, int64_t, int, const CpqrPlan&, cudaStream_t);
template cudaError_t csr_in<double>(const int64_t*, const int32_t*, const void*, int64_t, int64_t, int64_t, int,
                                    const CpqrPlan&, int*, cudaStream_t);
template cudaError_t csr_in<float>(const int64_t*, const int32_t*, const void*, int64_t, int64_t, int64_t, int,
                                   const CpqrPlan&, int*, cudaStream_t);
template cudaError_t zero_pad<double>(const CpqrPlan&, cudaStream_t);
template cudaError_t zero_pad<float>(const CpqrPlan&, cudaStream_t);
template cudaError_t cpqr_run<double>(const CpqrPlan&, cudaStream_t);
template cudaError_t cpqr_run<float>(const CpqrPlan&, cudaStream_t);

}  // namespace gbid

extern "C" int id_cpqr_timeline(long long* buf, int steps) {
    if (steps < 0 || (steps > 0 && !buf)) return ID_EINVAL;
    gbid::g_tl = steps > 0 ? buf : nullptr;
    gbid::g_tl_steps = steps;
    return ID_OK;
}

extern "C" int id_selftest_bounded_wait(void* work, size_t work_bytes, int* status, void* stream) {
    static_assert(256 + sizeof(gbid::State) <= ID_SELFTEST_WORK_BYTES, "self-test scratch");
    if (!work || !status || work_bytes < ID_SELFTEST_WORK_BYTES || (reinterpret_cast<uintptr_t>(work) & 255))
        return ID_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(work, 0, ID_SELFTEST_WORK_BYTES, s) != cudaSuccess) return ID_ECUDA;
    const unsigned* counter = static_cast<const unsigned*>(work);
    gbid::State* st = reinterpret_cast<gbid::State*>(static_cast<char*>(work) + 256);
    gbid::k_selftest_wait<<<1, 32, 0, s>>>(counter, st);
    if (cudaGetLastError() != cudaSuccess) return ID_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, &st->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ID_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ID_ECUDA;
    *status = (bits & gbid::kStatTimeout) ? ID_ETIMEOUT : ID_OK;
    return ID_OK;
}
