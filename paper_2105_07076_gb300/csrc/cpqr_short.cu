// Column-pivoted Householder QR of short FP32 working matrices (at most 640
// rows, panels of at most 32 pivots), for sm_103a: the CPQR of the sketch
// Y = Omega A of a randomized ID (Sec. 2.1 applied to Y as in Sec. 2.2).
//
// One persistent cooperative launch for all k steps, one CTA of 512 threads per
// SM, one grid barrier per pivot step. Step j (jj = j - j0 inside its panel):
//   A. every CTA reads the previous step's argmax partials (largest squared
//      residual norm, ties to the smallest original index) and forms the pivot
//      column x = W(j:m, p) - V(j:m, 0:jj) F(p, 0:jj)^T from its shared-memory
//      copy of the panel's reflectors (left-looking: the trailing matrix is
//      not updated inside a panel), with ||x(j+1:m)||^2 in FP32 pairs;
//   B. the reflector (beta, tau, scale in FP32), aux = -tau V^T v and the panel
//      copy's column jj; the CTA whose range holds position p swaps columns j
//      and p once every CTA has read them;
//   C. the trailing product over the CTA's contiguous, balanced range of
//      positions: g = v^T W(j:m, l), F(l, jj) = tau g + F(l, 0:jj) aux,
//      R(j, l) = W(j, l) - F(l, 0:jj) V(j, 0:jj)^T - F(l, jj), the FP64
//      downdate of the squared norm (exact recompute on cancellation) and the
//      CTA's argmax partial.                                 -- grid barrier
//   D. at a panel's last step, the compact-WY update of the trailing columns,
//      W(je:m, l) -= V(je:m, :) F(l, :)^T, each CTA on its share of the
//      columns from its panel copy and the F rows.           -- grid barrier
// The trailing product is latency-bound (one L2 round trip per column group
// and warp): a group of TPC threads takes one column (TPC = 16, 8, 4 or 2,
// picked each step so that a thread holds at most 12 vector loads of its
// column), so a warp keeps 32 / TPC columns in flight per round, and each
// column costs log2(TPC) shuffle levels instead of a full warp reduction.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "cpqr.cuh"
#include "cpqr_dev.cuh"
#include "gemm.cuh"
#include "tc.cuh"

namespace gbid {

namespace {

constexpr int kSThreads = 512;                          // one CTA per SM
constexpr int kSWarps = kSThreads / kWarp;              // 16
constexpr int kSMaxRows = 640;                          // the short-matrix bound (5 x 128)
constexpr int kSUnits = kSMaxRows / (kWarp * 4);        // 16-byte chunks per lane and column
constexpr int kSRows = (kSMaxRows + kSThreads - 1) / kSThreads;   // rows per thread in phase A
constexpr int kSPanel = 32;                             // widest panel
// In-kernel compact-WY update on the tensor cores: per CTA, tiles of 128 columns
// (the MMA's M, operand A = their F rows) by 256 rows (its N, operand B = the
// panel's V rows), K = the panel width (two 16-wide K blocks), 3xTF32 into a
// 256-column tensor-memory accumulator.
constexpr int kWyM = 128, kWyN = 256;
constexpr int kWyTileA = kWyM * 64, kWyTileB = kWyN * 64;   // bytes of one 64-byte-swizzled K16 tile
constexpr int kWyBytes = 4 * kWyTileA + 4 * kWyTileB;       // A and B: hi and lo, two K16 blocks each
constexpr unsigned long long kWySpin = 1ull << 24;

// Shared-memory layout of one panel launch (floats; every region 16-byte aligned).
struct SLayout {
    int r0;    // first row kept: the panel's first step rounded down to a multiple of 4
    int len;   // rows kept per column: m_pad - r0
    int ldp;   // panel copy leading dimension (len + 1: odd, so 32 panel columns hit 32 banks)
};

struct SParams {
    KParams K;
    SLayout L;
};

}  // namespace

__global__ void __launch_bounds__(kSThreads, 1) k_cpqr_short(const __grid_constant__ SParams SP) {
    const KParams& P = SP.K;
    const SLayout L = SP.L;
    const int m = P.m, n = P.n, ldw = P.ldw, ldf = P.ldf;
    const int t = threadIdx.x, lane = t % kWarp, w = t / kWarp;
    const int G = gridDim.x;
    const int m_pad = (m + 3) & ~3;
    // recompute threshold of the norm downdate: sqrt(eps) of FP32, the precision of the R entries
    const double tol3z = sqrt((double)FLT_EPSILON);
    unsigned epoch = 0;
    State* st = P.st;
    float* W = static_cast<float*>(P.W);
    float* F = static_cast<float*>(P.F);

    extern __shared__ __align__(16) float sm[];
    float* vpan = sm;                              // [32][ldp]: the panel's reflectors, rows r0.. (v_j = 1 kept as 0)
    float* v_s = vpan + kSPanel * L.ldp;           // len + 8: x (index i - j_al), zero at rows <= j
    float* wj_s = v_s + L.len + 8;                 // len: the old column j, rows r0.. (the owner's)
    float* fco = wj_s + L.len;                     // 32: F(p, 0:jj)
    float* fj_s = fco + kSPanel;                   // 32: F(j, 0:jj), the row that moves to position p
    float* vrow_s = fj_s + kSPanel;                // 32: V(j, 0:jj)
    float* aux_s = vrow_s + kSPanel;               // 32: aux
    // the WY update's operand tiles (1024-byte aligned for the 64-byte swizzle)
    unsigned char* wy_ops = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(aux_s + kSPanel) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ float red[kSWarps][kWarp];
    __shared__ float scf[4];       // beta, tau, scale
    __shared__ double swd[2];      // the old position j's vn1, vn2 (the column that moves to p)
    __shared__ int swi;            // its original index
    __shared__ float x0_s;
    __shared__ int stop_s;
    __shared__ __align__(8) uint64_t wy_bar;   // completion of the WY update's MMAs
    __shared__ uint32_t wy_tmem;               // its tensor-memory accumulator
    __shared__ int wy_abort;                   // a bounded wait on wy_bar gave up
    const uint64_t pol_last = l2_policy(true), pol_first = l2_policy(false);
    const bool wy_on = P.nb < P.j_end - P.j_begin;   // more than one panel: WY updates between them
    if (wy_on) {
        if (t == 0) {
            wy_abort = 0;
            tc::mb_init(&wy_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (w == 0) tc::tmem_alloc(&wy_tmem, kWyN);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    unsigned wy_phase = 0;   // parity of wy_bar's next completion

    // ---- squared column norms, perm, first argmax partials (the first panel only).
    // Each warp takes whole columns; the squares are summed in FP32 pairs after a
    // power-of-two prescale by the column's largest entry (no FP32 overflow or
    // underflow), and the sum goes to FP64 once.
    if (P.j_begin == 0) {
        if (blockIdx.x == 0 && t == 0) {
            st->rank = P.k;
            st->rank_tol = P.rank_tol;
        }
        ArgMax best = empty_argmax();
        double fro = 0.0;   // lane 0's share of ||X||_F^2
        for (int l = blockIdx.x * kSWarps + w; l < n; l += G * kSWarps) {
            const float* col = W + (int64_t)l * ldw;
            float xr[kSUnits * 4];
            float amax = 0.0f;
#pragma unroll
            for (int u = 0; u < kSUnits * 4; ++u) {
                const int i = lane + u * kWarp;
                xr[u] = i < m ? ld(col + i) : 0.0f;
                amax = fmaxf(amax, fabsf(xr[u]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            const float sig = sq_scale((double)amax * (double)amax);
            F2 s2{0.0f, 0.0f};
#pragma unroll
            for (int u = 0; u < kSUnits * 4; ++u) s2 = f2_add(s2, f2_sq(xr[u] * sig));
            s2 = warp_sum_f2(s2);
            if (lane == 0) {
                const double inv = (double)(1.0f / sig);   // exact: a power of two
                const double s = ((double)s2.hi + (double)s2.lo) * inv * inv;
                const bool fin = isfinite(amax) && isfinite(s);
                fro += s;
                P.vn1[l] = s;
                P.vn2[l] = tol3z * s;
                P.perm[l] = l;
                if (!fin) atomicOr(&st->status, kStatNonFinite);
                ArgMax c;
                c.val = fin ? s : -1.0;
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

    double r00 = P.j_begin > 0 ? ld(&st->r00) : 0.0;   // |R_00| (kept by thread 31, which forms the reflectors)
    for (int j = P.j_begin; j < P.j_end; ++j) {
        tl_stamp(P, j, 0);
        const int j0 = j / P.nb * P.nb;   // the panel's first step
        const int jj = j - j0;
        const int j_al = j & ~3;
        const int rows = m_pad - j_al;   // staged rows of this step (<= len)
        // this CTA's trailing positions: a contiguous, balanced range, swept in
        // alternating directions (the columns read last in one step are read first
        // in the next, while they are still in L2)
        const int ncols = n - j - 1;
        const int per = ncols > 0 ? ncols / G : 0, rem = ncols > 0 ? ncols % G : 0;
        const int c_lo = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
        const int c_cnt = ncols > 0 ? per + ((int)blockIdx.x < rem ? 1 : 0) : 0;
        const bool rev = (j & 1) != 0;
        auto pos_of = [&](int qc) { return j + 1 + c_lo + (rev ? c_cnt - 1 - qc : qc); };

        // ---- A. the argmax partials and column j's rows go out first
        ArgMax best = empty_argmax();
        if (t < G) best = ld_argmax(P.part + t);
        float wj_r[kSRows];
#pragma unroll
        for (int u = 0; u < kSRows; ++u) {
            const int i = t + u * kSThreads;
            wj_r[u] = i < m ? ld(W + (int64_t)j * ldw + i) : 0.0f;
        }
        if (t == 0) stop_s = timed_out(st) ? 1 : 0;   // one read, shared: the block breaks together
        best = block_argmax(best);   // (its barriers publish stop_s)
        if (stop_s) break;
        const int p = best.pos >= j ? best.pos : j;
        const float sig = sq_scale(best.val);   // prescale for the FP32 squares of the pivot column
        tl_stamp(P, j, 1);
        // The CTA whose trailing range holds position p (CTA 0 when p = j) swaps
        // columns j and p; it loads their norms and original indices now.
        int owner = 0;
        if (p != j) {
            const int qq = p - j - 1;
            owner = qq < rem * (per + 1) ? qq / (per + 1) : rem + (qq - rem * (per + 1)) / per;
        }
        const bool is_owner = (int)blockIdx.x == owner;
        double sw_a = 0.0, sw_b = 0.0;   // vn1 (thread 0), vn2 (thread 32), perm (thread 64) of j and p
        if (is_owner && p != j) {
            if (t == 0) {
                sw_a = ld(P.vn1 + j);
                sw_b = ld(P.vn1 + p);
            } else if (t == 32) {
                sw_a = ld(P.vn2 + j);
                sw_b = ld(P.vn2 + p);
            } else if (t == 64) {
                sw_a = (double)ld(P.perm + j);
                sw_b = (double)ld(P.perm + p);
            }
        }
        float wp_r[kSRows];
#pragma unroll
        for (int u = 0; u < kSRows; ++u) {
            const int i = t + u * kSThreads;
            wp_r[u] = i < m ? ld(W + (int64_t)p * ldw + i) : 0.0f;
        }
        for (int c = t; c < jj; c += kSThreads) fco[c] = ld(F + (int64_t)p * ldf + c);
        if (is_owner && p != j) {
            for (int c = t; c < jj; c += kSThreads) fj_s[c] = ld(F + (int64_t)j * ldf + c);
#pragma unroll
            for (int u = 0; u < kSRows; ++u) {
                const int i = t + u * kSThreads;
                if (i >= L.r0 && i < m_pad) wj_s[i - L.r0] = wj_r[u];
            }
        }
        __syncthreads();
        // x(i) = W(i, p) - sum_c V(i, c) F(p, c) on rows j..m-1; v_s = x below row j;
        // ||x(j+1:m)||^2 in FP32 pairs of the prescaled entries
        F2 sq{0.0f, 0.0f};
#pragma unroll
        for (int u = 0; u < kSRows; ++u) {
            const int i = t + u * kSThreads;
            if (i >= j_al && i < m_pad) {
                float x = 0.0f;
                if (i >= j && i < m) {
                    const float* vp = vpan + (i - L.r0);
                    float acc = 0.0f;
                    for (int c = 0; c < jj; ++c) acc += vp[c * L.ldp] * fco[c];
                    x = wp_r[u] - acc;
                }
                if (i == j) x0_s = x;
                v_s[i - j_al] = i > j ? x : 0.0f;
                if (i > j) sq = f2_add(sq, f2_sq(x * sig));
            }
        }
        const F2 S = block_sum_f2(sq);   // synchronises: x0_s and v_s are visible after it
        tl_stamp(P, j, 2);
        // This CTA has read columns j and p and F(p, :): the owner's swap below
        // waits for every CTA's signal, so these reads are never overtaken.
        if (t == 0) red_release_add(P.auxcnt + j, 1u);
        // Lane 31 of every warp has no aux work (panel columns number at most 31 before
        // the current one): the owner's wait for every CTA's reads runs on thread 511
        // and the reflector's scalars on thread 31, alongside the aux dots.
        if (is_owner && t == kSThreads - 1) wait_geq(P.auxcnt + j, (unsigned)G, st);

        // ---- B. aux(c) = -tau (scale V(j+1:m, c)^T x(j+1:m) + V(j, c)): thread t takes
        // panel column c = t % 32 over row chunk t / 32; the chunks meet in shared memory
        {
            const int c = t % kWarp, ch = t / kWarp;
            const int nr = m - (j + 1);
            const int per_r = nr > 0 ? (nr + kSWarps - 1) / kSWarps : 0;
            const int i0 = j + 1 + ch * per_r, i1 = min(m, i0 + per_r);
            float a = 0.0f;
            if (c < jj)
                for (int i = i0; i < i1; ++i) a += vpan[c * L.ldp + (i - L.r0)] * v_s[i - j_al];
            red[ch][c] = a;
        }
        // The reflector: alpha = sqrt(x0^2 + S) from the pair sum with one Newton
        // correction, tau = (beta - x0) / beta and scale = 1 / (x0 - beta) as rounded
        // FP32 divisions (|x0 - beta| = |x0| + alpha, never zero).
        if (t == kWarp - 1) {
            const float x0 = x0_s;
            const F2 a2 = f2_add(f2_sq(x0 * sig), S);   // (scaled by sig^2)
            float alpha = sqrtf(a2.hi);
            if (alpha > 0.0f) alpha += (fmaf(-alpha, alpha, a2.hi) + a2.lo) / (2.0f * alpha);
            alpha = alpha / sig;   // exact: a power of two
            float beta = 0.0f, tau = 0.0f, scale = 0.0f;
            if (alpha != 0.0f) {
                beta = x0 >= 0.0f ? -alpha : alpha;
                const float d = x0 - beta;
                tau = __fdiv_rn(-d, beta);
                scale = __fdiv_rn(1.0f, d);
            }
            scf[0] = beta;
            scf[1] = tau;
            scf[2] = scale;
            if (j == 0) r00 = fabs((double)beta);
            if (blockIdx.x == 0) {
                st->beta = beta;
                st->tau = tau;
                P.tau[j] = tau;
                if (j == 0) st->r00 = r00;
                if (r00 == 0.0 || fabs((double)beta) <= P.rank_tol * r00) atomicMin(&st->rank, j);
                if (!isfinite(beta)) atomicOr(&st->status, kStatNonFinite);
            }
        }
        __syncthreads();
        const float tauf = scf[1], scalef = scf[2];
        if (t < jj) {
            float sum = 0.0f;
#pragma unroll
            for (int g = 0; g < kSWarps; ++g) sum += red[g][t];
            const float vj = vpan[t * L.ldp + (j - L.r0)];
            aux_s[t] = -tauf * (scalef * sum + vj);
            vrow_s[t] = vj;
        }
        __syncthreads();   // the panel copy's column jj is written next
        for (int i = L.r0 + t; i < L.r0 + L.len; i += kSThreads)
            vpan[jj * L.ldp + (i - L.r0)] = (i > j && i < m) ? v_s[i - j_al] * scalef : 0.0f;
        // The owner swaps columns j and p, their norms and original indices (every CTA
        // has read the old columns: thread 511's wait ended before the barrier above);
        // nobody else reads either column, or position p's norms, during the rest of
        // the step.
        if (is_owner) {
            if (p != j) {
                if (t == 0) {
                    P.vn1[j] = sw_b;
                    P.vn1[p] = sw_a;
                    swd[0] = sw_a;
                } else if (t == 32) {
                    P.vn2[j] = sw_b;
                    P.vn2[p] = sw_a;
                    swd[1] = sw_a;
                } else if (t == 64) {
                    P.perm[j] = (int)sw_b;
                    P.perm[p] = (int)sw_a;
                    swi = (int)sw_a;
                }
            }
            const float betaf = scf[0];
#pragma unroll
            for (int u = 0; u < kSRows; ++u) {
                const int i = t + u * kSThreads;
                if (i < m) {
                    if (p != j) W[(int64_t)p * ldw + i] = wj_r[u];   // the old column j moves to p
                    if (i >= j || p != j)
                        W[(int64_t)j * ldw + i] = i < j ? wp_r[u] : (i == j ? betaf : v_s[i - j_al] * scalef);
                }
            }
        }
        __syncthreads();
        tl_stamp(P, j, 3);

        // ---- C. trailing product from the staged slots. Epilogues are batched:
        // lane q keeps the q-th finished column's sums, so F(l, jj), R(j, l) and the
        // FP64 downdate of up to 32 columns take one pass of full-warp instructions.
        ArgMax bestc = empty_argmax();
        const bool exact_norms = jj == 0;   // W(j:m, l) is exact at a panel's first step
        int nbat = 0;
        int b_l = -1, b_orig = 0;
        float b_ga = 0.0f, b_s1 = 0.0f, b_s2 = 0.0f, b_sq = 0.0f, b_wj = 0.0f;
        double b_nu = 0.0, b_nu2 = 0.0;
        auto flush = [&]() {
            // f = tau (scale g + W(j, l)) + F(l, :) aux, R(j, l) = W(j, l) - F(l, :) V(j, :)^T - f;
            // nu_new^2 = nu^2 - r^2 (one FMA), recomputed when it falls to the
            // threshold sqrt(eps) nu_exact^2 kept in vn2
            int flagged = 0;
            float f = 0.0f;
            if (lane < nbat) {
                f = tauf * (scalef * b_ga + b_wj) + b_s1;
                const float r = b_wj - b_s2 - f;
                F[(int64_t)b_l * ldf + jj] = f;
                W[(int64_t)b_l * ldw + j] = r;
                ArgMax cnd;
                cnd.orig = b_orig;
                cnd.pos = b_l;
                cnd.val = 0.0;
                const double ra = (double)r;
                if (exact_norms) {
                    const double S2 = (double)b_sq;   // ||W(j:m, l)||^2 from the product
                    if (S2 > 0.0) {
                        const double t2 = clamp_sq(fma(-ra, ra, S2));
                        if (t2 <= tol3z * S2) {
                            flagged = 1;
                        } else {
                            cnd.val = t2;
                            P.vn1[b_l] = t2;
                            P.vn2[b_l] = tol3z * t2;
                        }
                    }
                } else if (__double_as_longlong(b_nu) != 0) {
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
                // cancellation: the exact ||W(j+1:m, l) - V F(l, 0:jj+1)^T||^2 by the whole warp
                const int src = __ffs(fm) - 1;
                fm &= fm - 1;
                const int l = __shfl_sync(0xffffffffu, b_l, src);
                const float fl = __shfl_sync(0xffffffffu, f, src);
                const int orr = __shfl_sync(0xffffffffu, b_orig, src);
                const float* frow = F + (int64_t)((l == p && p != j) ? j : l) * ldf;
                const float* col = W + (int64_t)l * ldw;
                double sacc = 0.0;
                for (int i = j + 1 + lane; i < m; i += kWarp) {
                    float y = ld(col + i);
                    for (int c = 0; c < jj; ++c) y -= vpan[c * L.ldp + (i - L.r0)] * ld(frow + c);
                    y -= v_s[i - j_al] * scalef * fl;
                    sacc = fma((double)y, (double)y, sacc);
                }
                sacc = warp_sum(sacc);
                if (lane == src) {
                    P.vn1[l] = sacc;
                    P.vn2[l] = tol3z * sacc;
                    ArgMax cnd;
                    cnd.val = sacc;
                    cnd.orig = orr;
                    cnd.pos = l;
                    if (better(cnd, bestc)) bestc = cnd;
                    atomicAdd(&st->n_recompute, 1);
                }
            }
            nbat = 0;
        };
        const float* wjs_al = wj_s + (j_al - L.r0);   // the moved column's rows j_al..
        // One round: a group of TPC lanes per column, NC = 32 / TPC columns per warp;
        // thread `part` of a group holds rows j_al + 4 part + 4 TPC k (k < NL) of its
        // column and entries 4 (part + TPC e) .. + 3 of its F row.
        auto sweep = [&](auto tpc_c) {
            constexpr int TPC = decltype(tpc_c)::value;
            constexpr int NC = kWarp / TPC;
            constexpr int NL = TPC == 16 ? 10 : 12;             // rows <= 4 TPC NL
            constexpr int NF = (kSPanel / 4 + TPC - 1) / TPC;   // F-row chunks per thread
            const int cg = lane / TPC, part = lane % TPC;
            const int ngroups = (c_cnt + NC - 1) / NC;
            for (int gi = w; gi < ngroups; gi += kSWarps) {
                const int qc = gi * NC + cg;
                const bool has = qc < c_cnt;
                const int l = has ? pos_of(qc) : j;
                const bool mv = has && l == p && p != j;
                // the round's columns go to batch lanes nbat .. nbat + NC - 1, which load
                // their squared norms, thresholds and original indices now (for the flush)
                const int ncol = min(NC, c_cnt - gi * NC);
                const bool mine = lane >= nbat && lane < nbat + ncol;
                if (mine) {
                    const int lb = pos_of(gi * NC + lane - nbat);
                    const bool bmv = lb == p && p != j;
                    b_l = lb;
                    b_nu = bmv ? swd[0] : ld(P.vn1 + lb);
                    b_nu2 = bmv ? swd[1] : ld(P.vn2 + lb);
                    b_orig = bmv ? swi : ld(P.perm + lb);
                }
                const uint64_t pol = 2 * qc >= c_cnt ? pol_last : pol_first;
                const float* colp = W + (int64_t)l * ldw + j_al;
                float4 xv[NL];
#pragma unroll
                for (int k = 0; k < NL; ++k) {
                    const int o = 4 * part + 4 * TPC * k;
                    xv[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (has && o < rows)
                        xv[k] = mv ? *reinterpret_cast<const float4*>(wjs_al + o)
                                   : ld_hint(reinterpret_cast<const float4*>(colp + o), pol);
                }
                float4 fv[NF];
#pragma unroll
                for (int e = 0; e < NF; ++e) {
                    const int cb = 4 * (part + TPC * e);
                    fv[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (has && cb < jj)
                        fv[e] = mv ? *reinterpret_cast<const float4*>(fj_s + cb)
                                   : __ldcg(reinterpret_cast<const float4*>(F + (int64_t)l * ldf + cb));
                }
                // g = x(j+1:m)^T W(j+1:m, l) (x is zero at rows <= j); at a panel's first
                // step also ||W(j:m, l)||^2
                float a = 0.0f, qn = 0.0f;
#pragma unroll
                for (int k = 0; k < NL; ++k) {
                    const int o = 4 * part + 4 * TPC * k;
                    if (o < rows) {
                        const float4 yv = *reinterpret_cast<const float4*>(v_s + o);
                        a = dot_vec(xv[k], yv, a);
                        if (exact_norms) {
                            const float* xe = reinterpret_cast<const float*>(&xv[k]);
#pragma unroll
                            for (int z = 0; z < 4; ++z)
                                if (j_al + o + z >= j) qn = fmaf(xe[z], xe[z], qn);
                        }
                    }
                }
                // F(l, 0:jj) aux and F(l, 0:jj) V(j, 0:jj)^T (entries past jj masked)
                float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
                for (int e = 0; e < NF; ++e) {
                    const int cb = 4 * (part + TPC * e);
                    if (cb < jj) {
                        const float* fe = reinterpret_cast<const float*>(&fv[e]);
#pragma unroll
                        for (int z = 0; z < 4; ++z)
                            if (cb + z < jj) {
                                s1 = fmaf(fe[z], aux_s[cb + z], s1);
                                s2 = fmaf(fe[z], vrow_s[cb + z], s2);
                                if (mv) F[(int64_t)p * ldf + cb + z] = fe[z];   // column p carries the old F(j, :)
                            }
                    }
                }
                // W(j, l) sits in the group's first chunk (rows j_al .. j_al + 3)
                const int zj = j - j_al;
                const float wj_own = zj == 0 ? xv[0].x : (zj == 1 ? xv[0].y : (zj == 2 ? xv[0].z : xv[0].w));
#pragma unroll
                for (int o2 = 1; o2 < TPC; o2 <<= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o2);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, o2);
                    s2 += __shfl_xor_sync(0xffffffffu, s2, o2);
                    if (exact_norms) qn += __shfl_xor_sync(0xffffffffu, qn, o2);
                }
                const int src = mine ? (lane - nbat) * TPC : 0;
                const float ga = __shfl_sync(0xffffffffu, a, src);
                const float gs1 = __shfl_sync(0xffffffffu, s1, src);
                const float gs2 = __shfl_sync(0xffffffffu, s2, src);
                const float gq = __shfl_sync(0xffffffffu, qn, src);
                const float gwj = __shfl_sync(0xffffffffu, wj_own, src);
                if (mine) {
                    b_ga = ga;
                    b_s1 = gs1;
                    b_s2 = gs2;
                    b_sq = gq;
                    b_wj = gwj;
                }
                nbat += ncol;
                if (nbat > kWarp - NC) flush();
            }
        };
        // threads per column: the fewest that keep a thread at 12 vector loads or fewer
        if (rows > 384) sweep(std::integral_constant<int, 16>{});
        else if (rows > 192) sweep(std::integral_constant<int, 8>{});
        else if (rows > 96) sweep(std::integral_constant<int, 4>{});
        else sweep(std::integral_constant<int, 2>{});
        if (nbat > 0) flush();
        tl_stamp(P, j, 4);
        bestc = block_argmax(bestc);
        if (t == 0) P.part[blockIdx.x] = bestc;
        grid_sync(P.bar, epoch, st);
        tl_stamp(P, j, 5);

        // ---- compact-WY update at a panel's end on the tensor cores:
        // W(je:m, l) -= V(je:m, 0:nb) F(l, 0:nb)^T for this CTA's balanced share of the trailing
        // columns, as D(i, l) = sum_c V(i, c) F(l, c) (3xTF32: the operands split into TF32 hi and
        // lo parts and written in the 64-byte-swizzled K-major layout the MMA reads; A = 128 rows
        // of the panel's reflectors, B = 256 columns' F rows) and an epilogue that subtracts D from
        // W (TMEM lane = row i, so a warp's accesses to one column coalesce).
        if (wy_on && jj == P.nb - 1 && j + 1 < P.j_end && j + 1 < m) {
            const int je = j + 1;
            const int nw = n - je;
            const int perw = nw / G, remw = nw % G;
            const int w_lo = je + (int)blockIdx.x * perw + min((int)blockIdx.x, remw);
            const int w_cnt = perw + ((int)blockIdx.x < remw ? 1 : 0);
            const int nrow = m - je;
            const uint32_t idesc = tc::idesc_tf32(kWyM, kWyN);
            // element (r, c) of a K16 tile at r * 64 + ((c / 4) ^ ((r >> 1) & 3)) * 16 + (c % 4) * 4
            auto put = [&](unsigned char* tile_hi, unsigned char* tile_lo, int r, int c, float x) {
                const int off = r * 64 + (((c >> 2) ^ ((r >> 1) & 3)) << 4) + ((c & 3) << 2);
                const float h = tf32_hi(x);
                *reinterpret_cast<float*>(tile_hi + off) = h;
                *reinterpret_cast<float*>(tile_lo + off) = x - h;
            };
            unsigned char* a_hi = wy_ops;                      // [kt][128 x 64 B]: V rows
            unsigned char* a_lo = wy_ops + 2 * kWyTileA;
            unsigned char* b_hi = wy_ops + 4 * kWyTileA;       // [kt][256 x 64 B]: F rows
            unsigned char* b_lo = b_hi + 2 * kWyTileB;
            for (int nt = 0; nt < w_cnt; nt += kWyN) {
                const int ncnt = min(kWyN, w_cnt - nt);
                // B: the F rows of columns w_lo + nt .. (entries past the panel zero)
                for (int e = t; e < kWyN * kSPanel; e += kSThreads) {
                    const int r = e / kSPanel, c = e % kSPanel;
                    const float x = (r < ncnt && c <= jj) ? ld(F + (int64_t)(w_lo + nt + r) * ldf + c) : 0.0f;
                    put(b_hi + (c >> 4) * kWyTileB, b_lo + (c >> 4) * kWyTileB, r, c & 15, x);
                }
                for (int mt = 0; mt < nrow; mt += kWyM) {
                    const int mcnt = min(kWyM, nrow - mt);
                    // A: rows je + mt .. of the panel's reflectors (from the panel copy)
                    for (int e = t; e < kWyM * kSPanel; e += kSThreads) {
                        const int r = e / kSPanel, c = e % kSPanel;
                        const float x = (r < mcnt && c <= jj) ? vpan[c * L.ldp + (je + mt + r - L.r0)] : 0.0f;
                        put(a_hi + (c >> 4) * kWyTileA, a_lo + (c >> 4) * kWyTileA, r, c & 15, x);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA reads
                    tc::fence_before();
                    __syncthreads();   // (also: the previous tile's accumulator reads are done)
                    tc::fence_after();
                    if (t == 0) {
#pragma unroll
                        for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const unsigned o = kk * 32;   // 8 TF32 = 32 bytes along the swizzled row
                                const unsigned ah = tc::su32(a_hi + kt * kWyTileA) + o,
                                               al = tc::su32(a_lo + kt * kWyTileA) + o;
                                const unsigned bh = tc::su32(b_hi + kt * kWyTileB) + o,
                                               bl = tc::su32(b_lo + kt * kWyTileB) + o;
                                tc::umma_tf32(wy_tmem, tc::sdesc_sw64(al), tc::sdesc_sw64(bh), idesc,
                                              (kt | kk) ? 1u : 0u);
                                tc::umma_tf32(wy_tmem, tc::sdesc_sw64(ah), tc::sdesc_sw64(bl), idesc, 1u);
                                tc::umma_tf32(wy_tmem, tc::sdesc_sw64(ah), tc::sdesc_sw64(bh), idesc, 1u);
                            }
                        tc::umma_commit(&wy_bar);
                    }
                    int ok = 1;
                    if (lane == 0) ok = tc::mb_wait(&wy_bar, wy_phase, &wy_abort, kWySpin) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    wy_phase ^= 1u;
                    tc::fence_after();
                    if (!ok) {
                        if (t == 0) atomicOr(&st->status, kStatTimeout);
                    } else {
                        // epilogue: warp w reads TMEM lane quarter w % 4 (32 rows of W), the four warps
                        // of a quarter take alternate 32-column chunks; lane = row, so each column's
                        // read-modify-write is one coalesced 128-byte access per warp
                        const int q4 = w % 4, part4 = w / 4;
                        const int r = q4 * 32 + lane;   // A row: W row je + mt + r
                        const bool row_ok = r < mcnt;
                        float* wrow = W + (int64_t)(w_lo + nt) * ldw + je + mt + r;
                        for (int c0 = part4 * 32; c0 < kWyN; c0 += 128) {
                            uint32_t v[32];
                            TMEM_LD_X32(wy_tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0, v);
                            tc::tmem_wait_ld();
                            if (c0 < ncnt) {
                                float x[32];
#pragma unroll
                                for (int u = 0; u < 32; ++u)
                                    x[u] = (row_ok && c0 + u < ncnt) ? ld(wrow + (int64_t)(c0 + u) * ldw) : 0.0f;
#pragma unroll
                                for (int u = 0; u < 32; ++u)
                                    if (row_ok && c0 + u < ncnt) wrow[(int64_t)(c0 + u) * ldw] = x[u] - __uint_as_float(v[u]);
                            }
                        }
                    }
                    tc::fence_before();
                    __syncthreads();   // the operand tiles and the accumulator are free again
                    tc::fence_after();
                }
            }
            grid_sync(P.bar, epoch, st);   // the next panel reads the updated columns
        }
    }
    if (wy_on) {
        // (after a wait that gave up, an MMA may still run: wait again, bounded, before the free)
        if (t == 0 && wy_abort) {
            unsigned long long spins = 0;
            while (!tc::mb_test(&wy_bar, wy_phase ^ 1u) && ++spins < kWySpin) __nanosleep(64);
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (w == 0) tc::tmem_dealloc(wy_tmem, kWyN);
    }
}

// ------------------------------------------------------------------- host --
namespace {

int g_short_nsm = 0;

SLayout short_layout(int m, int j0) {
    SLayout L;
    const int m_pad = (m + 3) & ~3;
    L.r0 = j0 & ~3;
    L.len = m_pad - L.r0;
    L.ldp = L.len + 1;
    return L;
}

size_t short_bytes(const SLayout& L) {
    return sizeof(float) * ((size_t)kSPanel * L.ldp + (L.len + 8) + L.len + 4 * kSPanel) + 1024 + kWyBytes;
}

}  // namespace

cudaError_t cpqr_short_configure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_short_nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const SLayout L = short_layout(kSMaxRows, 0);   // the largest layout (the first panel at 640 rows)
    return cudaFuncSetAttribute(k_cpqr_short, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)short_bytes(L));
}

bool cpqr_short_rows(int m) { return m >= 1 && m <= kSMaxRows; }

int cpqr_short_grid() {
    // one CTA per SM for every panel's layout: the largest is checked
    const SLayout L = short_layout(kSMaxRows, 0);
    if (g_short_nsm < 1 || g_short_nsm > kSThreads) return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cpqr_short, kSThreads, short_bytes(L)) != cudaSuccess ||
        occ < 1)
        return 0;
    return g_short_nsm;
}

cudaError_t cpqr_short_launch(const KParams& K, int grid, cudaStream_t s) {
    SParams SP;
    SP.K = K;
    SP.L = short_layout(K.m, K.j_begin);
    if (grid < 1 || grid > kSThreads || K.nb < 1 || K.nb > kSPanel || !cpqr_short_rows(K.m))
        return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kSThreads);
    cfg.dynamicSmemBytes = short_bytes(SP.L);
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cpqr_short, SP);
}

}  // namespace gbid
