// Column-pivoted Householder QR of short FP32 working matrices (at most 640
// rows, panels of at most 32 pivots), for sm_103a: the CPQR of the sketch
// Y = Omega A of a randomized ID (Sec. 2.1 applied to Y as in Sec. 2.2).
//
// One persistent cooperative launch per panel, one CTA of 512 threads per SM,
// one grid barrier per pivot step. Step j (jj = j - j0 inside the panel):
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
// During a step the trailing columns do not change except at positions j and
// p, so each warp copies its next D column pairs (rows j..m with their F rows,
// squared norms and original indices) from L2 into shared memory with
// cp.async as soon as the step starts: the copies overlap phases A and B, and
// the product reads shared memory. Position p, rewritten by the swap, takes
// its data from the owner's shared copy of the old column j instead.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "cpqr.cuh"
#include "cpqr_dev.cuh"

namespace gbid {

namespace {

constexpr int kSThreads = 512;                          // one CTA per SM
constexpr int kSWarps = kSThreads / kWarp;              // 16
constexpr int kSMaxRows = 640;                          // the short-matrix bound (5 x 128)
constexpr int kSUnits = kSMaxRows / (kWarp * 4);        // 16-byte chunks per lane and column
constexpr int kSRows = (kSMaxRows + kSThreads - 1) / kSThreads;   // rows per thread in phase A
constexpr int kSPanel = 32;                             // widest panel
constexpr int kSMaxD = 8;                               // column-pair slots per warp, at most
constexpr int kSScal = 12;                              // slot tail: vn1, vn2 and perm 16-byte chunks

// Shared-memory layout of one panel launch (floats; every region 16-byte aligned).
struct SLayout {
    int r0;    // first staged row: the panel's first step rounded down to a multiple of 4
    int len;   // staged rows per column: m_pad - r0
    int ldp;   // panel copy leading dimension (len + 1: odd, so 32 panel columns hit 32 banks)
    int cs;    // column slot: len rows, the F row (32), the norm and index chunks (12)
    int D;     // column-pair slots per warp
    int perm16;   // perm is staged too (16-byte aligned, n a multiple of 4: no chunk runs past its end)
};

struct SParams {
    KParams K;
    SLayout L;
};

__device__ __forceinline__ void cp16(float* sdst, const float* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Wait until at most n of this thread's newest copy groups are still pending.
__device__ __forceinline__ void cp_wait_n(int n) {
    switch (n) {
        case 0: cp_wait<0>(); break;
        case 1: cp_wait<1>(); break;
        case 2: cp_wait<2>(); break;
        case 3: cp_wait<3>(); break;
        case 4: cp_wait<4>(); break;
        case 5: cp_wait<5>(); break;
        case 6: cp_wait<6>(); break;
        default: cp_wait<7>(); break;
    }
}

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
    float* my_slots = aux_s + kSPanel + (size_t)w * L.D * 2 * L.cs;   // this warp's D pair slots
    __shared__ float red[kSWarps][kWarp];
    __shared__ float scf[4];       // beta, tau, scale
    __shared__ double swd[2];      // the old position j's vn1, vn2 (the column that moves to p)
    __shared__ int swi;            // its original index
    __shared__ float x0_s;
    __shared__ int stop_s;

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

    const int j0 = P.j_begin;   // one panel per launch
    double r00 = j0 > 0 ? ld(&st->r00) : 0.0;   // |R_00| (thread 0)
    for (int j = j0; j < P.j_end; ++j) {
        tl_stamp(P, j, 0);
        const int jj = j - j0;
        const int j_al = j & ~3;
        const int rows = m_pad - j_al;   // staged rows of this step (<= len)
        // this CTA's trailing positions: a contiguous, balanced range, swept in
        // alternating directions; warp w takes the column pairs w, w + 16, ...
        const int ncols = n - j - 1;
        const int per = ncols > 0 ? ncols / G : 0, rem = ncols > 0 ? ncols % G : 0;
        const int c_lo = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
        const int c_cnt = ncols > 0 ? per + ((int)blockIdx.x < rem ? 1 : 0) : 0;
        const bool rev = (j & 1) != 0;
        const int npairs = (c_cnt + 1) / 2;
        const int my_pairs = npairs > w ? (npairs - w + kSWarps - 1) / kSWarps : 0;
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
        // then this warp's first D column pairs into its slots (one copy group per pair):
        // the rows j_al..m_pad of each column, its F row (the first jj entries), and the
        // 16-byte chunks holding its squared norm, recompute threshold and original index
        auto issue = [&](int r) {
            const int q = w + r * kSWarps;
            float* sl = my_slots + (size_t)(r % L.D) * 2 * L.cs;
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int qc = 2 * q + s2;
                if (qc < c_cnt) {
                    const int l = pos_of(qc);
                    const float* src = W + (int64_t)l * ldw + j_al;
                    float* dst = sl + s2 * L.cs;
#pragma unroll
                    for (int u = 0; u < kSUnits; ++u) {
                        const int o = lane * 4 + u * 128;
                        if (o < rows) cp16(dst + o, src + o);
                    }
                    const int e = lane - 16 * s2;   // lanes 16 s2 .. 16 s2 + 10 copy the tail
                    if (e >= 0 && e < 8 && 4 * e < jj) cp16(dst + L.len + 4 * e, F + (int64_t)l * ldf + 4 * e);
                    else if (e == 8) cp16(dst + L.len + 32, reinterpret_cast<const float*>(P.vn1 + (l & ~1)));
                    else if (e == 9) cp16(dst + L.len + 36, reinterpret_cast<const float*>(P.vn2 + (l & ~1)));
                    else if (e == 10 && L.perm16)
                        cp16(dst + L.len + 40, reinterpret_cast<const float*>(P.perm + (l & ~3)));
                }
            }
            cp_commit();
        };
        const int npre = min(L.D, my_pairs);
        for (int r = 0; r < npre; ++r) issue(r);
        int issued = npre;

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

        // ---- B. reflector: alpha = sqrt(x0^2 + S) from the pair sum with one Newton
        // correction, tau = (beta - x0) / beta and scale = 1 / (x0 - beta) as rounded
        // FP32 divisions (|x0 - beta| = |x0| + alpha, never zero)
        if (t == 0) {
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
        // aux(c) = -tau (scale V(j+1:m, c)^T x(j+1:m) + V(j, c)): thread t takes panel
        // column c = t % 32 over row chunk t / 32; the chunks meet in shared memory
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
        __syncthreads();
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
        // The owner swaps columns j and p, their norms and original indices, once
        // every CTA has read the old columns (phase A); nobody else reads either
        // column, or position p's norms, during the rest of the step.
        if (is_owner) {
            if (t == 0) wait_geq(P.auxcnt + j, (unsigned)G, st);
            __syncthreads();
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
        // lane q owns the q-th finished column of the batch, so the FP64 downdate
        // of up to 32 columns is one pass of full-warp instructions.
        ArgMax bestc = empty_argmax();
        const bool exact_norms = jj == 0;   // W(j:m, l) is exact at a panel's first step
        int nbat = 0;
        int b_l = -1, b_orig = 0;
        float b_r = 0.0f, b_f = 0.0f, b_sq = 0.0f;
        double b_nu = 0.0, b_nu2 = 0.0;
        auto flush = [&]() {
            // nu_new^2 = nu^2 - r^2 (one FMA); recompute when it falls to the
            // threshold sqrt(eps) nu_exact^2 kept in vn2
            int flagged = 0;
            if (lane < nbat) {
                ArgMax cnd;
                cnd.orig = b_orig;
                cnd.pos = b_l;
                cnd.val = 0.0;
                const double ra = (double)b_r;
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
                const float f = __shfl_sync(0xffffffffu, b_f, src);
                const int orr = __shfl_sync(0xffffffffu, b_orig, src);
                const float* frow = F + (int64_t)((l == p && p != j) ? j : l) * ldf;
                const float* col = W + (int64_t)l * ldw;
                double sacc = 0.0;
                for (int i = j + 1 + lane; i < m; i += kWarp) {
                    float y = ld(col + i);
                    for (int c = 0; c < jj; ++c) y -= vpan[c * L.ldp + (i - L.r0)] * ld(frow + c);
                    y -= v_s[i - j_al] * scalef * f;
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
        const float* wjs_al = wj_s + (j_al - L.r0);   // the moved column's staged rows
        for (int r = 0; r < my_pairs; ++r) {
            cp_wait_n(issued - r - 1);
            __syncwarp();   // every lane's copies of this pair have landed
            const int q = w + r * kSWarps;
            const int qc0 = 2 * q;
            const bool has1 = qc0 + 1 < c_cnt;
            const int l0 = pos_of(qc0), l1 = has1 ? pos_of(qc0 + 1) : l0;
            const float* sl = my_slots + (size_t)(r % L.D) * 2 * L.cs;
            const bool mv0 = l0 == p && p != j, mv1 = has1 && l1 == p && p != j;
            const float* d0 = mv0 ? wjs_al : sl;
            const float* d1 = mv1 ? wjs_al : sl + L.cs;
            const float f0 = lane < jj ? (mv0 ? fj_s[lane] : sl[L.len + lane]) : 0.0f;
            const float f1 = (has1 && lane < jj) ? (mv1 ? fj_s[lane] : sl[L.cs + L.len + lane]) : 0.0f;
            // g = x(j+1:m)^T W(j+1:m, l) (x is zero at rows <= j) and, at a panel's
            // first step, ||W(j:m, l)||^2
            float a0 = 0.0f, a1 = 0.0f, q0 = 0.0f, q1 = 0.0f;
#pragma unroll
            for (int u = 0; u < kSUnits; ++u) {
                const int o = lane * 4 + u * 128;
                if (o < rows) {
                    const float4 yv = *reinterpret_cast<const float4*>(v_s + o);
                    const float4 x0v = *reinterpret_cast<const float4*>(d0 + o);
                    a0 = dot_vec(x0v, yv, a0);
                    float4 x1v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (has1) {
                        x1v = *reinterpret_cast<const float4*>(d1 + o);
                        a1 = dot_vec(x1v, yv, a1);
                    }
                    if (exact_norms) {
                        const float* x0e = reinterpret_cast<const float*>(&x0v);
                        const float* x1e = reinterpret_cast<const float*>(&x1v);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j_al + o + e >= j) {
                                q0 = fmaf(x0e[e], x0e[e], q0);
                                q1 = fmaf(x1e[e], x1e[e], q1);
                            }
                    }
                }
            }
            float s10 = 0.0f, s20 = 0.0f, s11 = 0.0f, s21 = 0.0f;
            if (lane < jj) {
                const float ax = aux_s[lane], vr = vrow_s[lane];
                s10 = f0 * ax;
                s20 = f0 * vr;
                s11 = f1 * ax;
                s21 = f1 * vr;
                if (mv0 || mv1) F[(int64_t)p * ldf + lane] = fj_s[lane];   // column p carries the old F(j, :)
            }
            // The eight warp sums as one transposed butterfly: after three halving
            // exchanges each lane holds one partial of one of the eight, whose last
            // two levels finish it; the two batch lanes then fetch theirs.
            float v8[8] = {a0, a1, s10, s20, s11, s21, q0, q1};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const bool hi = (lane & 16) != 0;
                const float send = hi ? v8[qq] : v8[qq + 4];
                const float keep = hi ? v8[qq + 4] : v8[qq];
                v8[qq] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                const bool hi = (lane & 8) != 0;
                const float send = hi ? v8[qq] : v8[qq + 2];
                const float keep = hi ? v8[qq + 2] : v8[qq];
                v8[qq] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool hi = (lane & 4) != 0;
                const float send = hi ? v8[0] : v8[1];
                const float keep = hi ? v8[1] : v8[0];
                v8[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            v8[0] += __shfl_xor_sync(0xffffffffu, v8[0], 2);
            v8[0] += __shfl_xor_sync(0xffffffffu, v8[0], 1);
            // sum k now sits on lane 16 (k >> 2 & 1) + 8 (k >> 1 & 1) + 4 (k & 1)
            const int s0 = nbat, s1i = nbat + 1;
            const bool second = has1 && lane == s1i;
            const float ga = __shfl_sync(0xffffffffu, v8[0], second ? 4 : 0);     // a0 | a1
            const float gs1 = __shfl_sync(0xffffffffu, v8[0], second ? 16 : 8);   // s10 | s11
            const float gs2 = __shfl_sync(0xffffffffu, v8[0], second ? 20 : 12);  // s20 | s21
            const float gq = __shfl_sync(0xffffffffu, v8[0], second ? 28 : 24);   // q0 | q1
            if (lane == s0 || second) {
                const int lc = second ? l1 : l0;
                const bool mv = second ? mv1 : mv0;
                const float* dd = second ? d1 : d0;
                const float* tail = (second ? sl + L.cs : sl) + L.len + 32;
                const float wjl = dd[j - j_al];                 // W(j, l)
                b_l = lc;
                b_nu = mv ? swd[0] : reinterpret_cast<const double*>(tail)[lc & 1];
                b_nu2 = mv ? swd[1] : reinterpret_cast<const double*>(tail + 4)[lc & 1];
                b_orig = mv ? swi : (L.perm16 ? reinterpret_cast<const int*>(tail + 8)[lc & 3] : ld(P.perm + lc));
                const float f = tauf * (scalef * ga + wjl) + gs1;   // tau v^T W(j:m, l) + F(l, :) aux
                b_f = f;
                b_r = wjl - gs2 - f;                                // R(j, l)
                b_sq = gq;
                F[(int64_t)lc * ldf + jj] = f;
                W[(int64_t)lc * ldw + j] = b_r;
            }
            nbat += has1 ? 2 : 1;
            __syncwarp();   // every lane is done with this slot: refill it
            if (issued < my_pairs) {
                issue(issued);
                ++issued;
            }
            if (nbat >= kWarp - 1) flush();
        }
        if (nbat > 0) flush();
        tl_stamp(P, j, 4);
        bestc = block_argmax(bestc);
        if (t == 0) P.part[blockIdx.x] = bestc;
        grid_sync(P.bar, epoch, st);
        tl_stamp(P, j, 5);
    }
    cp_wait<0>();   // (only after an early stop can copies still be in flight)
}

// ------------------------------------------------------------------- host --
namespace {

int g_short_budget = 0;   // dynamic shared memory available to k_cpqr_short (bytes)
int g_short_nsm = 0;

SLayout short_layout(int m, int j0) {
    SLayout L;
    L.perm16 = 0;
    const int m_pad = (m + 3) & ~3;
    L.r0 = j0 & ~3;
    L.len = m_pad - L.r0;
    L.ldp = L.len + 1;
    L.cs = L.len + 32 + kSScal;
    const size_t fixed = sizeof(float) * ((size_t)kSPanel * L.ldp + (L.len + 8) + L.len + 4 * kSPanel);
    const size_t pair = sizeof(float) * 2 * (size_t)L.cs * kSWarps;
    L.D = (size_t)g_short_budget > fixed ? (int)std::min<size_t>(kSMaxD, ((size_t)g_short_budget - fixed) / pair) : 0;
    return L;
}

size_t short_bytes(const SLayout& L) {
    return sizeof(float) * ((size_t)kSPanel * L.ldp + (L.len + 8) + L.len + 4 * kSPanel +
                            (size_t)kSWarps * L.D * 2 * L.cs);
}

}  // namespace

cudaError_t cpqr_short_configure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_short_nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_cpqr_short)) != cudaSuccess) return e;
    g_short_budget = optin - (int)fa.sharedSizeBytes;
    return cudaFuncSetAttribute(k_cpqr_short, cudaFuncAttributeMaxDynamicSharedMemorySize, g_short_budget);
}

bool cpqr_short_rows(int m) { return m >= 1 && m <= kSMaxRows; }

int cpqr_short_grid() {
    // every panel's layout fits one CTA per SM: the widest (m = 640, the first panel) is checked
    const SLayout L = short_layout(kSMaxRows, 0);
    if (L.D < 1 || g_short_nsm < 1 || g_short_nsm > kSThreads) return 0;
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
    SP.L.perm16 = (reinterpret_cast<uintptr_t>(K.perm) % 16 == 0 && K.n % 4 == 0) ? 1 : 0;
    if (SP.L.D < 1 || grid < 1 || grid > kSThreads || K.j_end - K.j_begin > kSPanel) return cudaErrorInvalidConfiguration;
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
