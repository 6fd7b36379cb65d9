// Device helpers shared by the CPQR kernels (k_cpqr and the short-matrix
// kernel): vector types, block reductions, FP32-pair arithmetic, the bounded
// grid barrier, L2-coherent loads, the kernel parameters and the step timeline.
// Internal to the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbid {

template <typename T> struct Vec;

template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };

__device__ __forceinline__ double dot_vec(const double2& a, const double2& b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
}
__device__ __forceinline__ float dot_vec(const float4& a, const float4& b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

// Block-wide argmax; result valid in every thread (blockDim.x <= 1024).
static __device__ ArgMax block_argmax(ArgMax a) {
    __shared__ ArgMax red[32];
    a = warp_argmax(a);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int nw = blockDim.x / kWarp;
    __syncthreads();
    if (lane == 0) red[w] = a;
    __syncthreads();
    a = lane < nw ? red[lane] : empty_argmax();
    return warp_argmax(a);
}

// Deterministic block sum (fixed thread-to-element map and tree order).
static __device__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int nw = blockDim.x / kWarp;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < nw ? red[lane] : 0.0;
    return warp_sum(v);
}

// Double-float (hi + lo, FP32 pair) arithmetic on the FP32 pipe: this GPU
// issues FP64 at a small fraction of its FP32 rate, so the short steps'
// sums of squares carry about 44 bits in FP32 pairs instead (Knuth's TwoSum
// for the additions, an FMA for the exact error of each square).
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    F2 r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}
__device__ __forceinline__ F2 f2_sq(float x) {   // x^2 exactly
    F2 r;
    r.hi = x * x;
    r.lo = fmaf(x, x, -r.hi);
    return r;
}
__device__ __forceinline__ F2 warp_sum_f2(F2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F2 u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = f2_add(v, u);
    }
    return v;
}
// Comparisons of doubles in [0, inf] on the integer pipe (their bit patterns
// order as the values).
__device__ __forceinline__ bool dle(double a, double b) {
    return __double_as_longlong(a) <= __double_as_longlong(b);
}
// A downdated squared norm clamped to [0, inf]: below zero (cancellation) and
// NaN give 0.
__device__ __forceinline__ double clamp_sq(double t) {
    const long long b = __double_as_longlong(t);
    return (b > 0 && b <= 0x7FF0000000000000LL) ? t : 0.0;
}
// 2^-(e/2) for a squared norm 2^e (FP64), clamped to FP32's normal range: the
// power-of-two scale that brings a column of that norm near 1 before its
// entries are squared in FP32.
__device__ __forceinline__ float sq_scale(double nu2) {
    const long long b = __double_as_longlong(nu2);
    if (b <= 0 || b >= 0x7FF0000000000000LL) return 1.0f;
    int k = -((int)((b >> 52) & 0x7ff) - 1023) / 2;
    k = k < -126 ? -126 : (k > 126 ? 126 : k);
    return __int_as_float((k + 127) << 23);
}

// Deterministic block sum of FP32 pairs; the result is valid in every thread.
static __device__ F2 block_sum_f2(F2 v) {
    __shared__ F2 red_f2[32];
    v = warp_sum_f2(v);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int nw = blockDim.x / kWarp;
    __syncthreads();
    if (lane == 0) red_f2[w] = v;
    __syncthreads();
    if (lane < nw) v = red_f2[lane];
    else v.hi = v.lo = 0.0f;
    return warp_sum_f2(v);
}

// Deterministic block sum in the working precision.
template <typename T>
static __device__ T block_sum_t(T v) {
    __shared__ T red_t[32];
    v = warp_sum(v);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int nw = blockDim.x / kWarp;
    __syncthreads();
    if (lane == 0) red_t[w] = v;
    __syncthreads();
    v = lane < nw ? red_t[lane] : T(0);
    return warp_sum(v);
}

// ---------------------------------------------------------- grid barrier --
// Barrier across the co-resident CTAs of the cooperative launch: one
// monotonically growing arrival counter; barrier number b completes when the
// counter reaches (b + 1) * gridDim.x. The wait is bounded: after
// kSpinLimit polls it records kStatTimeout and returns; once that bit is set
// every later wait returns at once and the step loop stops, so the kernel
// always terminates.
constexpr unsigned long long kSpinLimit = 1ull << 22;

__device__ __forceinline__ bool timed_out(const State* st) {
    return (*(const volatile int*)&st->status & kStatTimeout) != 0;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *p >= target (bounded). Returns false on timeout.
static __device__ bool wait_geq(const unsigned* p, unsigned target, State* st) {
    unsigned long long spins = 0;
    while (ld_acquire(p) < target) {
        if ((spins & 31) == 31 && timed_out(st)) return false;   // another CTA gave up
        if (++spins > kSpinLimit) {
            atomicOr(&st->status, kStatTimeout);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// The block barrier orders the CTA's writes before thread 0's release, and
// thread 0's acquire before the other threads' reads; release and acquire at
// gpu scope carry the order between CTAs, so no separate fence is needed.
static __device__ void grid_sync(unsigned* bar, unsigned& epoch, State* st) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        red_release_add(bar, 1u);
        wait_geq(bar, epoch * gridDim.x, st);
    }
    __syncthreads();
}

// L2-coherent loads: data written by other CTAs of the same launch must not be
// served from this SM's L1.
template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }
__device__ __forceinline__ ArgMax ld_argmax(const ArgMax* p) {
    const int4 v = __ldcg(reinterpret_cast<const int4*>(p));
    ArgMax a;
    a.val = __hiloint2double(v.y, v.x);
    a.orig = v.z;
    a.pos = v.w;
    return a;
}

// Trailing-product loads with an L2 eviction hint. The sweep over a CTA's
// columns reverses every step, so the columns read in the second half of one
// sweep are read first in the next: those are loaded evict_last, the others
// evict_first.
__device__ __forceinline__ uint64_t l2_policy(bool last) {
    uint64_t pol;
    if (last) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ double2 ld_hint(const double2* p, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_hint(const float4* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

// VN consecutive entries of the pivot column x restricted to rows j+1..m-1
// (zero elsewhere), read from global memory when it is not cached.
template <typename T, typename V, int VN>
__device__ __forceinline__ V x_at(const T* xbuf, int i, int j, int m) {
    V out;
    T* o = reinterpret_cast<T*>(&out);
#pragma unroll
    for (int q = 0; q < VN; ++q) {
        const int ii = i + q;
        o[q] = ii <= j || ii >= m ? T(0) : __ldcg(xbuf + ii);
    }
    return out;
}

struct KParams {
    void* W;
    int ldw, m, n, k, nb;
    void* F;
    int ldf;
    void* xbuf;       // ldw: pivot column after the lazy update (rows >= j)
    double* vn1;
    double* vn2;
    int* perm;
    double* tau;
    ArgMax* part;     // gridDim.x argmax partials
    double* ssq;      // gridDim.x partial sums of squares
    void* aux;        // kMaxPanel
    unsigned* bar;    // grid-barrier arrival counter, zero on entry
    unsigned* auxcnt; // k per-step counters of finished aux entries, zero on entry
    State* st;
    double rank_tol;
    int rows_per_cta; // row chunk of the pivot-column phase (multiple of 32)
    int j_begin, j_end;   // the pivot steps of this launch (one panel when the WY update runs outside)
    int wy_outside;       // 1: no phase C; the compact-WY update runs as its own launch between panels
    long long* tl;        // step timeline (diagnostic, usually null): kTlSlots %globaltimer stamps per step
    int tl_steps;         // steps the timeline holds
};

// Step timeline: CTA 0, thread 0 stamps %globaltimer at the phase boundaries
// of every step j < tl_steps into tl[j * kTlSlots + q]:
//   0 step start, 1 pivot known, 2 pivot column and its norm formed,
//   3 reflector and aux ready (trailing product starts), 4 trailing product
//   done, 5 after the step's last grid barrier (6, 7 unused).
constexpr int kTlSlots = 8;
__device__ __forceinline__ void tl_stamp(const KParams& P, int j, int q) {
    if (P.tl != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && j < P.tl_steps) {
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        P.tl[(int64_t)j * kTlSlots + q] = t;
    }
}

// The short-matrix CPQR kernel (cpqr_short.cu): FP32, at most 640 rows,
// panels of at most 32 pivots, one cooperative launch (the compact-WY
// update between panels inside the kernel).
cudaError_t cpqr_short_configure();
bool cpqr_short_rows(int m);
int cpqr_short_grid();   // CTAs of its cooperative launch (0: cannot launch)
// Steps K.j_begin .. K.j_end - 1 (phase 0 when j_begin = 0; K.j_begin a multiple of K.nb).
cudaError_t cpqr_short_launch(const KParams& K, int grid, cudaStream_t s);

}  // namespace gbid
