// Shared device-side definitions of the ID library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbid.h"

namespace gbid {

constexpr int kWarp = 32;
constexpr int kMaxParts = 2048;     // argmax partial slots per producer kernel

// Device-side status bits collected during a decomposition.
enum : int { kStatNonFinite = 1, kStatTimeout = 2, kStatOverflow = 4, kStatBadInput = 8 };

// One candidate of the pivot search: residual norm, original index, position.
struct __align__(16) ArgMax {
    double val;
    int orig;
    int pos;
};

// Total order used for pivot selection: larger norm wins, equal norms go to
// the smaller ORIGINAL column index. An empty slot has val = -1.
// Every val is -1 or a non-negative double other than -0 (a norm, a squared
// norm, or a sum of squares): on that set the bit patterns read as signed
// 64-bit integers order exactly as the values, so the comparison runs on the
// integer pipe instead of the FP64 pipe.
__device__ __forceinline__ bool better(const ArgMax& a, const ArgMax& b) {
    const long long av = __double_as_longlong(a.val), bv = __double_as_longlong(b.val);
    return av > bv || (av == bv && a.orig < b.orig);
}

__device__ __forceinline__ ArgMax empty_argmax() {
    ArgMax a;
    a.val = -1.0;
    a.orig = 0x7fffffff;
    a.pos = -1;
    return a;
}

__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ArgMax b;
        b.val = __shfl_xor_sync(0xffffffffu, a.val, o);
        b.orig = __shfl_xor_sync(0xffffffffu, a.orig, o);
        b.pos = __shfl_xor_sync(0xffffffffu, a.pos, o);
        if (better(b, a)) a = b;
    }
    return a;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-decomposition device state. Lives in the workspace.
struct State {
    int p;              // pivot position of the current step
    int status;         // kStat* bits
    int rank;           // first j with a negligible |R_jj| (k if none)
    int n_recompute;
    double x0;          // x_j of the current pivot column after the lazy update
    double beta;        // R_jj
    double tau;         // reflector scalar
    double scale;       // 1 / (x_0 - beta): scales x into v with v_0 = 1
    double r00;         // |R_00|
    double rank_tol;    // sqrt(max(m, n)) * eps(working precision)
    double fro2;        // ||X||_F^2 from the initial column norms
};

// Device copy of id_info kept in the workspace.
struct DevInfo {
    id_info info;
    unsigned long long n_gt2;
    unsigned long long max_abs_z_bits;
};

// Z statistics of Definition 1 (count of |Z_ij| > 2, largest |Z_ij|): the
// block's partial counts and maxima (amax >= 0, +inf for a NaN) are reduced in
// shared memory and committed with one atomic of each per block. Every thread
// of the block must call it.
__device__ __forceinline__ void zstats_commit(unsigned long long gt2, double amax, DevInfo* info) {
    __shared__ unsigned long long s_gt2[32];
    __shared__ double s_amax[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gt2 += __shfl_xor_sync(0xffffffffu, gt2, o);
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp, nw = (blockDim.x + kWarp - 1) / kWarp;
    if (lane == 0) {
        s_gt2[w] = gt2;
        s_amax[w] = amax;
    }
    __syncthreads();
    if (w == 0) {
        gt2 = lane < nw ? s_gt2[lane] : 0ull;
        amax = lane < nw ? s_amax[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gt2 += __shfl_xor_sync(0xffffffffu, gt2, o);
            amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        if (lane == 0) {
            if (gt2) atomicAdd(&info->n_gt2, gt2);
            atomicMax(&info->max_abs_z_bits, (unsigned long long)__double_as_longlong(amax));
        }
    }
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace gbid
