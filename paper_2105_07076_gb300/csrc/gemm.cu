// Matrix products of the library: the FP32-accurate 3xTF32 product on the
// tensor cores (tcgen05 + TMA) and the FP64 SIMT product. See gemm.cuh for
// the operand convention and the split.
//
// k_gemm_tf32x3: one 128 x BN output tile per CTA, 6 warps.
//   warp 0 (lane 0)  TMA: per K block of 16 (one 64-byte swizzle row of FP32)
//                    the hi and lo tiles of A (128 x 16) and of B (BN x 16),
//                    64B-swizzled, onto one mbarrier;
//   warp 1 (lane 0)  tcgen05.mma kind::tf32, M = 128, N = BN, K = 8, twice per
//                    K block, three products each (lo_a hi_b, hi_a lo_b,
//                    hi_a hi_b) into one FP32 accumulator in tensor memory;
//                    the stage is released by tcgen05.commit;
//   warps 2-5        epilogue: tcgen05.ld of their 32-lane quarter, the
//                    alpha/beta update and the stores.
// Every mbarrier wait is bounded; on expiry the kernel records kStatTimeout,
// stops issuing, waits (bounded) for the MMAs already issued and frees its
// tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "gemm.cuh"
#include "gbid.h"
#include "tc.cuh"

namespace gbid {
namespace {

constexpr int kGThreads = 192;
constexpr int kGBK = 16;                            // K per stage: 16 FP32 = 64 bytes = one SW64 row
constexpr unsigned long long kGSpin = 1ull << 24;
constexpr size_t kGSmemMax = 200 * 1024;

// CPS CTAs per SM share its shared memory (and tensor memory): with two, one
// CTA's epilogue overlaps the other's main loop.
template <int BN, int CPS> struct GemmShape {
    static constexpr int kStage = 2 * 128 * 64 + 2 * BN * 64;   // A hi/lo + B hi/lo, bytes (multiple of 1024)
    static constexpr int kStages0 = (int)((kGSmemMax / CPS - 1024) / kStage);
    static constexpr int kStages = kStages0 > 8 ? 8 : kStages0;
    static constexpr size_t kSmem = (size_t)kStages * kStage + 1024;
};

struct GParams {
    int M, N, KB, kb_per_split;
    TfEpilogue ep;
    int* status;
};

template <int BN, int CPS>
__global__ void __launch_bounds__(kGThreads, CPS) k_gemm_tf32x3(const __grid_constant__ CUtensorMap tAh,
                                                              const __grid_constant__ CUtensorMap tAl,
                                                              const __grid_constant__ CUtensorMap tBh,
                                                              const __grid_constant__ CUtensorMap tBl, GParams P) {
    using Sh = GemmShape<BN, CPS>;
    constexpr int NS = Sh::kStages;
    extern __shared__ __align__(1024) unsigned char g_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ __align__(8) uint64_t accf;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int t = threadIdx.x, w = t / 32, lane = t % 32;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN, z = blockIdx.z;
    const int kb0 = z * P.kb_per_split;
    const int kb1 = min(P.KB, kb0 + P.kb_per_split);
    const int nkb = kb1 - kb0;   // >= 1 (the host sizes the slices)
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(g_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    volatile int* abrt = &abort_flag;

    if (t == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            tc::mb_init(&full[s], 1);
            tc::mb_init(&empty[s], 1);
        }
        tc::mb_init(&accf, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (w == 0) tc::tmem_alloc(&tmem_base, BN);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;

    if (w == 0) {
        // ---- TMA producer
        if (lane == 0) {
            for (int it = 0; it < nkb; ++it) {
                const int s = it % NS;
                const unsigned use = it / NS;
                if (use > 0 && !tc::mb_wait(&empty[s], (use - 1) & 1u, abrt, kGSpin)) break;
                unsigned char* st = base + (size_t)s * Sh::kStage;
                tc::mb_expect_tx(&full[s], (unsigned)Sh::kStage);
                const int kx = (kb0 + it) * kGBK;
                tc::tma_load_2d(st, &tAh, kx, m0, &full[s]);
                tc::tma_load_2d(st + 128 * 64, &tAl, kx, m0, &full[s]);
                tc::tma_load_2d(st + 2 * 128 * 64, &tBh, kx, n0, &full[s]);
                tc::tma_load_2d(st + 2 * 128 * 64 + BN * 64, &tBl, kx, n0, &full[s]);
            }
        }
        __syncwarp();
    } else if (w == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(128, BN);
            for (int it = 0; it < nkb; ++it) {
                const int s = it % NS;
                if (!tc::mb_wait(&full[s], (it / NS) & 1u, abrt, kGSpin)) break;
                tc::fence_after();
                const unsigned st = tc::su32(base + (size_t)s * Sh::kStage);
                const unsigned ah = st, al = st + 128 * 64, bh = st + 2 * 128 * 64, bl = bh + BN * 64;
#pragma unroll
                for (int kk = 0; kk < kGBK / 8; ++kk) {
                    const unsigned o = kk * 32;   // 8 TF32 = 32 bytes along the swizzled row
                    tc::umma_tf32(tmem, tc::sdesc_sw64(al + o), tc::sdesc_sw64(bh + o), idesc, (it | kk) ? 1u : 0u);
                    tc::umma_tf32(tmem, tc::sdesc_sw64(ah + o), tc::sdesc_sw64(bl + o), idesc, 1u);
                    tc::umma_tf32(tmem, tc::sdesc_sw64(ah + o), tc::sdesc_sw64(bh + o), idesc, 1u);
                }
                tc::umma_commit(&empty[s]);   // stage s free once these MMAs have read it
            }
            tc::umma_commit(&accf);           // every MMA issued so far is complete
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 2..5): accumulators -> alpha acc + beta cin -> d
        const TfEpilogue& E = P.ep;
        const int q4 = w % 4;   // this warp's TMEM lane quarter
        const int i = m0 + q4 * 32 + lane;
        if (E.cin != nullptr) {
            // the addend does not depend on the products: its lines go to L2
            // while the main loop runs (two prefetches cover a misaligned span)
            const int i0w = m0 + q4 * 32, i1w = min(i0w + 31, P.M - 1);
            const int jlim = min(P.N, E.cin_cols);
            if (E.cin_trans) {
                for (int jj = lane; jj < BN && n0 + jj < jlim && i0w < P.M; jj += 32) {
                    const float* row = E.cin + (int64_t)(n0 + jj) * E.ldc;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + i0w));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + i1w));
                }
            } else if (i < P.M) {
                const float* row = E.cin + (int64_t)i * E.ldc;
                for (int c0 = 0; c0 < BN && n0 + c0 < jlim; c0 += 32) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + n0 + c0));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + min(n0 + c0 + 31, jlim - 1)));
                }
            }
        }
        const bool ok = tc::mb_wait(&accf, 0u, abrt, kGSpin);
        tc::fence_after();
        const bool skip = E.skip != nullptr && *E.skip != 0;
        if (ok && !skip) {
            const int64_t zoff = (int64_t)z * E.z_stride;
            float* d = E.d + zoff;
            float* dl = E.d_lo ? E.d_lo + zoff : nullptr;
            const bool vec = !E.d_trans && (E.ldd & 3) == 0 && ((reinterpret_cast<uintptr_t>(d) & 15) == 0) &&
                             (!dl || (reinterpret_cast<uintptr_t>(dl) & 15) == 0);
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                TMEM_LD_X32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0, r);
                tc::tmem_wait_ld();
                if (i >= P.M) continue;
                const int j0 = n0 + c0;
                if (j0 >= P.N) continue;
                float v[32];
                const int jlim = min(P.N, E.cin_cols);
                if (E.cin != nullptr && !E.cin_trans && j0 + 32 <= jlim && (E.ldc & 3) == 0 &&
                    (reinterpret_cast<uintptr_t>(E.cin) & 15) == 0) {
                    // a row segment of the addend: eight 16-byte loads
                    const float4* c4 = reinterpret_cast<const float4*>(E.cin + (int64_t)i * E.ldc + j0);
                    float4 cv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) cv[u] = c4[u];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        v[4 * u] = fmaf(E.beta, cv[u].x, E.alpha * __uint_as_float(r[4 * u]));
                        v[4 * u + 1] = fmaf(E.beta, cv[u].y, E.alpha * __uint_as_float(r[4 * u + 1]));
                        v[4 * u + 2] = fmaf(E.beta, cv[u].z, E.alpha * __uint_as_float(r[4 * u + 2]));
                        v[4 * u + 3] = fmaf(E.beta, cv[u].w, E.alpha * __uint_as_float(r[4 * u + 3]));
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int j = j0 + u;
                        float x = E.alpha * __uint_as_float(r[u]);
                        if (E.cin != nullptr && j < jlim)
                            x = fmaf(E.beta, E.cin_trans ? E.cin[(int64_t)j * E.ldc + i] : E.cin[(int64_t)i * E.ldc + j],
                                     x);
                        v[u] = x;
                    }
                }
                if (vec && j0 + 32 <= P.N) {
                    float4* dh4 = reinterpret_cast<float4*>(d + (int64_t)i * E.ldd + j0);
                    float4* dl4 = dl ? reinterpret_cast<float4*>(dl + (int64_t)i * E.ldd + j0) : nullptr;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (dl4) {
                            float4 h, l;
                            h.x = tf32_hi(v[4 * u]);
                            h.y = tf32_hi(v[4 * u + 1]);
                            h.z = tf32_hi(v[4 * u + 2]);
                            h.w = tf32_hi(v[4 * u + 3]);
                            l.x = v[4 * u] - h.x;
                            l.y = v[4 * u + 1] - h.y;
                            l.z = v[4 * u + 2] - h.z;
                            l.w = v[4 * u + 3] - h.w;
                            dh4[u] = h;
                            dl4[u] = l;
                        } else {
                            dh4[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int j = j0 + u;
                        if (j >= P.N) break;
                        const int64_t o = E.d_trans ? (int64_t)j * E.ldd + i : (int64_t)i * E.ldd + j;
                        if (dl) {
                            const float h = tf32_hi(v[u]);
                            d[o] = h;
                            dl[o] = v[u] - h;
                        } else {
                            d[o] = v[u];
                        }
                    }
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (*abrt) {
        // stopped early: make sure no MMA still writes tensor memory (bounded)
        if (t == 0) {
            unsigned long long spins = 0;
            while (!tc::mb_test(&accf, 0u) && ++spins < kGSpin) __nanosleep(64);
            atomicOr(P.status, kStatTimeout);
        }
        __syncthreads();
    }
    if (w == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, BN);
    }
}

// ------------------------------------------------------------- operand split --
template <typename S>
__global__ void k_split_rows(const S* __restrict__ src, int64_t lds, int rows, int cols, int Kp, float* __restrict__ hi,
                             float* __restrict__ lo, int64_t ldo) {
    const int64_t total = (int64_t)rows * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Kp), c = (int)(e % Kp);
        const float x = c < cols ? (float)src[(int64_t)r * lds + c] : 0.0f;
        const float h = tf32_hi(x);
        hi[(int64_t)r * ldo + c] = h;
        lo[(int64_t)r * ldo + c] = x - h;
    }
}

// Transposed source through a 32 x 32 shared-memory tile: dst(r, c) = S[c * lds + r].
template <typename S>
__global__ void __launch_bounds__(256) k_split_cols(const S* __restrict__ src, int64_t lds, int rows, int cols, int Kp,
                                                    float* __restrict__ hi, float* __restrict__ lo, int64_t ldo) {
    __shared__ float tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int q = ty; q < 32; q += 8) {
        const int c = c0 + q, r = r0 + tx;   // read along r (contiguous in the source)
        tile[q][tx] = (c < cols && r < rows) ? (float)src[(int64_t)c * lds + r] : 0.0f;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, c = c0 + tx;   // write along c
        if (r < rows && c < Kp) {
            const float x = tile[tx][q];
            const float h = tf32_hi(x);
            hi[(int64_t)r * ldo + c] = h;
            lo[(int64_t)r * ldo + c] = x - h;
        }
    }
}

// ----------------------------------------------------------------- FP64 GEMM --
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs per thread (rows
// ty + 16 a, columns tx + 16 b), K in steps of 16 through shared memory.
constexpr int kDT = 64, kDK = 16;

template <int TA, int TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A,
                                               int64_t lda, const double* __restrict__ B, int64_t ldb, double beta,
                                               double* __restrict__ C, int64_t ldc) {
    __shared__ double As[kDK][kDT + 1], Bs[kDK][kDT + 1];
    const int m0 = blockIdx.y * kDT, n0 = blockIdx.x * kDT;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kDK) {
        __syncthreads();
        for (int e = t; e < kDK * kDT; e += 256) {
            // op(A)(i, kk): TA = 1 reads along i (A[kk][i] contiguous), TA = 0 along kk
            const int i = TA ? e % kDT : e / kDK, kk = TA ? e / kDT : e % kDK;
            const int gi = m0 + i, gk = k0 + kk;
            As[kk][i] = (gi < M && gk < K) ? (TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk]) : 0.0;
            // op(B)(kk, j): TB = 0 reads along j, TB = 1 along kk
            const int j = TB ? e / kDK : e % kDT, kb = TB ? e % kDK : e / kDT;
            const int gj = n0 + j, gkb = k0 + kb;
            Bs[kb][j] = (gj < N && gkb < K) ? (TB ? B[(int64_t)gj * ldb + gkb] : B[(int64_t)gkb * ldb + gj]) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kDK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = m0 + ty + 16 * a;
        if (i >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = n0 + tx + 16 * b;
            if (j >= N) continue;
            double* c = C + (int64_t)i * ldc + j;
            *c = beta != 0.0 ? fma(alpha, acc[a][b], beta * *c) : alpha * acc[a][b];
        }
    }
}

// Batched small FP64 products, C_z = alpha A_z B_z + beta C_z (row-major, no
// transposes): 16 x 16 output tiles, one output per thread, so that even a
// few small products spread over the GPU (the FP64 pipe issues about two
// fused multiply-adds per clock per SM, so a product needs every SM).
__global__ void __launch_bounds__(256) k_dgemm16(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                 int64_t lda, int64_t sa, const double* __restrict__ B, int64_t ldb,
                                                 int64_t sb, double beta, double* __restrict__ C, int64_t ldc,
                                                 int64_t sc) {
    __shared__ double As[16][17], Bs[16][17];
    const int z = blockIdx.z;
    A += z * sa;
    B += z * sb;
    C += z * sc;
    const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        __syncthreads();
        As[ty][tx] = (m0 + ty < M && k0 + tx < K) ? A[(int64_t)(m0 + ty) * lda + k0 + tx] : 0.0;
        Bs[ty][tx] = (k0 + ty < K && n0 + tx < N) ? B[(int64_t)(k0 + ty) * ldb + n0 + tx] : 0.0;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    }
    const int i = m0 + ty, j = n0 + tx;
    if (i < M && j < N) {
        double* c = C + (int64_t)i * ldc + j;
        *c = beta != 0.0 ? fma(alpha, acc, beta * *c) : alpha * acc;
    }
}

// ------------------------------------------------------------------- host --
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// FP32 operand rows x kp (row pitch ld elements), boxes of 16 x box_rows, 64-byte swizzle.
bool operand_map(CUtensorMap* map, const float* ptr, int64_t kp, int rows, int64_t ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !ptr || rows < 1) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld & 3)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)kGBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int CPS>
int launch_tf32x3(const TfOperand& A, const TfOperand& B, int M, int N, int K, int splits, const TfEpilogue& ep,
                  int* status, cudaStream_t s) {
    CUtensorMap tAh, tAl, tBh, tBl;
    if (!operand_map(&tAh, A.hi, K, A.rows, A.ld, 128) || !operand_map(&tAl, A.lo, K, A.rows, A.ld, 128) ||
        !operand_map(&tBh, B.hi, K, B.rows, B.ld, BN) || !operand_map(&tBl, B.lo, K, B.rows, B.ld, BN))
        return ID_EINVAL;
    GParams P;
    P.M = M;
    P.N = N;
    P.KB = K / kGBK;
    if (splits < 1) splits = 1;
    if (splits > P.KB) splits = P.KB;
    P.kb_per_split = (P.KB + splits - 1) / splits;
    splits = (P.KB + P.kb_per_split - 1) / P.kb_per_split;   // every slice non-empty
    if (splits > 1 && (ep.cin != nullptr || ep.z_stride == 0)) return ID_EINVAL;
    if (splits > 65535) return ID_EINVAL;
    P.ep = ep;
    P.status = status;
    dim3 grid((N + BN - 1) / BN, (M + 127) / 128, splits);
    if (grid.y > 65535) return ID_EINVAL;
    k_gemm_tf32x3<BN, CPS><<<grid, kGThreads, GemmShape<BN, CPS>::kSmem, s>>>(tAh, tAl, tBh, tBl, P);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

int g_nsm_gemm = 148;   // SMs of the device (set by gemm_configure)

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

__global__ void k_gemm_status(const int* status, DevInfo* info) {
    id_info r = {};
    r.status = (*status & kStatTimeout) ? ID_ETIMEOUT : ID_OK;
    r.err_est = -1.0;
    info->info = r;
}

}  // namespace

template <int BN, int CPS>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(k_gemm_tf32x3<BN, CPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GemmShape<BN, CPS>::kSmem);
}

cudaError_t gemm_configure() {
    cudaError_t e;
    if ((e = configure_one<64, 1>()) != cudaSuccess || (e = configure_one<128, 1>()) != cudaSuccess ||
        (e = configure_one<256, 1>()) != cudaSuccess || (e = configure_one<64, 2>()) != cudaSuccess ||
        (e = configure_one<128, 2>()) != cudaSuccess || (e = configure_one<256, 2>()) != cudaSuccess)
        return e;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
        g_nsm_gemm = nsm;
    return cudaSuccess;
}

template <typename S>
cudaError_t split_tf32(const S* src, int64_t lds, int trans, int rows, int cols, int Kp, float* hi, float* lo,
                       int64_t ldo, cudaStream_t s) {
    if (rows < 1 || Kp < 1) return cudaSuccess;
    if (!trans) {
        const int64_t total = (int64_t)rows * Kp;
        const int64_t g = (total + 255) / 256;
        k_split_rows<S><<<(int)(g < 8192 ? g : 8192), 256, 0, s>>>(src, lds, rows, cols, Kp, hi, lo, ldo);
    } else {
        dim3 grid((Kp + 31) / 32, (rows + 31) / 32);
        if (grid.y > 65535) return cudaErrorInvalidValue;
        k_split_cols<S><<<grid, 256, 0, s>>>(src, lds, rows, cols, Kp, hi, lo, ldo);
    }
    return cudaGetLastError();
}
template cudaError_t split_tf32<float>(const float*, int64_t, int, int, int, int, float*, float*, int64_t,
                                       cudaStream_t);
template cudaError_t split_tf32<double>(const double*, int64_t, int, int, int, int, float*, float*, int64_t,
                                        cudaStream_t);

int gemm_tf32x3(const TfOperand& A, const TfOperand& B, int M, int N, int K, int splits, const TfEpilogue& ep,
                int* status, cudaStream_t s) {
    if (M < 1 || N < 1) return ID_OK;
    if (K < kGBK || K % kGBK != 0 || !ep.d || !status) return ID_EINVAL;
    const int bn = gemm_bn(N);
    // Two CTAs per SM (one's epilogue overlapping the other's main loop) when
    // the grid fills more than one CTA per SM; a grid of at most one wave
    // keeps one CTA per SM and its deeper pipeline.
    const int kb = K / kGBK, sp = splits < 1 ? 1 : (splits > kb ? kb : splits);
    const int64_t ctas = (int64_t)((N + bn - 1) / bn) * ((M + 127) / 128) * sp;
    if (ctas > g_nsm_gemm) {
        if (bn == 64) return launch_tf32x3<64, 2>(A, B, M, N, K, splits, ep, status, s);
        if (bn == 128) return launch_tf32x3<128, 2>(A, B, M, N, K, splits, ep, status, s);
        return launch_tf32x3<256, 2>(A, B, M, N, K, splits, ep, status, s);
    }
    if (bn == 64) return launch_tf32x3<64, 1>(A, B, M, N, K, splits, ep, status, s);
    if (bn == 128) return launch_tf32x3<128, 1>(A, B, M, N, K, splits, ep, status, s);
    return launch_tf32x3<256, 1>(A, B, M, N, K, splits, ep, status, s);
}

cudaError_t dgemm(int ta, int tb, int M, int N, int K, double alpha, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s) {
    if (M < 1 || N < 1) return cudaSuccess;
    dim3 grid((N + kDT - 1) / kDT, (M + kDT - 1) / kDT);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (!ta && !tb) k_dgemm<0, 0><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb) k_dgemm<0, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb) k_dgemm<1, 0><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else k_dgemm<1, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

cudaError_t gemm_status_to_info(const int* status, DevInfo* info, cudaStream_t s) {
    k_gemm_status<<<1, 1, 0, s>>>(status, info);
    return cudaGetLastError();
}

cudaError_t dgemm_batched(int M, int N, int K, double alpha, const double* A, int64_t lda, int64_t sa,
                          const double* B, int64_t ldb, int64_t sb, double beta, double* C, int64_t ldc, int64_t sc,
                          int batch, cudaStream_t s) {
    if (M < 1 || N < 1 || batch < 1) return cudaSuccess;
    dim3 grid((N + 15) / 16, (M + 15) / 16, batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    k_dgemm16<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sa, B, ldb, sb, beta, C, ldc, sc);
    return cudaGetLastError();
}

size_t gemm_f32_bytes(int M, int N, int K) {
    const size_t kp = (size_t)kpad16(K);
    return 2 * al256(4 * (size_t)M * kp) + 2 * al256(4 * (size_t)N * kp);
}

int gemm_f32_ex(int ta, int tb, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                int64_t ldb, float beta, const float* Cin, int64_t ldcin, float* D, int64_t ldd, void* ws, int* status,
                cudaStream_t s) {
    if (M < 1 || N < 1) return ID_OK;
    if (K < 1) return ID_EINVAL;
    const int kp = (int)kpad16(K);
    char* w = static_cast<char*>(ws);
    float* ah = reinterpret_cast<float*>(w);
    float* alo = reinterpret_cast<float*>(w + al256(4 * (size_t)M * kp));
    float* bh = reinterpret_cast<float*>(w + 2 * al256(4 * (size_t)M * kp));
    float* blo = reinterpret_cast<float*>(w + 2 * al256(4 * (size_t)M * kp) + al256(4 * (size_t)N * kp));
    // A operand (M x K): op(A)(i, k); B operand (N x K): op(B)(k, j) read as (j, k)
    if (split_tf32<float>(A, lda, ta ? 1 : 0, M, K, kp, ah, alo, kp, s) != cudaSuccess) return ID_ECUDA;
    if (split_tf32<float>(B, ldb, tb ? 0 : 1, N, K, kp, bh, blo, kp, s) != cudaSuccess) return ID_ECUDA;
    TfOperand oa{ah, alo, kp, M}, ob{bh, blo, kp, N};
    TfEpilogue ep;
    ep.alpha = alpha;
    ep.beta = beta;
    ep.cin = beta != 0.0f ? Cin : nullptr;
    ep.ldc = ldcin;
    ep.d = D;
    ep.ldd = ldd;
    return gemm_tf32x3(oa, ob, M, N, kp, 1, ep, status, s);
}

int gemm_f32(int ta, int tb, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
             int64_t ldb, float beta, float* C, int64_t ldc, void* ws, int* status, cudaStream_t s) {
    return gemm_f32_ex(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, ws, status, s);
}

}  // namespace gbid
