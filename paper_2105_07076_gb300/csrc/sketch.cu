// Gaussian row sketch Y = Omega A on the 5th-generation tensor cores (tcgen05).
//
// Omega: l x m BF16 (row-major), A: m x n FP32 (row-major), Y: l x n FP32.
// As a GEMM: M = l (Omega's rows, padded to 128-row blocks), N = n, K = m.
// One CTA owns all of M (up to kMaxMB blocks of 128 rows, accumulators in
// tensor memory) for BN columns of A, so A is read from HBM exactly once.
//
// Per K block of kBK = 32 (one 64-byte swizzle row of BF16):
//   warp 0 (lane 0)  TMA: Omega block MB x (128 x 32) BF16, 64B-swizzled,
//                    and the FP32 A tile 32 x BN (no swizzle), one mbarrier;
//   warps 2-9        convert the FP32 tile to BF16 (round to nearest even)
//                    and write it K-major, 64B-swizzled: the B operand;
//   warp 1 (lane 0)  tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in TMEM),
//                    M = 128, N = BN, K = 16, twice per 128-row block; the
//                    stage is released by tcgen05.commit.
// Epilogue: warps 2-9 read the accumulators with tcgen05.ld (each warp its
// 32-lane quarter of TMEM, two warps per quarter splitting the 32-column
// chunks) and store Y. kStages stages are in flight.
// One CTA fits an SM, so the column tiles run in waves of #SMs CTAs. When the
// last wave would be short, its tiles are split along K into `parts` slices
// (one more CTA each) so that it fills the SMs; the slices' accumulators go
// to a scratch buffer and k_sketch_tail sums them in slice order.
// Every mbarrier wait is bounded; on expiry the kernel records a timeout,
// stops issuing, waits (bounded) for work already issued and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "cpqr.cuh"
#include "gbid.h"
#include "trace.cuh"

namespace gbid {
namespace {

constexpr int kSkThreads = 320;     // 10 warps: TMA, MMA, eight converter / epilogue warps
constexpr int kConvWarps = 8;
constexpr int kBK = 32;             // K per stage: 32 BF16 = 64 bytes = one SW64 row
constexpr int kStages = 3;
constexpr int kMaxMB = 5;           // l <= 640
constexpr int kTmemCols = 512;
constexpr unsigned long long kSkSpin = 1ull << 24;
constexpr size_t kSkSmemMax = 200 * 1024;   // dynamic shared memory (the static part is ~1 KB)

__device__ __forceinline__ unsigned su32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mb_init(uint64_t* b, unsigned cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false once this CTA gave up (then every later wait returns at once).
__device__ bool mb_wait(uint64_t* b, unsigned parity, volatile int* abort_flag) {
    unsigned long long spins = 0;
    while (!mb_test(b, parity)) {
        if (*abort_flag) return false;
        if (++spins > kSkSpin) {
            *abort_flag = 1;
            return false;
        }
        if (spins > 64) __nanosleep(32);
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw64(unsigned saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading-dimension byte offset (unused when swizzled)
    d |= (uint64_t)(512 >> 4) << 32;                 // stride-dimension byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
    d |= (uint64_t)4 << 61;                          // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                      // D format FP32
           | (1u << 7)                    // A format BF16
           | (1u << 10)                   // B format BF16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

#define TMEM_LD_X32(taddr, r)                                                                                    \
    asm volatile(                                                                                                \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                       \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),        \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),  \
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),            \
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),            \
          "=r"(r[30]), "=r"(r[31])                                                                               \
        : "r"(taddr))

struct SkParams {
    int M, N, K, MB, BN;
    float* Y;
    int64_t ldy;
    int* status;
    int n_full;       // CTAs 0 .. n_full - 1 take whole column tiles
    int parts;        // the later CTAs take K slices of the remaining tiles
    int kb_part;      // K blocks per slice
    float* scratch;   // slice (t, p) of tail tile t: M x BN floats at ((t parts + p) M) BN
};

// Dynamic shared memory, 1024-byte aligned: per stage, MB Omega blocks
// (128 x 64 B), the FP32 A tile (32 x BN x 4 B) and the converted BF16 tile
// (BN x 64 B).
__host__ __device__ inline size_t sk_stage_bytes(int MB, int BN) {
    const size_t om = (size_t)MB * 128 * 64;
    const size_t af = (size_t)kBK * BN * 4;
    const size_t bc = (size_t)BN * 64;
    return (om + af + bc + 1023) / 1024 * 1024;
}

__global__ void __launch_bounds__(kSkThreads, 1) k_sketch(const __grid_constant__ CUtensorMap tm_om,
                                                          const __grid_constant__ CUtensorMap tm_a, SkParams P) {
    extern __shared__ __align__(1024) unsigned char sk_raw[];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t conv[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    __shared__ __align__(8) uint64_t accf;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int t = threadIdx.x, w = t / 32, lane = t % 32;
    const int MB = P.MB, BN = P.BN;
    const int KB_all = (P.K + kBK - 1) / kBK;
    int tile = blockIdx.x, part = -1, kb_lo = 0, kb_hi = KB_all;
    if ((int)blockIdx.x >= P.n_full) {
        const int q = blockIdx.x - P.n_full;
        tile = P.n_full + q / P.parts;
        part = q % P.parts;
        kb_lo = part * P.kb_part;
        kb_hi = min(KB_all, kb_lo + P.kb_part);
    }
    const int n0 = tile * BN;
    const int KB = kb_hi - kb_lo;   // this CTA's K blocks (>= 1: the host sizes the slices)
    const size_t SB = sk_stage_bytes(MB, BN);
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sk_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    auto om_tile = [&](int s, int mb) { return base + (size_t)s * SB + (size_t)mb * 128 * 64; };
    auto af_tile = [&](int s) { return reinterpret_cast<float*>(base + (size_t)s * SB + (size_t)MB * 128 * 64); };
    auto bc_tile = [&](int s) {
        return base + (size_t)s * SB + (size_t)MB * 128 * 64 + (size_t)kBK * BN * 4;
    };
    volatile int* abrt = &abort_flag;

    if (t == 0) {
        abort_flag = 0;
        for (int s = 0; s < kStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&conv[s], kConvWarps);
            mb_init(&empty[s], 1);
        }
        mb_init(&accf, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (w == 0) {
        // ---- TMA producer
        if (lane == 0) {
            const unsigned bytes = (unsigned)(MB * 128 * 64 + kBK * BN * 4);
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % kStages;
                const unsigned use = kb / kStages;
                if (use > 0 && !mb_wait(&empty[s], (use - 1) & 1u, abrt)) break;
                mb_expect_tx(&full[s], bytes);
                const int kx = (kb_lo + kb) * kBK;
                for (int mb = 0; mb < MB; ++mb) tma_load_2d(om_tile(s, mb), &tm_om, kx, mb * 128, &full[s]);
                tma_load_2d(af_tile(s), &tm_a, n0, kx, &full[s]);
            }
        }
        __syncwarp();
    } else if (w == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, BN);
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % kStages;
                if (!mb_wait(&conv[s], (kb / kStages) & 1u, abrt)) break;
                tc_fence_after();
                const unsigned bsm = su32(bc_tile(s));
#pragma unroll 1
                for (int mb = 0; mb < MB; ++mb) {
                    const unsigned asm_ = su32(om_tile(s, mb));
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)
                        umma_bf16(tmem + (uint32_t)(mb * BN), sdesc_sw64(asm_ + kk * 32), sdesc_sw64(bsm + kk * 32),
                                  idesc, (kb | kk) ? 1u : 0u);
                }
                umma_commit(&empty[s]);   // stage s free once these MMAs have read it
            }
            umma_commit(&accf);           // every MMA issued so far is complete
        }
        __syncwarp();
    } else {
        // ---- converters (warps 2..9): FP32 tile -> BF16, K-major, 64-byte swizzle
        const int ct = t - 64;   // 0..32 * kConvWarps - 1
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % kStages;
            if (!mb_wait(&full[s], (kb / kStages) & 1u, abrt)) break;
            const float* af = af_tile(s);
            unsigned char* bc = bc_tile(s);
            for (int u = ct; u < BN * 4; u += 32 * kConvWarps) {
                const int r = u % BN, kc = u / BN;   // row r of the operand (column n0 + r of A), K chunk kc
                uint32_t packed[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float lo = af[(kc * 8 + 2 * q) * BN + r];
                    const float hi = af[(kc * 8 + 2 * q + 1) * BN + r];
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
                    packed[q] = *reinterpret_cast<const uint32_t*>(&h2);
                }
                const int chunk = kc ^ ((r >> 1) & 3);
                *reinterpret_cast<uint4*>(bc + r * 64 + chunk * 16) =
                    make_uint4(packed[0], packed[1], packed[2], packed[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> MMA reads
            __syncwarp();
            if (lane == 0) mb_arrive(&conv[s]);
        }
        // ---- epilogue: accumulators -> Y
        const bool ok = mb_wait(&accf, 0u, abrt);
        tc_fence_after();
        if (ok) {
            const int q4 = w % 4;          // this warp's TMEM lane quarter
            const int half = (w - 2) / 4;  // the two warps of a quarter take alternate 32-column chunks
            for (int mb = 0; mb < MB; ++mb) {
                const int row = mb * 128 + q4 * 32 + lane;
                for (int c0 = 32 * half; c0 < BN; c0 += 64) {
                    uint32_t r[32];
                    TMEM_LD_X32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(mb * BN + c0), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row < P.M && part >= 0) {
                        // a K slice: the whole 32-column chunk to the scratch (16-byte stores)
                        float4* y4 = reinterpret_cast<float4*>(
                            P.scratch + ((int64_t)((tile - P.n_full) * P.parts + part) * P.M + row) * BN + c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            y4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                                __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                    } else if (row < P.M) {
                        float* yrow = P.Y + (int64_t)row * P.ldy + n0 + c0;
                        const int lim = min(32, P.N - (n0 + c0));
                        if (lim == 32 && (P.ldy & 3) == 0 && (reinterpret_cast<uintptr_t>(P.Y) & 15) == 0) {
                            float4* y4 = reinterpret_cast<float4*>(yrow);   // eight 16-byte stores
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                y4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                                    __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (i < lim) yrow[i] = __uint_as_float(r[i]);
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abrt) {
        // stop point reached early: make sure no MMA still writes TMEM (bounded)
        if (t == 0) {
            unsigned long long spins = 0;
            while (!mb_test(&accf, 0u) && ++spins < kSkSpin) __nanosleep(64);
            atomicOr(P.status, kStatTimeout);
        }
        __syncthreads();
    }
    if (w == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Y(row, n0 + c) of the split tail tiles: the sum of their K slices in slice order.
__global__ void __launch_bounds__(256) k_sketch_tail(const float* __restrict__ scratch, int n_full, int ntail,
                                                     int parts, int M, int N, int BN, float* __restrict__ Y,
                                                     int64_t ldy) {
    const int64_t total = (int64_t)ntail * M * BN;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % BN);
        const int64_t rt = e / BN;
        const int row = (int)(rt % M), ti = (int)(rt / M);
        const int col = (n_full + ti) * BN + c;
        if (col >= N) continue;
        float v = 0.0f;
        for (int p = 0; p < parts; ++p) v += scratch[((int64_t)(ti * parts + p) * M + row) * BN + c];
        Y[(int64_t)row * ldy + col] = v;
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

bool make_map_2d(CUtensorMap* map, CUtensorMapDataType dt, size_t esize, const void* ptr, uint64_t inner,
                 uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    (void)esize;
    return fn(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sketch_bn(int MB) {
    // TMEM: MB accumulators of BN FP32 columns in 512 columns; BN a multiple of 16
    // (MMA N constraint for M = 128) and of 32 (epilogue load width).
    int bn = (kTmemCols / MB) / 32 * 32;
    if (bn > 256) bn = 256;
    return bn;
}

}  // namespace

namespace {
int g_sk_nsm = 0;   // SMs of the device (set by sketch_configure)

// The tail split of n columns: slices per tail tile (1: no split) and whole tiles.
void sketch_split(int64_t n, int BN, int* n_full, int* parts, int* ntail) {
    const int tiles = (int)((n + BN - 1) / BN);
    *n_full = tiles;
    *parts = 1;
    *ntail = 0;
    if (g_sk_nsm < 1) return;
    const int tail = tiles % g_sk_nsm;
    if (tail == 0 || tiles < g_sk_nsm) return;
    const int p = std::min(8, g_sk_nsm / tail);
    if (p < 2) return;
    *n_full = tiles - tail;
    *parts = p;
    *ntail = tail;
}
}  // namespace

cudaError_t sketch_configure() {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_sk_nsm, cudaDevAttrMultiProcessorCount, dev);
    return cudaFuncSetAttribute(k_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSkSmemMax);
}

size_t sketch_scratch_bytes(int64_t n, int64_t l) {
    const int MB = (int)((l + 127) / 128);
    if (MB < 1 || MB > kMaxMB) return 0;
    int n_full, parts, ntail;
    sketch_split(n, sketch_bn(MB), &n_full, &parts, &ntail);
    return (size_t)ntail * parts * (size_t)l * sketch_bn(MB) * sizeof(float);
}

int sketch_launch_count(int64_t n, int64_t l, size_t scratch_bytes) {
    const size_t need = sketch_scratch_bytes(n, l);
    return 1 + (need > 0 && scratch_bytes >= need ? 1 : 0);
}

// Y (l x n, ldy) = Omega (l x m BF16, ldo) * A (m x n FP32, lda). Returns an id_status.
int sketch_run(const float* A, int64_t m, int64_t n, int64_t lda, const uint16_t* Om, int64_t l, int64_t ldo, float* Y,
               int64_t ldy, int* status, cudaStream_t s, float* scratch, size_t scratch_bytes) {
    const int MB = (int)((l + 127) / 128);
    if (MB < 1 || MB > kMaxMB) return ID_EINVAL;
    const int BN = sketch_bn(MB);
    CUtensorMap tm_om, tm_a;
    if (!make_map_2d(&tm_om, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Om, (uint64_t)m, (uint64_t)l,
                     (uint64_t)ldo * 2, kBK, 128, CU_TENSOR_MAP_SWIZZLE_64B))
        return ID_EINVAL;
    if (!make_map_2d(&tm_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, (uint64_t)n, (uint64_t)m, (uint64_t)lda * 4,
                     (uint32_t)BN, kBK, CU_TENSOR_MAP_SWIZZLE_NONE))
        return ID_EINVAL;
    SkParams P;
    P.M = (int)l;
    P.N = (int)n;
    P.K = (int)m;
    P.MB = MB;
    P.BN = BN;
    P.Y = Y;
    P.ldy = ldy;
    P.status = status;
    int n_full, parts, ntail;
    sketch_split(n, BN, &n_full, &parts, &ntail);
    const int KB = (int)((m + kBK - 1) / kBK);
    const size_t need = (size_t)ntail * parts * (size_t)l * BN * sizeof(float);
    if (ntail == 0 || scratch == nullptr || scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 15) ||
        KB < parts) {
        n_full = (int)((n + BN - 1) / BN);   // no split: every CTA a whole tile
        parts = 1;
        ntail = 0;
    }
    P.kb_part = (KB + parts - 1) / parts;
    parts = (KB + P.kb_part - 1) / P.kb_part;   // every slice non-empty
    P.n_full = n_full;
    P.parts = parts;
    P.scratch = scratch;
    const size_t smem = (size_t)kStages * sk_stage_bytes(MB, BN) + 1024;
    if (smem > kSkSmemMax) return ID_EINVAL;
    const int grid = n_full + ntail * parts;
    const int tr = trace_begin(TraceKind::kSketch, s);
    k_sketch<<<grid, kSkThreads, smem, s>>>(tm_om, tm_a, P);
    if (ntail > 0) {
        const int64_t tot = (int64_t)ntail * l * BN;
        k_sketch_tail<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(scratch, n_full, ntail, parts,
                                                                                    (int)l, (int)n, BN, Y, ldy);
    }
    trace_end(tr, s);
    return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ECUDA;
}

}  // namespace gbid
