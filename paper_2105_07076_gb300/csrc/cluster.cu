// Small IDs on one thread-block cluster, the matrix held in distributed shared
// memory (Sec. 2.1: CPQR stopped after k pivots, T = R11^{-1} R12, Z).
//
// A cluster of CS CTAs (2..16) splits the n_x columns of X (A, or A^T when
// m > n: the Sec. 2 footnote) into contiguous ranges; CTA r keeps its columns
// in shared memory for the whole decomposition, so after the first read of A
// every step runs from on-chip memory. Per pivot step j:
//   1. each CTA finds its best not-yet-chosen column (largest squared
//      residual norm, ties to the smallest original index) and writes the
//      candidate into every CTA's shared memory;       -- cluster barrier
//   2. every CTA picks the same winner p and applies the same position swap;
//      the CTA that owns p forms the reflector (beta = -sign(x_j) ||x||,
//      v_j = 1, tau = (beta - x_j) / beta), stores R(j, p) and v in its slice,
//      and writes v, beta and tau into every CTA;      -- cluster barrier
//   3. every CTA applies I - tau v v^T to its remaining columns and takes the
//      exact squared residual norms of the updated columns (scaled by a power
//      of two near 1 / the largest column norm).
// Then R11 is gathered from its owners into each CTA and every CTA solves its
// own columns' T = R11^{-1} R12 in FP64 (a warp per four right-hand sides,
// lane = row, R pre-divided by its diagonal) and writes Z. No grid-wide
// barrier, no global-memory scratch: on a 200 x 400 FP64 ID the persistent
// grid kernel spends ~25 us per step in barriers and L2 round trips.
// The cluster barriers are hardware barriers of the cluster's own CTAs, which
// are co-scheduled by the launch; there is no spin-wait on memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "cpqr.cuh"
#include "gbid.h"

namespace cg = cooperative_groups;

namespace gbid {
namespace {

constexpr int kCThreads = 256;
constexpr int kCWarps = kCThreads / kWarp;
constexpr int kCMaxCS = 16;     // 16 needs the non-portable cluster size (checked at run time)
constexpr int kCMaxK = 64;
constexpr int kCMaxRows = 1024;
constexpr size_t kCSmemMax = 225 * 1024;   // dynamic; the static arrays (~0.5 KB) share the 227 KB opt-in

template <typename T>
struct CCand {
    T val;
    int orig;
    int pad;
};

struct CLayout {
    int mxp, nc;
    size_t Ws, nrm, vbuf, perm, ipos, done, r11, total;
};

__host__ __device__ inline size_t c_al(size_t x) { return (x + 15) / 16 * 16; }

template <typename T>
__host__ __device__ inline CLayout c_layout(int mx, int nx, int k, int cs) {
    CLayout L;
    L.mxp = (mx + 3) / 4 * 4;
    L.nc = (nx + cs - 1) / cs;
    size_t off = 0;
    L.Ws = off;
    off = c_al(off + sizeof(T) * (size_t)L.mxp * L.nc);
    L.nrm = off;
    off = c_al(off + sizeof(T) * (size_t)L.nc);
    L.vbuf = off;
    off = c_al(off + sizeof(T) * (size_t)L.mxp);
    L.perm = off;
    off = c_al(off + 4 * (size_t)nx);
    L.ipos = off;
    off = c_al(off + 4 * (size_t)nx);
    L.done = off;
    off = c_al(off + (size_t)L.nc);
    L.r11 = off;
    off = c_al(off + 8 * (size_t)k * (k + 1));
    L.total = off;
    return L;
}

template <typename T>
__device__ __forceinline__ bool c_better(const CCand<T>& a, const CCand<T>& b) {
    return a.val > b.val || (a.val == b.val && a.orig < b.orig);
}

template <typename T>
__device__ CCand<T> c_warp_best(CCand<T> a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CCand<T> b;
        b.val = __shfl_xor_sync(0xffffffffu, a.val, o);
        b.orig = __shfl_xor_sync(0xffffffffu, a.orig, o);
        b.pad = 0;
        if (c_better(b, a)) a = b;
    }
    return a;
}

template <typename T>
__device__ CCand<T> c_block_best(CCand<T> a, CCand<T>* red) {
    a = c_warp_best(a);
    const int w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    __syncthreads();
    if (lane == 0) red[w] = a;
    __syncthreads();
    if (lane < kCWarps) a = red[lane];
    else {
        a.val = T(-1);
        a.orig = 0x7fffffff;
    }
    return c_warp_best(a);
}

template <typename T>
__global__ void __launch_bounds__(kCThreads, 1) k_id_cluster(const T* __restrict__ A, int64_t lda, int trans, int mx,
                                                            int nx, int k, int32_t* J, T* Z, int64_t ldz,
                                                            DevInfo* dinfo) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int r = (int)cluster.block_rank();
    const CLayout L = c_layout<T>(mx, nx, k, cs);
    const int mxp = L.mxp, nc = L.nc;
    extern __shared__ __align__(16) unsigned char smem[];
    T* Ws = reinterpret_cast<T*>(smem + L.Ws);           // Ws[lc * mxp + i]
    T* nrm = reinterpret_cast<T*>(smem + L.nrm);
    T* vbuf = reinterpret_cast<T*>(smem + L.vbuf);
    int* perm = reinterpret_cast<int*>(smem + L.perm);   // position -> column
    int* ipos = reinterpret_cast<int*>(smem + L.ipos);   // column -> position
    unsigned char* done = smem + L.done;
    double* r11 = reinterpret_cast<double*>(smem + L.r11);
    __shared__ CCand<T> cand[2][kCMaxCS];
    __shared__ CCand<T> red[kCWarps];
    __shared__ double scal[2][2];                          // beta, tau per step parity
    __shared__ double redd[kCWarps];
    __shared__ int s_flag;
    const int t = threadIdx.x, lane = t % kWarp, w = t / kWarp;
    const int c0 = r * nc, ncr = max(0, min(nc, nx - c0));   // this CTA's columns [c0, c0 + ncr)
    const double eps = sizeof(T) == 8 ? DBL_EPSILON : (double)FLT_EPSILON;

    // ---- load X's columns, perm, norms
    if (!trans) {
        for (int e = t; e < mx * ncr; e += kCThreads) {
            const int i = e / ncr, lc = e - i * ncr;
            Ws[lc * mxp + i] = A[(int64_t)i * lda + c0 + lc];
        }
    } else {
        for (int e = t; e < mx * ncr; e += kCThreads) {
            const int lc = e / mx, i = e - lc * mx;
            Ws[lc * mxp + i] = A[(int64_t)(c0 + lc) * lda + i];
        }
    }
    for (int l = t; l < nx; l += kCThreads) {
        perm[l] = l;
        ipos[l] = l;
    }
    for (int lc = t; lc < nc; lc += kCThreads) done[lc] = lc < ncr ? 0 : 1;
    if (t == 0) s_flag = 0;
    __syncthreads();
    double cmax = 0.0;                                     // largest squared column norm of this CTA
    for (int lc = w; lc < ncr; lc += kCWarps) {
        double sacc = 0.0;
        for (int i = lane; i < mx; i += kWarp) {
            const double x = (double)Ws[lc * mxp + i];
            sacc = fma(x, x, sacc);
        }
        sacc = warp_sum(sacc);
        if (lane == 0 && !isfinite(sacc)) s_flag = 1;
        cmax = fmax(cmax, sacc);
    }
    // cluster-wide largest norm -> power-of-two scale for the squared norms;
    // a non-finite column anywhere is reported by rank 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    if (lane == 0) redd[w] = cmax;
    __syncthreads();
    if (t == 0 && r != 0 && s_flag) atomicOr(cluster.map_shared_rank(&s_flag, 0), 1);
    cluster.sync();
    T ysc = T(1);
    {
        double gmax = 0.0;
        for (int q = 0; q < cs; ++q) {
            const double* rem = cluster.map_shared_rank(&redd[0], q);
            double v = 0.0;
            for (int g = 0; g < kCWarps; ++g) v = fmax(v, rem[g]);
            gmax = fmax(gmax, v);
        }
        if (sizeof(T) == 4 && gmax > 0.0 && isfinite(gmax)) {   // FP32 squares only
            int e2;
            frexp(sqrt(gmax), &e2);
            ysc = (T)ldexp(1.0, -e2);
        }
    }
    // squared norms of the scaled columns, the convention of the pivot steps
    for (int lc = w; lc < ncr; lc += kCWarps) {
        T sq = T(0);
        for (int i = lane; i < mx; i += kWarp) {
            const T y = Ws[lc * mxp + i] * ysc;
            sq += y * y;
        }
        sq = warp_sum(sq);
        if (lane == 0) nrm[lc] = sq;
    }
    cluster.sync();

    double r00 = 0.0;
    int rank = k;
    const double rank_tol = sqrt((double)nx) * eps;
    for (int j = 0; j < k; ++j) {
        const int par = j & 1;
        // 1. local candidate -> every CTA
        CCand<T> best;
        best.val = T(-1);
        best.orig = 0x7fffffff;
        best.pad = 0;
        for (int lc = t; lc < ncr; lc += kCThreads) {
            if (done[lc]) continue;
            CCand<T> c;
            const T v = nrm[lc];
            c.val = v == v && v < T(INFINITY) ? v : T(-1);
            c.orig = c0 + lc;
            c.pad = 0;
            if (c_better(c, best)) best = c;
        }
        best = c_block_best(best, red);
        if (t < cs) {
            CCand<T>* rem = cluster.map_shared_rank(&cand[par][0], t);
            rem[r] = best;
        }
        cluster.sync();
        // 2. winner, swap, reflector by the owner
        CCand<T> win = cand[par][0];
        for (int q = 1; q < cs; ++q)
            if (c_better(cand[par][q], win)) win = cand[par][q];
        const int pcol = win.orig;
        const int owner = pcol / nc;
        if (t == 0) {
            const int pp = ipos[pcol], cj = perm[j];
            perm[pp] = cj;
            ipos[cj] = pp;
            perm[j] = pcol;
            ipos[pcol] = j;
        }
        if (r == owner) {
            const int lc = pcol - c0;
            if (t == 0) done[lc] = 1;
            T* x = Ws + lc * mxp;
            if (w == 0) {
                double ss = 0.0;
                for (int i = j + 1 + lane; i < mx; i += kWarp) {
                    const double xv = (double)x[i];
                    ss = fma(xv, xv, ss);
                }
                ss = warp_sum(ss);
                const double x0 = (double)x[j];
                const double alpha = sqrt(fma(x0, x0, ss));
                double beta = 0.0, tau = 0.0, scale = 0.0;
                if (alpha != 0.0) {
                    beta = x0 >= 0.0 ? -alpha : alpha;
                    tau = (beta - x0) / beta;
                    scale = 1.0 / (x0 - beta);
                }
                const T scaleT = (T)scale;
                for (int i = j + 1 + lane; i < mx; i += kWarp) x[i] = x[i] * scaleT;
                if (lane == 0) {
                    x[j] = (T)beta;
                    for (int q = 0; q < cs; ++q) {
                        double* rem = cluster.map_shared_rank(&scal[par][0], q);
                        rem[0] = beta;
                        rem[1] = tau;
                    }
                }
            }
            __syncthreads();
            // v (v_j = 1, zero above j) into every CTA
            for (int e = t; e < cs * mxp; e += kCThreads) {
                const int q = e / mxp, i = e - q * mxp;
                T* rem = cluster.map_shared_rank(vbuf, q);
                rem[i] = i < j || i >= mx ? T(0) : (i == j ? T(1) : x[i]);
            }
        }
        cluster.sync();
        const double beta = scal[par][0];
        const T tauT = (T)scal[par][1];
        if (j == 0) r00 = fabs(beta);
        if (rank == k && (r00 == 0.0 || fabs(beta) <= rank_tol * r00)) rank = j;
        // 3. update this CTA's remaining columns; exact scaled squared norms
        for (int lc = w; lc < ncr; lc += kCWarps) {
            if (done[lc]) continue;
            T* y = Ws + lc * mxp;
            T d = T(0);
            for (int i = j + lane; i < mx; i += kWarp) d += vbuf[i] * y[i];
            d = warp_sum(d);
            const T td = tauT * d;
            T sq = T(0);
            for (int i = j + lane; i < mx; i += kWarp) {
                const T yi = y[i] - td * vbuf[i];
                y[i] = yi;
                if constexpr (sizeof(T) == 8) {
                    if (i > j) sq = fma(yi, yi, sq);       // FP64: no range issue, one FMA
                } else {
                    if (i > j) sq += (yi * ysc) * (yi * ysc);
                }
            }
            sq = warp_sum(sq);
            if (lane == 0) nrm[lc] = sq;
        }
        __syncthreads();
    }
    cluster.sync();

    // ---- R11 (FP64, pre-divided by its diagonal above it) from the owners
    for (int e = t; e < k * k; e += kCThreads) {
        const int i = e / k, q = e - i * k;
        double v = 0.0;
        if (i <= q) {
            const int col = perm[q], own = col / nc;
            const T* rem = cluster.map_shared_rank(Ws, own);
            v = (double)rem[(col - own * nc) * mxp + i];
        }
        r11[i * (k + 1) + q] = v;
    }
    __syncthreads();
    for (int e = t; e < k * k; e += kCThreads) {
        const int i = e / k, q = e - i * k;
        if (i < q) r11[i * (k + 1) + q] /= r11[q * (k + 1) + q];
    }
    __syncthreads();

    // ---- T for this CTA's columns (positions >= k), Z
    const bool two = k > kWarp;
    T zmax = T(0);
    float gt2 = 0.0f;
    for (int g0 = 4 * w; g0 < ncr; g0 += 4 * kCWarps) {
        double x[4][2];
        int colq[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int lc = g0 + qq;
            colq[qq] = (lc < ncr && !done[lc]) ? lc : -1;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int i = lane + kWarp * s;
                x[qq][s] = (colq[qq] >= 0 && i < k) ? (double)Ws[colq[qq] * mxp + i] : 0.0;
            }
        }
        for (int i = k - 1; i >= 0; --i) {
            const int own = i % kWarp, sl = i / kWarp;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const double bi = __shfl_sync(0xffffffffu, sl ? x[qq][1] : x[qq][0], own);
                if (lane < i) x[qq][0] = fma(-r11[lane * (k + 1) + i], bi, x[qq][0]);
                if (two && lane + kWarp < i) x[qq][1] = fma(-r11[(lane + kWarp) * (k + 1) + i], bi, x[qq][1]);
            }
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            if (colq[qq] < 0) continue;
            const int col = c0 + colq[qq];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int i = lane + kWarp * s;
                if (i < k) {
                    const T z = (T)(x[qq][s] / r11[i * (k + 1) + i]);
                    Z[(int64_t)i * ldz + col] = z;
                    const T a = fabs(z);
                    zmax = a == a ? fmax(zmax, a) : T(INFINITY);
                    if (a > T(2)) gt2 += 1.0f;
                }
            }
        }
    }
    // identity block and J by rank 0
    if (r == 0) {
        for (int e = t; e < k * k; e += kCThreads) {
            const int i = e / k, l = e - i * k;
            Z[(int64_t)i * ldz + perm[l]] = i == l ? T(1) : T(0);
        }
        for (int l = t; l < k; l += kCThreads) J[l] = perm[l];
    }
    // statistics: block reduction, then one atomic per CTA
    double zm = (double)zmax, g2 = (double)gt2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zm = fmax(zm, __shfl_xor_sync(0xffffffffu, zm, o));
        g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    }
    __syncthreads();
    if (lane == 0) redd[w] = zm;
    __syncthreads();
    if (t == 0) {
        double v = 1.0;   // the identity block holds ones
        for (int g = 0; g < kCWarps; ++g) v = fmax(v, redd[g]);
        atomicMax(&dinfo->max_abs_z_bits, (unsigned long long)__double_as_longlong(v));
    }
    __syncthreads();
    if (lane == 0) redd[w] = g2;
    __syncthreads();
    if (t == 0) {
        double v = 0.0;
        for (int g = 0; g < kCWarps; ++g) v += redd[g];
        if (v > 0.0) atomicAdd(&dinfo->n_gt2, (unsigned long long)v);
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
    if (r == 0 && t == 0) {
        __threadfence();
        id_info res = {};
        res.status = s_flag ? ID_ENONFINITE : (rank < k ? ID_RANK_DEFICIENT : ID_OK);
        res.rank = rank;
        res.transposed = trans;
        res.n_recompute = 0;
        res.r00 = r00;
        res.nb = 0;
        res.engine = 2;
        res.err_est = -1.0;
        dinfo->info = res;
    }
}

__global__ void k_cluster_stats(DevInfo* d) {
    id_info r = d->info;
    r.n_gt2 = (int64_t)d->n_gt2;
    r.max_abs_z = __longlong_as_double((long long)d->max_abs_z_bits);
    d->info = r;
}

// Kernel attributes belong to each device's context: the flags are kept per
// device index (and per dtype).
constexpr int kCMaxDevices = 64;
std::mutex g_cmu;
bool g_cconf[kCMaxDevices][2] = {};
bool g_c16[kCMaxDevices][2] = {};   // a 16-CTA cluster with the largest shared memory is schedulable

int cluster_dev() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCMaxDevices) return 0;
    return dev;
}

template <typename T>
cudaError_t cluster_configure() {
    std::lock_guard<std::mutex> lk(g_cmu);
    const int slot = sizeof(T) == 8 ? 0 : 1;
    const int dev = cluster_dev();
    if (g_cconf[dev][slot]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_id_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCSmemMax);
    if (e != cudaSuccess) return e;
    if (cudaFuncSetAttribute(k_id_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kCThreads);
        cfg.dynamicSmemBytes = kCSmemMax;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 16;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_id_cluster<T>, &cfg) == cudaSuccess && nclusters > 0)
            g_c16[dev][slot] = true;
        cudaGetLastError();   // a refused query leaves no error behind
    }
    g_cconf[dev][slot] = true;
    return cudaSuccess;
}

}  // namespace

// Cluster size for a problem the cluster engine takes (0: it does not).
template <typename T>
int cluster_size(int64_t m, int64_t n, int64_t k) {
    const int64_t mx = m < n ? m : n, nx = m < n ? n : m;
    if (k > kCMaxK || mx > kCMaxRows || nx > 8192) return 0;
    cluster_configure<T>();   // (on a machine without a GPU this fails and the portable cap holds)
    cudaGetLastError();
    const int cap = g_c16[cluster_dev()][sizeof(T) == 8 ? 0 : 1] ? 16 : 8;
    // at least ceil(n_x / 64) CTAs (per-step work per CTA) and at least what
    // fits; FP64 takes the widest cluster (its arithmetic runs at 2 lanes per
    // clock per SM, so every SM counts)
    int cs = 2;
    const int want = sizeof(T) == 8 ? cap : 2;
    while (cs < cap && (cs < want || cs * 64 < nx || c_layout<T>((int)mx, (int)nx, (int)k, cs).total > kCSmemMax))
        cs *= 2;
    while (cs > 2 && (nx + cs - 1) / cs < 4) cs /= 2;   // at least 4 columns per CTA
    return c_layout<T>((int)mx, (int)nx, (int)k, cs).total <= kCSmemMax ? cs : 0;
}

template <typename T>
cudaError_t cluster_run(const void* A, int64_t lda, int trans, int mx, int nx, int k, int32_t* J, void* Z,
                        int64_t ldz, DevInfo* dinfo, cudaStream_t s) {
    const int cs = cluster_size<T>(trans ? nx : mx, trans ? mx : nx, k);
    if (cs == 0) return cudaErrorInvalidValue;
    cudaError_t e = cluster_configure<T>();
    if (e != cudaSuccess) return e;
    const CLayout L = c_layout<T>(mx, nx, k, cs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_id_cluster<T>, static_cast<const T*>(A), lda, trans, mx, nx, k, J,
                           static_cast<T*>(Z), ldz, dinfo);
    if (e != cudaSuccess) return e;
    k_cluster_stats<<<1, 1, 0, s>>>(dinfo);
    return cudaGetLastError();
}

template int cluster_size<double>(int64_t, int64_t, int64_t);
template int cluster_size<float>(int64_t, int64_t, int64_t);
template cudaError_t cluster_run<double>(const void*, int64_t, int, int, int, int, int32_t*, void*, int64_t, DevInfo*,
                                         cudaStream_t);
template cudaError_t cluster_run<float>(const void*, int64_t, int, int, int, int, int32_t*, void*, int64_t, DevInfo*,
                                        cudaStream_t);

}  // namespace gbid
