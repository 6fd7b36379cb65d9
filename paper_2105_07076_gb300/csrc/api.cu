// C ABI of the ID library: argument checks, workspace layout, launch order.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "cpqr.cuh"
#include "gemm.cuh"
#include "gbid.h"
#include "trace.cuh"

namespace gbid {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Panel width actually used.
// FP64: left-looking (nb = k) unless the per-step corrections through all k
// stored reflectors, about 2 k (m + n) FP64 operations per step, would outgrow
// a compact-WY update every 32 steps (about m n per step): FP64 arithmetic is
// the scarce resource.
// FP32: panels of 64. Each panel start recomputes the residual norms exactly,
// which bounds the drift of the FP64 downdate fed by FP32 R entries; the WY
// updates are cheap in FP32.
int pick_nb(id_dtype dt, int m, int n, int k, const id_opts* opts) {
    int nb = (opts && opts->nb > 0) ? opts->nb : 0;
    if (nb == 0) {
        // lazy (nb = k) while re-reading the n x k F panel costs less than the
        // blocked WY update's sweeps over W; else 32-column panels
        const double lazy = 2.0 * k * ((double)m + (double)n);
        const double wy = (double)m * (double)n;
        nb = lazy <= wy ? k : 32;
    }
    if (nb > k) nb = k;
    if (nb > kMaxPanel) nb = kMaxPanel;
    if (nb < 1) nb = 1;
    return nb;
}

struct Layout {
    size_t info, state, W, F, xbuf, ssq, sync, vn1, vn2, perm, tau, part3, aux, T, wy, total;
    int m, n, ldw, nb, ldf;
};

// m, n: working (X) dimensions, m <= n. with_w: reserve W/perm/tau (id_decompose)
// or take them from the caller (id_cpqr). with_t: reserve the FP64 T buffer.
Layout make_layout(id_dtype dt, int m, int n, int k, const id_opts* opts, bool with_w, bool with_t,
                   int ldw = 0) {
    Layout L{};
    const size_t s = dt == ID_F64 ? 8 : 4;
    L.m = m;
    L.n = n;
    L.ldw = ldw > 0 ? ldw : (int)round_up(m, 8);
    L.nb = pick_nb(dt, m, n, k, opts);
    L.ldf = (int)round_up(L.nb, 4);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L.info = take(sizeof(DevInfo));
    L.state = take(sizeof(State));
    L.W = with_w ? take(s * (size_t)L.ldw * n) : 0;
    L.F = take(s * (size_t)L.ldf * n);
    L.xbuf = take(s * (size_t)L.ldw);
    L.ssq = take(8 * (size_t)kMaxParts);
    L.sync = take(sync_bytes(k));
    L.vn1 = take(8 * (size_t)n);
    L.vn2 = take(8 * (size_t)n);
    L.perm = with_w ? take(4 * (size_t)n) : 0;
    L.tau = with_w ? take(8 * (size_t)k) : 0;
    L.part3 = take(sizeof(ArgMax) * kMaxParts);
    L.aux = take(s * kMaxPanel);
    L.T = with_t ? take(8 * (size_t)k * (n - k > 0 ? n - k : 1)) : 0;
    // FP32 panels narrower than k: operand scratch of the tensor-core WY update
    L.wy = (dt == ID_F32 && L.nb < k) ? take(wy_bytes(m, n, L.nb)) : 0;
    L.total = off;
    return L;
}

CpqrPlan make_plan(const Layout& L, char* base, void* W, int32_t* perm, double* tau, int k, int64_t mu, int64_t nu) {
    CpqrPlan P{};
    P.m = L.m;
    P.n = L.n;
    P.ldw = L.ldw;
    P.k = k;
    P.nb = L.nb;
    P.m_user = mu;
    P.n_user = nu;
    P.W = W ? W : base + L.W;
    P.F = base + L.F;
    P.ldf = L.ldf;
    P.xbuf = base + L.xbuf;
    P.ssq = reinterpret_cast<double*>(base + L.ssq);
    P.sync = base + L.sync;
    P.vn1 = reinterpret_cast<double*>(base + L.vn1);
    P.vn2 = reinterpret_cast<double*>(base + L.vn2);
    P.perm = perm ? perm : reinterpret_cast<int*>(base + L.perm);
    P.tau = tau ? tau : reinterpret_cast<double*>(base + L.tau);
    P.part3 = reinterpret_cast<ArgMax*>(base + L.part3);
    P.aux = base + L.aux;
    P.st = reinterpret_cast<State*>(base + L.state);
    P.wy_ws = L.wy ? base + L.wy : nullptr;
    return P;
}

// Kernel launches of cpqr_run on an m x n working matrix: one persistent
// launch, or for FP32 panels narrower than k one launch per panel with the
// tensor-core WY update (two operand splits and the product) between panels
// while rows remain below the panel.
int64_t cpqr_launch_count(id_dtype dt, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    const int nb = pick_nb(dt, (int)m, (int)n, (int)k, opts);
    int64_t c = 1;
    if (dt == ID_F32 && cpqr_short_rows((int)m) && nb <= 32) return c;   // one launch, the WY update inside
    if (dt == ID_F32 && nb < k)
        for (int64_t je = nb; je < k; je += nb) c += 1 + (m > je ? 3 : 0);
    return c;
}

bool sizes_ok(int64_t m, int64_t n, int64_t k) {
    if (m < 1 || n < 1 || k < 1) return false;
    const int64_t mn = m < n ? m : n, mx = m < n ? n : m;
    if (k > mn) return false;
    // k indexes a grid dimension of the Z scatter and sizes the solve's tile
    if (k > 16384) return false;
    // the pivot-step cluster keeps a 1/8 share of a column in shared memory
    // and one GEMV CTA owns at most 256 of 2048 * 256 trailing columns
    if (mx > (int64_t)kMaxParts * 256 || mn > 65536) return false;
    return true;
}

// Kernel attributes (the opt-in to large dynamic shared memory) belong to each
// device's context, so they are set once per device index.
constexpr int kMaxDevices = 64;
std::mutex g_conf_mu;
bool g_conf_done[kMaxDevices] = {};

int configure_once() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    std::lock_guard<std::mutex> lk(g_conf_mu);
    if (g_conf_done[dev]) return 0;
    if (cpqr_configure<double>() != cudaSuccess) return -1;
    if (cpqr_configure<float>() != cudaSuccess) return -1;
    if (solve_configure() != cudaSuccess) return -1;
    if (sketch_configure() != cudaSuccess) return -1;
    if (gemm_configure() != cudaSuccess) return -1;
    g_conf_done[dev] = true;
    return 0;
}

int read_info(const void* work, id_info* info, cudaStream_t s) {
    const DevInfo* d = reinterpret_cast<const DevInfo*>(work);
    if (cudaMemcpyAsync(info, &d->info, sizeof(id_info), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ID_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ID_ECUDA;
    return info->status;
}

// The normal-equation route to Z (opts->zsolve = 1): column IDs on the grid engine.
int zsolve_of(const id_opts* opts) { return opts ? opts->zsolve : 0; }

// Engine choice: the cluster kernel when asked for, or by default when the
// problem fits it (the persistent grid kernel pays grid-wide barriers and L2
// round trips every step, which dominate small problems).
template <typename T>
bool use_cluster(int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    const int eng = opts ? opts->engine : 0;
    if (eng == 1 || zsolve_of(opts) == 1) return false;
    // FP64 arithmetic runs at 2 lanes per clock per SM on this GPU: by default an
    // FP64 problem takes the cluster only when a 16-CTA cluster can hold it
    // (200 x 400, k = 20: 361 us on 16 CTAs, 539 us on 8, 524 us on the grid).
    const int cs = cluster_size<T>(m, n, k);
    if (eng == 0 && sizeof(T) == 8) return cs >= 16;
    return cs > 0;
}

bool engine_ok(id_dtype dt, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    const int eng = opts ? opts->engine : 0;
    if (eng < 0 || eng > 2) return false;
    const int zs = zsolve_of(opts);
    if (zs < 0 || zs > 1 || (zs == 1 && (m > n || eng == 2))) return false;
    if (eng == 2) return (dt == ID_F64 ? cluster_size<double>(m, n, k) : cluster_size<float>(m, n, k)) > 0;
    return true;
}

template <typename T>
int decompose_impl(const void* A, int64_t m, int64_t n, int64_t lda, int64_t k, const id_opts* opts, int32_t* J,
                   void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info, cudaStream_t s) {
    const int trans = m > n ? 1 : 0;
    const int mx = (int)(trans ? n : m), nx = (int)(trans ? m : n);
    const id_dtype dt = sizeof(T) == 8 ? ID_F64 : ID_F32;
    const Layout L = make_layout(dt, mx, nx, (int)k, opts, true, true);
    const bool zs = zsolve_of(opts) == 1;
    if (work_bytes < L.total + (zs ? sampled_z_bytes(m, n, k) : 0)) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    char* base = static_cast<char*>(work);
    if (use_cluster<T>(m, n, k, opts)) {
        DevInfo* d = reinterpret_cast<DevInfo*>(base + L.info);
        if (cudaMemsetAsync(d, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
        if (cluster_run<T>(A, lda, trans, mx, nx, (int)k, J, Z, ldz, d, s) != cudaSuccess) return ID_ECUDA;
        if (info) return read_info(work, info, s);
        return ID_OK;
    }
    CpqrPlan P = make_plan(L, base, nullptr, nullptr, nullptr, (int)k, m, n);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base + L.info);
    if (cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
    if (copy_in<T>(A, lda, trans, P, s) != cudaSuccess) return ID_ECUDA;
    if (cpqr_run<T>(P, s) != cudaSuccess) return ID_ECUDA;
    if (zs) {   // the paper's route: J = P_k, then R_k^T R_k Z = C^T A against A (m <= n here)
        if (finalize_info(P.st, dinfo, (int)k, 0, P.nb, s) != cudaSuccess) return ID_ECUDA;
        if (error_estimate(P.vn1, (int)k, nx, P.st, dinfo, s) != cudaSuccess) return ID_ECUDA;
        if (sample_map_j(P.perm, nullptr, (int)k, J, s) != cudaSuccess) return ID_ECUDA;
        const int rc = sampled_z_run<T>(A, m, n, lda, (int)k, J, P.W, P.ldw, Z, ldz, base + L.total, dinfo, s);
        if (rc != ID_OK) return rc;
        if (info) return read_info(work, info, s);
        return ID_OK;
    }
    double* Tm = reinterpret_cast<double*>(base + L.T);
    const int ldt = nx - (int)k > 0 ? nx - (int)k : 1;
    if (solve_run<T>(P.W, P.ldw, (int)k, nx, Tm, ldt, s) != cudaSuccess) return ID_ECUDA;
    if (scatter_z<T>(P.perm, Tm, ldt, (int)k, nx, Z, ldz, J, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (finalize_info(P.st, dinfo, (int)k, trans, P.nb, s) != cudaSuccess) return ID_ECUDA;
    if (error_estimate(P.vn1, (int)k, nx, P.st, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

template <typename T>
int cpqr_impl(void* X, int64_t m, int64_t n, int64_t ldx, int64_t k, const id_opts* opts, int32_t* perm,
              double* tau, void* work, size_t work_bytes, id_info* info, cudaStream_t s) {
    const id_dtype dt = sizeof(T) == 8 ? ID_F64 : ID_F32;
    const Layout L = make_layout(dt, (int)m, (int)n, (int)k, opts, false, false, (int)ldx);
    if (work_bytes < L.total) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    char* base = static_cast<char*>(work);
    CpqrPlan P = make_plan(L, base, X, perm, tau, (int)k, m, n);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base + L.info);
    if (cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
    if (zero_pad<T>(P, s) != cudaSuccess) return ID_ECUDA;
    if (cpqr_run<T>(P, s) != cudaSuccess) return ID_ECUDA;
    if (finalize_info(P.st, dinfo, (int)k, 0, P.nb, s) != cudaSuccess) return ID_ECUDA;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int64_t rid_ldy(int64_t n) { return (n + 3) / 4 * 4; }

// Workspace of the randomized ID: the CPQR/solve layout of the l x n sketch,
// then Y itself and the sketch kernel's status word.
bool rid_refine(const id_opts* opts) { return !opts || opts->refine >= 0; }

size_t rid_bytes(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts, Layout* out) {
    const Layout L = make_layout(ID_F32, (int)l, (int)n, (int)k, opts, true, true);
    if (out) *out = L;
    const size_t base = L.total + align_up(4 * (size_t)l * rid_ldy(n)) + kAlign;
    return base + (rid_refine(opts) ? refine_bytes(m, n, k) : 0);
}

// Sparse (CSR) input: the matrix is formed in the working layout directly,
// then the grid-engine path of decompose_impl.
template <typename T>
int decompose_csr_impl(const int64_t* rowptr, const int32_t* colind, const void* vals, int64_t m, int64_t n,
                       int64_t nnz, int64_t k, const id_opts* opts, int32_t* J, void* Z, int64_t ldz, void* work,
                       size_t work_bytes, id_info* info, cudaStream_t s) {
    const int trans = m > n ? 1 : 0;
    const int mx = (int)(trans ? n : m), nx = (int)(trans ? m : n);
    const id_dtype dt = sizeof(T) == 8 ? ID_F64 : ID_F32;
    const Layout L = make_layout(dt, mx, nx, (int)k, opts, true, true);
    if (work_bytes < L.total + align_up(16)) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    char* base = static_cast<char*>(work);
    CpqrPlan P = make_plan(L, base, nullptr, nullptr, nullptr, (int)k, m, n);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base + L.info);
    int* flag = reinterpret_cast<int*>(base + L.total);
    if (cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    if (csr_in<T>(rowptr, colind, vals, m, n, nnz, trans, P, flag, s) != cudaSuccess) return ID_ECUDA;
    if (cpqr_run<T>(P, s) != cudaSuccess) return ID_ECUDA;
    double* Tm = reinterpret_cast<double*>(base + L.T);
    const int ldt = nx - (int)k > 0 ? nx - (int)k : 1;
    if (solve_run<T>(P.W, P.ldw, (int)k, nx, Tm, ldt, s) != cudaSuccess) return ID_ECUDA;
    if (scatter_z<T>(P.perm, Tm, ldt, (int)k, nx, Z, ldz, J, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (finalize_info(P.st, dinfo, (int)k, trans, P.nb, s, flag) != cudaSuccess) return ID_ECUDA;
    if (error_estimate(P.vn1, (int)k, nx, P.st, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

}  // namespace
}  // namespace gbid

using namespace gbid;

extern "C" {

size_t id_cpqr_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k, const id_opts* opts) {
    if ((dtype != ID_F64 && dtype != ID_F32) || !sizes_ok(m, n, k) || m > n || ldx < m || ldx % 8 != 0) return 0;
    return make_layout(dtype, (int)m, (int)n, (int)k, opts, false, false, (int)ldx).total;
}

size_t id_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    if ((dtype != ID_F64 && dtype != ID_F32) || !sizes_ok(m, n, k)) return 0;
    const int zs = zsolve_of(opts);
    if (zs < 0 || zs > 1 || (zs == 1 && m > n)) return 0;
    const int mx = (int)(m > n ? n : m), nx = (int)(m > n ? m : n);
    return make_layout(dtype, mx, nx, (int)k, opts, true, true).total + (zs ? sampled_z_bytes(m, n, k) : 0);
}

int id_decompose(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const id_opts* opts,
                 int32_t* J, void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!A || !J || !Z || !work) return ID_EINVAL;
    if (dtype != ID_F64 && dtype != ID_F32) return ID_EINVAL;
    if (!sizes_ok(m, n, k)) return ID_EINVAL;
    const int64_t nz = m > n ? m : n;
    if (lda < n || ldz < nz) return ID_EINVAL;
    if (!aligned(work, 256)) return ID_EINVAL;
    if (opts && opts->nb < 0) return ID_EINVAL;
    if (!engine_ok(dtype, m, n, k, opts)) return ID_EINVAL;
    if (zsolve_of(opts) == 1 && (lda > INT32_MAX || ldz > INT32_MAX)) return ID_EINVAL;   // the FP64 GEMMs' ints
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == ID_F64) return decompose_impl<double>(A, m, n, lda, k, opts, J, Z, ldz, work, work_bytes, info, s);
    return decompose_impl<float>(A, m, n, lda, k, opts, J, Z, ldz, work, work_bytes, info, s);
}

size_t id_decompose_host_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    const size_t base = id_workspace_size(dtype, m, n, k, opts);
    if (!base) return 0;
    const size_t s = dtype == ID_F64 ? 8 : 4;
    const int64_t nz = m > n ? m : n;
    return base + align_up(s * (size_t)m * n) + align_up(4 * (size_t)k) + align_up(s * (size_t)k * nz);
}

int id_decompose_host(const void* A_host, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                      const id_opts* opts, int32_t* J_host, void* Z_host, int64_t ldz, void* work, size_t work_bytes,
                      id_info* info, void* stream) {
    if (!A_host || !J_host || !Z_host || !work) return ID_EINVAL;
    if (dtype != ID_F64 && dtype != ID_F32) return ID_EINVAL;
    if (!sizes_ok(m, n, k)) return ID_EINVAL;
    const int64_t nz = m > n ? m : n;
    if (lda < n || ldz < nz) return ID_EINVAL;
    if (!aligned(work, 256)) return ID_EINVAL;
    const size_t need = id_decompose_host_workspace_size(dtype, m, n, k, opts);
    if (work_bytes < need) return ID_ENOMEM;
    const size_t s = dtype == ID_F64 ? 8 : 4;
    const size_t base = id_workspace_size(dtype, m, n, k, opts);
    char* w = static_cast<char*>(work);
    char* dA = w + base;
    int32_t* dJ = reinterpret_cast<int32_t*>(dA + align_up(s * (size_t)m * n));
    char* dZ = reinterpret_cast<char*>(dJ) + align_up(4 * (size_t)k);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpy2DAsync(dA, s * n, A_host, s * lda, s * n, m, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ID_ECUDA;
    const int rc = id_decompose(dA, dtype, m, n, n, k, opts, dJ, dZ, nz, work, base, nullptr, stream);
    if (rc != ID_OK) return rc;
    if (cudaMemcpyAsync(J_host, dJ, 4 * (size_t)k, cudaMemcpyDeviceToHost, st) != cudaSuccess) return ID_ECUDA;
    if (cudaMemcpy2DAsync(Z_host, s * ldz, dZ, s * nz, s * nz, k, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ID_ECUDA;
    id_info tmp;
    id_info* out = info ? info : &tmp;
    return read_info(work, out, st);
}

int id_cpqr(void* X, id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k, const id_opts* opts,
            int32_t* perm, double* tau, void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!X || !perm || !tau || !work) return ID_EINVAL;
    if (dtype != ID_F64 && dtype != ID_F32) return ID_EINVAL;
    if (!sizes_ok(m, n, k) || m > n) return ID_EINVAL;
    if (ldx < m || ldx % 8 != 0) return ID_EINVAL;
    if (!aligned(work, 256) || !aligned(X, 16)) return ID_EINVAL;
    if (opts && opts->nb < 0) return ID_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == ID_F64) return cpqr_impl<double>(X, m, n, ldx, k, opts, perm, tau, work, work_bytes, info, s);
    return cpqr_impl<float>(X, m, n, ldx, k, opts, perm, tau, work, work_bytes, info, s);
}

int id_cpqr_residual_norms(const void* work, id_dtype dtype, int64_t m, int64_t n, int64_t ldx, int64_t k,
                           const id_opts* opts, double* out, void* stream) {
    if (!work || !out) return ID_EINVAL;
    if (id_cpqr_workspace_size(dtype, m, n, ldx, k, opts) == 0) return ID_EINVAL;
    const Layout L = make_layout(dtype, (int)m, (int)n, (int)k, opts, false, false, (int)ldx);
    const char* base = static_cast<const char*>(work);
    return norms_from_squares(reinterpret_cast<const double*>(base + L.vn1), out, (int)n,
                              static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? ID_OK
               : ID_ECUDA;
}

int id_solve(const void* X, id_dtype dtype, int64_t n, int64_t ldx, int64_t k, double* T, int64_t ldt, void* stream) {
    if (!X || !T) return ID_EINVAL;
    if (dtype != ID_F64 && dtype != ID_F32) return ID_EINVAL;
    if (k < 1 || n < k || ldx < k || (n > k && ldt < n - k)) return ID_EINVAL;
    if (n > ((int64_t)1 << 30) || ldx > ((int64_t)1 << 30)) return ID_EINVAL;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = dtype == ID_F64 ? solve_run<double>(X, (int)ldx, (int)k, (int)n, T, (int)ldt, s)
                                    : solve_run<float>(X, (int)ldx, (int)k, (int)n, T, (int)ldt, s);
    return e == cudaSuccess ? ID_OK : ID_ECUDA;
}

size_t id_sketch_workspace_size(void) { return 1024; }

size_t id_sketch_scratch_size(int64_t n, int64_t l) {
    if (n < 1 || l < 1 || l > 640 || n > ((int64_t)1 << 31) - 1) return 0;
    if (configure_once()) return 0;
    return sketch_scratch_bytes(n, l);
}

size_t id_rid_workspace_size(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts) {
    if (m < 1 || n < 1 || k < 1 || l < k || l > 640 || l > m || m > n || !sizes_ok(l, n, k)) return 0;
    return rid_bytes(m, n, l, k, opts, nullptr);
}

int id_decompose_randomized(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda,
                            const uint16_t* Omega_bf16, int64_t l, int64_t ldo, int64_t k, const id_opts* opts,
                            int32_t* J, void* Z, int64_t ldz, void* work, size_t work_bytes, id_info* info,
                            void* stream) {
    if (!A || !Omega_bf16 || !J || !Z || !work) return ID_EINVAL;
    if (dtype != ID_F32) return ID_EINVAL;
    const size_t need = id_rid_workspace_size(m, n, l, k, opts);
    if (need == 0) return ID_EINVAL;
    if (lda < n || lda % 4 != 0 || ldo < m || ldo % 8 != 0 || ldz < n) return ID_EINVAL;
    if (lda > INT32_MAX || ldz > INT32_MAX) return ID_EINVAL;   // leading dimensions of the refinement's GEMMs
    if (!aligned(A, 16) || !aligned(Omega_bf16, 16) || !aligned(work, 256)) return ID_EINVAL;
    if (opts && opts->nb < 0) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L;
    rid_bytes(m, n, l, k, opts, &L);
    char* base = static_cast<char*>(work);
    const int64_t ldy = rid_ldy(n);
    float* Y = reinterpret_cast<float*>(base + L.total);
    int* sk_status = reinterpret_cast<int*>(base + L.total + align_up(4 * (size_t)l * ldy));
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base + L.info);
    if (cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
    if (cudaMemsetAsync(sk_status, 0, sizeof(int), s) != cudaSuccess) return ID_ECUDA;
    // 1. Y = Omega A (tensor cores); the CPQR's working matrix, not yet in use, is the
    // scratch of the sketch's K-split last wave
    CpqrPlan P = make_plan(L, base, nullptr, nullptr, nullptr, (int)k, l, n);
    int rc = sketch_run(static_cast<const float*>(A), m, n, lda, Omega_bf16, l, ldo, Y, ldy, sk_status, s,
                        static_cast<float*>(P.W), sizeof(float) * (size_t)P.ldw * (size_t)n);
    if (rc != ID_OK) return rc;
    // 2. k-step CPQR of Y (FP32 matrix, FP64 norms), 3. T = R11^{-1} R12 of Y in FP64, 4. Z
    if (copy_in<float>(Y, ldy, 0, P, s) != cudaSuccess) return ID_ECUDA;
    if (cpqr_run<float>(P, s) != cudaSuccess) return ID_ECUDA;
    double* Tm = reinterpret_cast<double*>(base + L.T);
    const int ldt = (int)n - (int)k > 0 ? (int)n - (int)k : 1;
    // with the refinement on, this T only seeds the least-squares step: FP32 arithmetic suffices
    if (solve_run<float>(P.W, P.ldw, (int)k, (int)n, Tm, ldt, s, rid_refine(opts)) != cudaSuccess) return ID_ECUDA;
    if (scatter_z<float>(P.perm, Tm, ldt, (int)k, (int)n, Z, ldz, J, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (finalize_info(P.st, dinfo, (int)k, 0, P.nb, s, sk_status) != cudaSuccess) return ID_ECUDA;
    // 5. one least-squares refinement of T against A_J
    if (rid_refine(opts)) {
        void* rws = base + L.total + align_up(4 * (size_t)l * ldy) + kAlign;
        rc = refine_run(static_cast<const float*>(A), m, n, lda, (int)k, J, static_cast<float*>(Z), ldz, rws, dinfo,
                        s);
        if (rc != ID_OK) return rc;
    }
    if (info) return read_info(work, info, s);
    return ID_OK;
}

// ---------------------------------------------------------------- Optim RID --
namespace {
size_t sampled_bytes(id_dtype dt, int64_t m, int64_t n, int64_t p, int64_t k, const id_opts* opts, Layout* out) {
    const Layout L = make_layout(dt, (int)m, (int)p, (int)k, opts, true, false);
    if (out) *out = L;
    return L.total + align_up(4 * (size_t)p) + sampled_z_bytes(m, n, k);
}

bool sampled_sizes_ok(int64_t m, int64_t n, int64_t p, int64_t k) {
    if (m < 1 || n < 1 || p < 1 || k < 1 || p > n || k > p || k > m || k > 16384) return false;
    if (m > ((int64_t)1 << 31) - 1 || n > ((int64_t)1 << 31) - 1) return false;
    return sizes_ok(m, p, k);
}
}  // namespace

size_t id_sampled_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t p, int64_t k, const id_opts* opts) {
    if ((dtype != ID_F64 && dtype != ID_F32) || !sampled_sizes_ok(m, n, p, k)) return 0;
    return sampled_bytes(dtype, m, n, p, k, opts, nullptr);
}

int id_decompose_sampled(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, const int32_t* idx,
                         int64_t p, int64_t k, const id_opts* opts, int32_t* J, void* Z, int64_t ldz, void* work,
                         size_t work_bytes, id_info* info, void* stream) {
    if (!A || !idx || !J || !Z || !work) return ID_EINVAL;
    const size_t need = id_sampled_workspace_size(dtype, m, n, p, k, opts);
    if (need == 0) return ID_EINVAL;
    if (lda < n || ldz < n || !aligned(work, 256)) return ID_EINVAL;
    if (lda > INT32_MAX || ldz > INT32_MAX) return ID_EINVAL;   // leading dimensions of the FP64 GEMMs
    if (opts && opts->nb < 0) return ID_EINVAL;
    {   // the sample: distinct indices in [0, n)
        std::vector<unsigned char> seen((size_t)n, 0);
        for (int64_t l = 0; l < p; ++l) {
            if (idx[l] < 0 || idx[l] >= n || seen[(size_t)idx[l]]) return ID_EINVAL;
            seen[(size_t)idx[l]] = 1;
        }
    }
    if (work_bytes < need) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Layout L;
    sampled_bytes(dtype, m, n, p, k, opts, &L);
    char* base = static_cast<char*>(work);
    int32_t* idx_dev = reinterpret_cast<int32_t*>(base + L.total);
    void* zws = base + L.total + align_up(4 * (size_t)p);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base + L.info);
    if (cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s) != cudaSuccess) return ID_ECUDA;
    if (cudaMemcpyAsync(idx_dev, idx, 4 * (size_t)p, cudaMemcpyHostToDevice, s) != cudaSuccess) return ID_ECUDA;
    CpqrPlan P = make_plan(L, base, nullptr, nullptr, nullptr, (int)k, m, p);
    const bool f64 = dtype == ID_F64;
    // 1. A_S = A[:, idx] into the working layout, 2. k CPQR steps on it
    if ((f64 ? sample_gather_run<double>(A, lda, (int)m, idx_dev, (int)p, P.W, P.ldw, s)
             : sample_gather_run<float>(A, lda, (int)m, idx_dev, (int)p, P.W, P.ldw, s)) != cudaSuccess)
        return ID_ECUDA;
    if ((f64 ? cpqr_run<double>(P, s) : cpqr_run<float>(P, s)) != cudaSuccess) return ID_ECUDA;
    if (finalize_info(P.st, dinfo, (int)k, 0, P.nb, s) != cudaSuccess) return ID_ECUDA;
    // 3. J = idx[P_k], 4. Z from the normal equations against all of A
    if (sample_map_j(P.perm, idx_dev, (int)k, J, s) != cudaSuccess) return ID_ECUDA;
    const int rc = f64 ? sampled_z_run<double>(A, m, n, lda, (int)k, J, P.W, P.ldw, Z, ldz, zws, dinfo, s)
                       : sampled_z_run<float>(A, m, n, lda, (int)k, J, P.W, P.ldw, Z, ldz, zws, dinfo, s);
    if (rc != ID_OK) return rc;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

size_t id_backward_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k) {
    if (dtype != ID_F32 || m < 1 || n < 1 || k < 1 || k > m || m > n || k > 16384) return 0;
    if (m > ((int64_t)1 << 31) - 1 || n > ((int64_t)1 << 31) - 1) return 0;
    return align_up(sizeof(DevInfo)) + backward_bytes(m, n, k);
}

int id_backward(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J,
                const void* Z, int64_t ldz, const void* dZ, int64_t lddz, void* dA, int64_t ldda, void* work,
                size_t work_bytes, id_info* info, void* stream) {
    if (!A || !J || !Z || !dZ || !dA || !work) return ID_EINVAL;
    const size_t need = id_backward_workspace_size(dtype, m, n, k);
    if (need == 0) return ID_EINVAL;
    if (lda < n || ldz < n || lddz < n || ldda < n || !aligned(work, 256)) return ID_EINVAL;
    if (lda > INT32_MAX || ldz > INT32_MAX || lddz > INT32_MAX || ldda > INT32_MAX) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevInfo* dinfo = static_cast<DevInfo*>(work);
    if (refine_info_init(dinfo, (int)k, s) != cudaSuccess) return ID_ECUDA;
    const int rc = backward_run(static_cast<const float*>(A), m, n, lda, (int)k, J, static_cast<const float*>(Z), ldz,
                                static_cast<const float*>(dZ), lddz, static_cast<float*>(dA), ldda,
                                static_cast<char*>(work) + align_up(sizeof(DevInfo)), dinfo, s);
    if (rc != ID_OK) return rc;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

size_t id_refine_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k) {
    if (dtype != ID_F32 || m < 1 || n < 1 || k < 1 || k > m || m > n || k > 16384) return 0;
    if (m > ((int64_t)1 << 31) - 1 || n > ((int64_t)1 << 31) - 1) return 0;
    return align_up(sizeof(DevInfo)) + refine_bytes(m, n, k);
}

int id_refine(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J, void* Z,
              int64_t ldz, void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!A || !J || !Z || !work) return ID_EINVAL;
    const size_t need = id_refine_workspace_size(dtype, m, n, k);
    if (need == 0) return ID_EINVAL;
    if (lda < n || ldz < n || !aligned(work, 256)) return ID_EINVAL;
    if (lda > INT32_MAX || ldz > INT32_MAX) return ID_EINVAL;   // leading dimensions of the GEMMs
    if (work_bytes < need) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevInfo* dinfo = static_cast<DevInfo*>(work);
    if (refine_info_init(dinfo, (int)k, s) != cudaSuccess) return ID_ECUDA;
    const int rc = refine_run(static_cast<const float*>(A), m, n, lda, (int)k, J, static_cast<float*>(Z), ldz,
                              static_cast<char*>(work) + align_up(sizeof(DevInfo)), dinfo, s);
    if (rc != ID_OK) return rc;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

int id_sketch(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, const uint16_t* Omega_bf16, int64_t l,
              int64_t ldo, float* Y, int64_t ldy, void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!A || !Omega_bf16 || !Y || !work) return ID_EINVAL;
    if (dtype != ID_F32) return ID_EINVAL;
    if (m < 1 || n < 1 || l < 1 || l > 640 || m > ((int64_t)1 << 31) - 1 || n > ((int64_t)1 << 31) - 1)
        return ID_EINVAL;
    if (lda < n || lda % 4 != 0 || ldo < m || ldo % 8 != 0 || ldy < n) return ID_EINVAL;
    if (!aligned(A, 16) || !aligned(Omega_bf16, 16) || !aligned(work, 256)) return ID_EINVAL;
    if (work_bytes < id_sketch_workspace_size()) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(work);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base);
    State* st = reinterpret_cast<State*>(base + align_up(sizeof(DevInfo)));
    if (cudaMemsetAsync(work, 0, id_sketch_workspace_size(), s) != cudaSuccess) return ID_ECUDA;
    // the split of a short last wave, when the caller's workspace has room for it
    float* scratch = work_bytes >= id_sketch_workspace_size() + sketch_scratch_bytes(n, l)
                         ? reinterpret_cast<float*>(base + id_sketch_workspace_size())
                         : nullptr;
    const int rc = sketch_run(static_cast<const float*>(A), m, n, lda, Omega_bf16, l, ldo, Y, ldy, &st->status, s,
                              scratch, work_bytes - id_sketch_workspace_size());
    if (rc != ID_OK) return rc;
    if (finalize_info(st, dinfo, 0, 0, 0, s) != cudaSuccess) return ID_ECUDA;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

int id_info_read(const void* work, id_info* info, void* stream) {
    if (!work || !info) return ID_EINVAL;
    return read_info(work, info, static_cast<cudaStream_t>(stream));
}

int64_t id_rid_launch_count(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts) {
    if (id_rid_workspace_size(m, n, l, k, opts) == 0) return -1;
    // sketch (and the sum of its K-split last wave), copy-in, CPQR of the sketch, solve (when
    // n > k), Z scatter, status, refinement
    const size_t w_bytes = sizeof(float) * (size_t)round_up(l, 8) * (size_t)n;
    return 3 + sketch_launch_count(n, l, w_bytes) + cpqr_launch_count(ID_F32, l, n, k, opts) + (n > k ? 1 : 0) +
           (rid_refine(opts) ? refine_launch_count(m, n, k) : 0);
}

int64_t id_launch_count(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    if ((dtype != ID_F64 && dtype != ID_F32) || !sizes_ok(m, n, k) || !engine_ok(dtype, m, n, k, opts)) return -1;
    if (zsolve_of(opts) == 1) return -1;   // not counted: the launches of the blocked inverse depend on k
    const bool cl = dtype == ID_F64 ? use_cluster<double>(m, n, k, opts) : use_cluster<float>(m, n, k, opts);
    if (cl) return 2;   // the cluster kernel and its statistics kernel
    const int64_t nx = m > n ? m : n, mx = m > n ? n : m;
    // copy-in, CPQR, back substitution (when n > k), Z scatter, status, error estimate
    return 4 + cpqr_launch_count(dtype, mx, nx, k, opts) + (nx > k ? 1 : 0);
}

size_t id_reconstruct_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, int32_t transposed) {
    if (dtype != ID_F64 && dtype != ID_F32) return 0;
    if (m < 1 || n < 1 || k < 1 || k > (transposed ? m : n) || m > INT32_MAX || n > INT32_MAX) return 0;
    if (transposed != 0 && transposed != 1) return 0;
    return align_up(sizeof(DevInfo)) + reconstruct_bytes(m, n, k, transposed, dtype == ID_F64 ? 8 : 4);
}

int id_reconstruct(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k, const int32_t* J,
                   const void* Z, int64_t ldz, int32_t transposed, void* Out, int64_t ldo, void* work,
                   size_t work_bytes, id_info* info, void* stream) {
    if (!A || !J || !Z || !Out || !work) return ID_EINVAL;
    const size_t need = id_reconstruct_workspace_size(dtype, m, n, k, transposed);
    if (need == 0) return ID_EINVAL;
    const int64_t zw = transposed ? m : n;
    if (lda < n || ldo < n || ldz < zw || lda > INT32_MAX || ldo > INT32_MAX || ldz > INT32_MAX) return ID_EINVAL;
    if (!aligned(work, 256)) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(work);
    void* rws = static_cast<char*>(work) + align_up(sizeof(DevInfo));
    const int rc = dtype == ID_F64
                       ? reconstruct_run<double>(A, m, n, lda, (int)k, J, Z, ldz, transposed, Out, ldo, rws, dinfo, s)
                       : reconstruct_run<float>(A, m, n, lda, (int)k, J, Z, ldz, transposed, Out, ldo, rws, dinfo, s);
    if (rc != ID_OK) return rc;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

size_t id_gemm_workspace_size(id_dtype dtype, int64_t M, int64_t N, int64_t K) {
    if (dtype != ID_F64 && dtype != ID_F32) return 0;
    if (M < 1 || N < 1 || K < 1 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX - 16) return 0;
    const size_t head = align_up(sizeof(DevInfo)) + kAlign;
    return head + (dtype == ID_F32 ? gemm_f32_bytes((int)M, (int)N, (int)K) : 0);
}

int id_gemm(id_dtype dtype, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K, double alpha, const void* A,
            int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, void* work, size_t work_bytes,
            id_info* info, void* stream) {
    if (!A || !B || !C || !work || (ta != 0 && ta != 1) || (tb != 0 && tb != 1)) return ID_EINVAL;
    const size_t need = id_gemm_workspace_size(dtype, M, N, K);
    if (need == 0) return ID_EINVAL;
    // row widths: op(A) M x K is stored M x K (ta = 0) or K x M; likewise B, C
    if (lda < (ta ? M : K) || ldb < (tb ? K : N) || ldc < N) return ID_EINVAL;
    if (!aligned(work, 256)) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    if (configure_once()) return ID_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(work);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(base);
    int* status = reinterpret_cast<int*>(base + align_up(sizeof(DevInfo)));
    if (cudaMemsetAsync(base, 0, align_up(sizeof(DevInfo)) + kAlign, s) != cudaSuccess) return ID_ECUDA;
    int rc = ID_OK;
    if (dtype == ID_F64) {
        if (dgemm(ta, tb, (int)M, (int)N, (int)K, alpha, static_cast<const double*>(A), lda,
                  static_cast<const double*>(B), ldb, beta, static_cast<double*>(C), ldc, s) != cudaSuccess)
            return ID_ECUDA;
    } else {
        rc = gemm_f32(ta, tb, (int)M, (int)N, (int)K, (float)alpha, static_cast<const float*>(A), lda,
                      static_cast<const float*>(B), ldb, (float)beta, static_cast<float*>(C), ldc,
                      base + align_up(sizeof(DevInfo)) + kAlign, status, s);
        if (rc != ID_OK) return rc;
    }
    if (gemm_status_to_info(status, dinfo, s) != cudaSuccess) return ID_ECUDA;
    if (info) return read_info(work, info, s);
    return ID_OK;
}

size_t id_csr_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    if (opts && (opts->engine == 2 || opts->zsolve != 0)) return 0;
    const size_t w = id_workspace_size(dtype, m, n, k, opts);
    return w ? w + align_up(16) : 0;
}

int id_decompose_csr(const int64_t* rowptr, const int32_t* colind, const void* values, id_dtype dtype, int64_t m,
                     int64_t n, int64_t nnz, int64_t k, const id_opts* opts, int32_t* J, void* Z, int64_t ldz,
                     void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!rowptr || !J || !Z || !work || nnz < 0 || (nnz > 0 && (!colind || !values))) return ID_EINVAL;
    const size_t need = id_csr_workspace_size(dtype, m, n, k, opts);
    if (need == 0) return ID_EINVAL;
    if (ldz < (m > n ? m : n) || !aligned(work, 256)) return ID_EINVAL;
    if (opts && opts->nb < 0) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == ID_F64)
        return decompose_csr_impl<double>(rowptr, colind, values, m, n, nnz, k, opts, J, Z, ldz, work, work_bytes,
                                          info, s);
    return decompose_csr_impl<float>(rowptr, colind, values, m, n, nnz, k, opts, J, Z, ldz, work, work_bytes, info, s);
}

// Two-sided ID: stage 1 on A (a column ID for m <= n, a row ID for m > n),
// then the other ID of the skeleton S (m x k, or k x n). Regions: stage 1's
// workspace, S, a flag word, stage 2's workspace.
namespace {
struct TwoSided {
    size_t ws1, S, flag, ws2, total;
    int64_t sm, sn;   // S is sm x sn row-major
    bool second;      // stage 2 runs an ID (S is not k x k)
};
bool two_sided_layout(id_dtype dt, int64_t m, int64_t n, int64_t k, const id_opts* opts, TwoSided* L) {
    const size_t w1 = id_workspace_size(dt, m, n, k, opts);
    if (!w1) return false;
    L->sm = m <= n ? m : k;
    L->sn = m <= n ? k : n;
    L->second = m <= n ? m > k : n > k;
    const size_t w2 = L->second ? id_workspace_size(dt, L->sm, L->sn, k, nullptr) : align_up(sizeof(DevInfo));
    if (!w2) return false;
    const size_t s = dt == ID_F64 ? 8 : 4;
    L->ws1 = 0;
    L->S = align_up(w1);
    L->flag = L->S + align_up(s * (size_t)L->sm * L->sn);
    L->ws2 = L->flag + align_up(16);
    L->total = L->ws2 + align_up(w2);
    return true;
}
}  // namespace

size_t id_two_sided_workspace_size(id_dtype dtype, int64_t m, int64_t n, int64_t k, const id_opts* opts) {
    if (dtype != ID_F64 && dtype != ID_F32) return 0;
    if (zsolve_of(opts) != 0) return 0;
    TwoSided L;
    return two_sided_layout(dtype, m, n, k, opts, &L) ? L.total : 0;
}

int id_decompose_two_sided(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                           const id_opts* opts, int32_t* I, int32_t* J, void* X, int64_t ldx, void* Z, int64_t ldz,
                           void* work, size_t work_bytes, id_info* info, void* stream) {
    if (!A || !I || !J || !X || !Z || !work) return ID_EINVAL;
    const size_t need = id_two_sided_workspace_size(dtype, m, n, k, opts);
    if (need == 0) return ID_EINVAL;
    if (lda < n || ldx < m || ldz < n || !aligned(work, 256)) return ID_EINVAL;
    if (opts && opts->nb < 0) return ID_EINVAL;
    if (!engine_ok(dtype, m, n, k, opts)) return ID_EINVAL;
    if (work_bytes < need) return ID_ENOMEM;
    TwoSided L;
    two_sided_layout(dtype, m, n, k, opts, &L);
    char* base = static_cast<char*>(work);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool f64 = dtype == ID_F64;
    const bool cols_first = m <= n;
    // stage 1: the column ID (J, Z) of A, or for m > n its row ID (I, X)
    int rc = id_decompose(A, dtype, m, n, lda, k, opts, cols_first ? J : I, cols_first ? Z : X, cols_first ? ldz : ldx,
                          base + L.ws1, L.S, nullptr, stream);
    if (rc != ID_OK) return rc;
    // the skeleton: C = A[:, J] (m x k) or R = A[I, :] (k x n)
    int* flag = reinterpret_cast<int*>(base + L.flag);
    if (cudaMemsetAsync(flag, 0, 16, s) != cudaSuccess) return ID_ECUDA;
    if ((f64 ? gather_skeleton<double>(A, lda, m, n, (int)k, cols_first ? J : I, cols_first ? 0 : 1, base + L.S, flag, s)
             : gather_skeleton<float>(A, lda, m, n, (int)k, cols_first ? J : I, cols_first ? 0 : 1, base + L.S, flag,
                                      s)) != cudaSuccess)
        return ID_ECUDA;
    // stage 2: the row ID (I, X) of C, or the column ID (J, Z) of R
    int32_t* idx2 = cols_first ? I : J;
    void* Z2 = cols_first ? X : Z;
    const int64_t ld2 = cols_first ? ldx : ldz;
    if (L.second) {
        rc = id_decompose(base + L.S, dtype, L.sm, L.sn, L.sn, k, nullptr, idx2, Z2, ld2, base + L.ws2,
                          L.total - L.ws2, nullptr, stream);
        if (rc != ID_OK) return rc;
    } else {
        DevInfo* d2 = reinterpret_cast<DevInfo*>(base + L.ws2);
        if ((f64 ? identity_id<double>(idx2, Z2, ld2, (int)k, d2, s) : identity_id<float>(idx2, Z2, ld2, (int)k, d2, s)) !=
            cudaSuccess)
            return ID_ECUDA;
    }
    if (!info) return ID_OK;
    const int s1 = read_info(base + L.ws1, &info[0], s);
    const int s2 = read_info(base + L.ws2, &info[1], s);
    return s1 != ID_OK ? s1 : s2;
}

int id_trace_enable(int capacity) { return trace_enable(capacity) == 0 ? ID_OK : ID_ECUDA; }

int id_trace_read(double* ms, int64_t* launches, int nkinds) {
    if (!ms || !launches || nkinds < 1) return ID_EINVAL;
    return trace_read(ms, launches, nkinds);
}

const char* id_version(void) { return "gbid 0.1 (sm_103a)"; }

}  // extern "C"
