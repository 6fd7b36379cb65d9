// id_rid_pipe: randomized IDs (Sec. 2.2) of a stream of host matrices, with the
// copies of neighbouring IDs overlapping the compute of the current one.
//
// ID i takes slot b = i mod 2:
//   H2D stream:     [wait: ID i-2's compute is done with slot b] A, Omega -> slot b; record in[b]
//   caller stream:  [wait in[b]; wait: ID i-2's outputs have left slot b]
//                   id_decompose_randomized on slot b; its status -> slot b; record done[b]
//   D2H stream:     [wait done[b]] J, Z, status -> the caller's host buffers; record out[b]
// So while ID i runs, ID i+1's inputs arrive and ID i-1's outputs leave. The IDs
// share one randomized workspace, used in order on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "gbid.h"

struct id_rid_pipe {
    int64_t m, n, l, k;
    id_opts opts;
    bool has_opts;
    int dev;
    int64_t lda_d, ldo_d;   // device slot leading dimensions (A: 16-byte rows; Omega: 8 BF16 multiple)
    cudaStream_t h2d, d2h;
    cudaEvent_t in[2], done[2], out[2];
    float* A[2];
    uint16_t* Om[2];
    int32_t* J[2];
    float* Z[2];
    id_info* info[2];
    void* ws;
    size_t ws_bytes;
    int64_t count;     // IDs submitted so far
    void* stream;      // the caller's stream of the first submit
};

namespace {

constexpr size_t kPipeAlign = 256;
size_t up(size_t x) { return (x + kPipeAlign - 1) / kPipeAlign * kPipeAlign; }

struct PipeLayout {
    size_t A, Om, J, Z, info, slot, ws, total;
};

// Byte offsets within `work`: two slots, then the randomized workspace.
bool pipe_layout(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts, PipeLayout* L) {
    const size_t ws = id_rid_workspace_size(m, n, l, k, opts);
    if (ws == 0) return false;
    const int64_t lda = (n + 3) / 4 * 4, ldo = (m + 7) / 8 * 8;
    L->A = 0;
    L->Om = up(4 * (size_t)m * lda);
    L->J = L->Om + up(2 * (size_t)l * ldo);
    L->Z = L->J + up(4 * (size_t)k);
    L->info = L->Z + up(4 * (size_t)k * n);
    L->slot = L->info + up(sizeof(id_info));
    L->ws = 2 * L->slot;
    L->total = L->ws + ws;
    return true;
}

}  // namespace

size_t id_rid_pipe_workspace_size(int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts) {
    PipeLayout L;
    return pipe_layout(m, n, l, k, opts, &L) ? L.total : 0;
}

void id_rid_pipe_destroy(id_rid_pipe* p) {
    if (!p) return;
    int cur = 0;
    const bool swap = cudaGetDevice(&cur) == cudaSuccess && cur != p->dev && cudaSetDevice(p->dev) == cudaSuccess;
    if (p->h2d) cudaStreamSynchronize(p->h2d);
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    for (int b = 0; b < 2; ++b) {
        if (p->in[b]) cudaEventDestroy(p->in[b]);
        if (p->done[b]) cudaEventDestroy(p->done[b]);
        if (p->out[b]) cudaEventDestroy(p->out[b]);
    }
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    if (swap) cudaSetDevice(cur);
    delete p;
}

int id_rid_pipe_create(id_rid_pipe** out, int64_t m, int64_t n, int64_t l, int64_t k, const id_opts* opts,
                       void* work, size_t work_bytes) {
    if (!out || !work) return ID_EINVAL;
    *out = nullptr;
    if (reinterpret_cast<uintptr_t>(work) % kPipeAlign != 0) return ID_EINVAL;
    PipeLayout L;
    if (!pipe_layout(m, n, l, k, opts, &L)) return ID_EINVAL;
    if (work_bytes < L.total) return ID_ENOMEM;
    id_rid_pipe* p = new (std::nothrow) id_rid_pipe();
    if (!p) return ID_ENOMEM;
    p->m = m;
    p->n = n;
    p->l = l;
    p->k = k;
    p->has_opts = opts != nullptr;
    if (opts) p->opts = *opts;
    p->lda_d = (n + 3) / 4 * 4;
    p->ldo_d = (m + 7) / 8 * 8;
    char* base = static_cast<char*>(work);
    for (int b = 0; b < 2; ++b) {
        char* s = base + b * L.slot;
        p->A[b] = reinterpret_cast<float*>(s + L.A);
        p->Om[b] = reinterpret_cast<uint16_t*>(s + L.Om);
        p->J[b] = reinterpret_cast<int32_t*>(s + L.J);
        p->Z[b] = reinterpret_cast<float*>(s + L.Z);
        p->info[b] = reinterpret_cast<id_info*>(s + L.info);
    }
    p->ws = base + L.ws;
    p->ws_bytes = work_bytes - L.ws;
    bool ok = cudaGetDevice(&p->dev) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&p->in[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->done[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->out[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        id_rid_pipe_destroy(p);
        return ID_ECUDA;
    }
    *out = p;
    return ID_OK;
}

int id_rid_pipe_submit(id_rid_pipe* p, const float* A_host, int64_t lda, const uint16_t* Omega_host, int64_t ldo,
                       int32_t* J_host, float* Z_host, int64_t ldz, id_info* info_host, void* stream) {
    if (!p || !A_host || !Omega_host || !J_host || !Z_host) return ID_EINVAL;
    if (lda < p->n || ldo < p->m || ldz < p->n) return ID_EINVAL;
    if (p->count > 0 && stream != p->stream) return ID_EINVAL;   // one compute stream per pipe
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != p->dev) return ID_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int b = (int)(p->count & 1);
    const bool reuse = p->count >= 2;   // slot b held ID count - 2
    // inputs -> slot b, once ID count - 2 has finished computing on it
    if (reuse && cudaStreamWaitEvent(p->h2d, p->done[b], 0) != cudaSuccess) return ID_ECUDA;
    if (cudaMemcpy2DAsync(p->A[b], 4 * p->lda_d, A_host, 4 * lda, 4 * p->n, p->m, cudaMemcpyHostToDevice, p->h2d) !=
            cudaSuccess ||
        cudaMemcpy2DAsync(p->Om[b], 2 * p->ldo_d, Omega_host, 2 * ldo, 2 * p->m, p->l, cudaMemcpyHostToDevice,
                          p->h2d) != cudaSuccess ||
        cudaEventRecord(p->in[b], p->h2d) != cudaSuccess)
        return ID_ECUDA;
    // the ID on the caller's stream, after its inputs and after slot b's previous outputs left
    if (cudaStreamWaitEvent(s, p->in[b], 0) != cudaSuccess) return ID_ECUDA;
    if (reuse && cudaStreamWaitEvent(s, p->out[b], 0) != cudaSuccess) return ID_ECUDA;
    const int rc = id_decompose_randomized(p->A[b], ID_F32, p->m, p->n, p->lda_d, p->Om[b], p->l, p->ldo_d, p->k,
                                           p->has_opts ? &p->opts : nullptr, p->J[b], p->Z[b], p->n, p->ws,
                                           p->ws_bytes, nullptr, stream);
    if (rc != ID_OK) return rc;
    // its status sits at the start of the workspace until the next ID resets it
    if (cudaMemcpyAsync(p->info[b], p->ws, sizeof(id_info), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaEventRecord(p->done[b], s) != cudaSuccess)
        return ID_ECUDA;
    // outputs -> the caller's host buffers
    if (cudaStreamWaitEvent(p->d2h, p->done[b], 0) != cudaSuccess ||
        cudaMemcpyAsync(J_host, p->J[b], 4 * (size_t)p->k, cudaMemcpyDeviceToHost, p->d2h) != cudaSuccess ||
        cudaMemcpy2DAsync(Z_host, 4 * ldz, p->Z[b], 4 * p->n, 4 * p->n, p->k, cudaMemcpyDeviceToHost, p->d2h) !=
            cudaSuccess)
        return ID_ECUDA;
    if (info_host &&
        cudaMemcpyAsync(info_host, p->info[b], sizeof(id_info), cudaMemcpyDeviceToHost, p->d2h) != cudaSuccess)
        return ID_ECUDA;
    if (cudaEventRecord(p->out[b], p->d2h) != cudaSuccess) return ID_ECUDA;
    if (p->count == 0) p->stream = stream;
    ++p->count;
    return ID_OK;
}

int id_rid_pipe_sync(id_rid_pipe* p) {
    if (!p) return ID_EINVAL;
    // every ID's copy-out waits for its compute, which waits for its copy-in; the copy-in stream
    // too, for a submit that failed after its inputs were enqueued
    return cudaStreamSynchronize(p->h2d) == cudaSuccess && cudaStreamSynchronize(p->d2h) == cudaSuccess ? ID_OK
                                                                                                        : ID_ECUDA;
}
