// Kernel-class timing: CUDA event pairs around the launches of the per-step
// kernels, recorded on the caller's stream while tracing is enabled.
#include <cuda_runtime.h>

#include <vector>

#include "trace.cuh"

namespace gbid {
namespace {

struct Trace {
    bool enabled = false;
    int capacity = 0;
    int used = 0;
    std::vector<cudaEvent_t> ev;     // 2 per record
    std::vector<int> kind;
};

Trace g_trace;

}  // namespace

bool trace_on() { return g_trace.enabled && g_trace.used < g_trace.capacity; }

int trace_begin(TraceKind k, cudaStream_t s) {
    if (!trace_on()) return -1;
    const int i = g_trace.used++;
    g_trace.kind[i] = (int)k;
    cudaEventRecord(g_trace.ev[2 * i], s);
    return i;
}

void trace_end(int i, cudaStream_t s) {
    if (i >= 0) cudaEventRecord(g_trace.ev[2 * i + 1], s);
}

int trace_enable(int capacity) {
    for (cudaEvent_t e : g_trace.ev) cudaEventDestroy(e);
    g_trace = Trace();
    if (capacity <= 0) return 0;
    g_trace.ev.resize(2 * (size_t)capacity);
    g_trace.kind.resize(capacity);
    for (auto& e : g_trace.ev)
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
    g_trace.capacity = capacity;
    g_trace.enabled = true;
    return 0;
}

int trace_read(double* ms, int64_t* count, int nkinds) {
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        count[k] = 0;
    }
    for (int i = 0; i < g_trace.used; ++i) {
        if (cudaEventSynchronize(g_trace.ev[2 * i + 1]) != cudaSuccess) return -1;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_trace.ev[2 * i], g_trace.ev[2 * i + 1]) != cudaSuccess) return -1;
        const int k = g_trace.kind[i];
        if (k >= 0 && k < nkinds) {
            ms[k] += t;
            count[k] += 1;
        }
    }
    const int n = g_trace.used;
    g_trace.used = 0;
    return n;
}

}  // namespace gbid
