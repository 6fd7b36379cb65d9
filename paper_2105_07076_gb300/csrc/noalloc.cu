// id_decompose_noalloc: the decomposition with its scratch in a fixed device
// array that the library carries, for callers that cannot allocate.
//
// Some callers may not call cudaMalloc (or any allocating routine): code that
// runs while another thread holds a global-mode stream capture (allocation is
// illegal then), plug-ins hosted by a framework that owns every byte of device
// memory through its own pool, and real-time loops that must not take the
// allocator's locks. They pass A, J and Z; the scratch comes from g_scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "gbid.h"

namespace {

// Fixed scratch: every GPU that loads this library keeps it until the process exits.
__device__ __align__(256) unsigned char g_scratch[ID_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mtx;

// Device address of g_scratch on the current device. In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ID_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mtx);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return ID_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ID_OK;
}

}  // namespace

extern "C" int id_decompose_noalloc(const void* A, id_dtype dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                                    const id_opts* opts, int32_t* J, void* Z, int64_t ldz, id_info* info,
                                    void* stream) {
    const size_t need = id_workspace_size(dtype, m, n, k, opts);
    if (need == 0) return ID_EINVAL;
    if (need > (size_t)ID_NOALLOC_SCRATCH_BYTES) return ID_ENOMEM;   // problem too large for the fixed scratch
    void* ws = nullptr;
    const int rc = scratch_for_current_device(&ws);
    if (rc != ID_OK) return rc;
    return id_decompose(A, dtype, m, n, lda, k, opts, J, Z, ldz, ws, (size_t)ID_NOALLOC_SCRATCH_BYTES, info, stream);
}
