// Internal tracing hooks (see id_trace_enable in gbid.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbid {

enum class TraceKind : int { kCpqr = 0, kSolve = 1, kSketch = 2, kCopyIn = 3, kScatter = 4, kBatched = 5, kRefine = 6, kSampledZ = 7, kCount = 8 };

bool trace_on();
int trace_begin(TraceKind k, cudaStream_t s);   // returns a record id, -1 when not tracing
void trace_end(int id, cudaStream_t s);
int trace_enable(int capacity);
int trace_read(double* ms, int64_t* count, int nkinds);

}  // namespace gbid
