// Entry points of the W > 64 kernels beyond the anchored alignment.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "genasm_internal.h"

namespace ga {

// The free-start first window for 64 < W <= 128: the locate step with 128-bit
// vectors (writes each pair's start to ref_start), then the wide alignment
// from those starts. Workspace: wide_workspace_bytes(p.n_pairs).
cudaError_t launch_wide_locate(const AlignParams& p, const uint32_t* start_span, int32_t* ref_start,
                               void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace ga
