// mp_common.cuh -- host-side helpers shared by the libmpgpu translation units:
// status handling, launch sizing from the device's SM count, argument checks.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpgpu.h"

namespace mp {

// CUDA error of the last failed call, per host thread (read by mp_last_cuda_error).
int &last_cuda_error();

inline mp_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MP_OK;
    last_cuda_error() = (int)e;
    return MP_ECUDA;
}

inline mp_status launch_status() { return cuda_status(cudaGetLastError()); }

// Streaming multiprocessors of the current device (cached per device).
int sm_count();

inline cudaStream_t as_stream(mp_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Grid size for a grid-stride loop over n items: enough blocks to fill every SM
// `per_sm` times, never more than the work needs.
inline unsigned grid_for(int64_t n, int threads, int per_sm)
{
    int64_t need = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    int64_t g = need < cap ? need : cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// Plane-layout argument check: K planes of n elements with plane stride ps.
inline bool planes_ok(const void *p, int64_t n, int64_t ps)
{
    if (n == 0) return true;
    return p != nullptr && ps >= n;
}

}  // namespace mp
