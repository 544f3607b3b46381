// gf_runtime.h -- host-side structures shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gf.h"

namespace gf {

// Bytes at the start of every device workspace/plan buffer reserved for
// self-resetting work counters (zeroed at allocation; each persistent kernel
// returns its counters to zero when its last CTA finishes).
constexpr size_t kCounterBytes = 8192;  // 512 counters (a blocked decode runs two batches per step)

struct Workspace {
    int device = 0;
    void *dev = nullptr;
    size_t dev_size = 0;
    void *host = nullptr;
    size_t host_size = 0;
    cudaEvent_t staged = nullptr;
    int reserve_device(size_t bytes, cudaStream_t stream);
    int reserve_host(size_t bytes);
    int upload(size_t bytes, cudaStream_t stream);  // host[0, bytes) -> dev[kCounterBytes, ...)
};

Workspace *workspace_for(cudaStream_t stream);

// Work counters of one persistent launch.
struct WorkCounter {
    unsigned long long next;  // next tile to hand out
    unsigned long long done;  // CTAs finished
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Per-device status word in device memory (zero = OK); kernels with bounded
// waits write GF_ETIMEOUT into it.  Allocated on first use.
int *device_status_word();

}  // namespace gf
