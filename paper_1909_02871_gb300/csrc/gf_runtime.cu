// gf_runtime.cu -- host runtime of the library: status strings, device
// properties, the device-side status word, and per-stream workspaces.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "gf_internal.cuh"
#include "gf_encode.h"
#include "gf_runtime.h"

namespace gf {


int current_device()
{
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int sm_count()
{
    static std::mutex mu;
    static std::map<int, int> cache;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
    return n;
}

int *device_status_word()
{
    static std::mutex mu;
    static std::map<int, int *> words;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(mu);
    auto it = words.find(dev);
    if (it != words.end()) return it->second;
    int *p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemset(p, 0, sizeof(int));
    words[dev] = p;
    return p;
}

int cuda_status(cudaError_t e)
{
    return e == cudaSuccess ? GF_OK : GF_ECUDA;
}

// ---------------------------------------------------------------------------
// per-(device, stream) workspace
// ---------------------------------------------------------------------------

static std::mutex g_ws_mu;
static std::map<std::pair<int, uintptr_t>, Workspace *> g_ws;

Workspace *workspace_for(cudaStream_t stream)
{
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_ws_mu);
    auto key = std::make_pair(dev, (uintptr_t)stream);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second;
    Workspace *ws = new Workspace();
    ws->device = dev;
    g_ws[key] = ws;
    return ws;
}

// Device buffer of at least `bytes`, stream-ordered: a larger buffer replaces
// the old one after the work already queued on `stream`.  The first
// kCounterBytes are zeroed when a buffer is (re)allocated.
int Workspace::reserve_device(size_t bytes, cudaStream_t stream)
{
    if (bytes <= dev_size && dev) return GF_OK;
    size_t want = bytes < (1u << 20) ? (1u << 20) : bytes + bytes / 4;
    if (dev) {
        cudaFreeAsync(dev, stream);
        dev = nullptr;
        dev_size = 0;
    }
    void *p = nullptr;
    if (cudaMallocAsync(&p, want, stream) != cudaSuccess) {
        cudaGetLastError();
        return GF_ENOMEM;
    }
    if (cudaMemsetAsync(p, 0, kCounterBytes, stream) != cudaSuccess) return GF_ECUDA;
    dev = p;
    dev_size = want;
    return GF_OK;
}

// Pinned host staging buffer of at least `bytes`; waits until the previous
// upload from it has been consumed by the device.
int Workspace::reserve_host(size_t bytes)
{
    if (staged) {
        if (cudaEventSynchronize(staged) != cudaSuccess) return GF_ECUDA;
    }
    if (bytes <= host_size && host) return GF_OK;
    if (host) cudaFreeHost(host);
    host = nullptr;
    host_size = 0;
    size_t want = bytes < (1u << 16) ? (1u << 16) : bytes + bytes / 4;
    if (cudaHostAlloc(&host, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        host = nullptr;
        return GF_ENOMEM;
    }
    host_size = want;
    return GF_OK;
}

int Workspace::upload(size_t bytes, cudaStream_t stream)
{
    if (cudaMemcpyAsync((char *)dev + kCounterBytes, host, bytes, cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
        return GF_ECUDA;
    if (!staged && cudaEventCreateWithFlags(&staged, cudaEventDisableTiming) != cudaSuccess) return GF_ECUDA;
    return cuda_status(cudaEventRecord(staged, stream));
}

}  // namespace gf

using namespace gf;

extern "C" const char *gf_strerror(int status)
{
    switch (status) {
    case GF_OK: return "GF_OK";
    case GF_EINVAL: return "GF_EINVAL: invalid argument";
    case GF_EOVERLAP: return "GF_EOVERLAP: regions overlap";
    case GF_ENOMEM: return "GF_ENOMEM: allocation failed";
    case GF_ERANK: return "GF_ERANK: rank deficient";
    case GF_ETIMEOUT: return "GF_ETIMEOUT: device wait gave up";
    case GF_ECUDA: return "GF_ECUDA: CUDA error";
    case GF_ENOTSUP: return "GF_ENOTSUP: not supported on this device or field";
    case GF_EBUSY: return "GF_EBUSY: result not ready yet";
    default: return "unknown status";
    }
}

extern "C" int gf_version(void) { return 10000; }

extern "C" int gf_device_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return GF_ECUDA;
    int *w = device_status_word();
    if (!w) return GF_ENOMEM;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GF_ECUDA;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    return v;
}

extern "C" int gf_selftest_wait(int abort_first, gf_stream_t stream)
{
    return gf::launch_wait_selftest(abort_first, reinterpret_cast<cudaStream_t>(stream));
}
