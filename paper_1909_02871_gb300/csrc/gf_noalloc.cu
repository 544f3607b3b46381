// gf_noalloc.cu -- single-generation decode that allocates nothing.
//
// gf_decode_batched keeps its per-call scratch (the elimination transform X,
// the device copies of the descriptors and the work counter) in a workspace
// that the library grows with the CUDA allocator.  Some callers cannot let a
// decode call allocate: a packet-processing data path that decodes
// generations as they complete and must not stall on the allocator (whose
// first call on a device can synchronise it), or a process that has handed
// all device memory to its own pool at start-up.  gf_decode_noalloc serves
// them with the same two kernels (coefficient Gauss-Jordan, then the
// table-path encode as the payload phase) and a fixed scratch area that is a
// file-scope __device__ array of kNoAllocBytes, resident on every device that
// loads the library until the process exits.
//
// The array's host-side name is only a stand-in: its device address is
// looked up once per device with cudaGetSymbolAddress, on the first call
// made with that device current.  That first call should therefore come
// before any stream capture.  Each call hands its descriptors to a one-thread
// set-up kernel as kernel arguments (passed by value, so nothing on the host
// is read after the call returns); that kernel writes them into the array
// and clears the work counter that must start at zero.  All calls share the
// array and it keeps the last call's contents.  Calls whose work overlaps on
// the GPU (other streams, other threads) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "gf_decode.h"
#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

int launch_decode_coef_raw(const DecGen *d_gens, int n_gens, size_t smem, cudaStream_t stream);
long long table_tiles_for(EncGen &g);
int launch_table_raw(const EncGen *d_gens, const long long *d_tile_start, int n_gens, long long total,
                     WorkCounter *ctr, cudaStream_t stream);

constexpr size_t kNoAllocBytes = 256 * 1024;   // GF_NOALLOC_SCRATCH_BYTES
constexpr size_t kNoAllocCounter = 0;          // WorkCounter of the payload phase
constexpr size_t kNoAllocDecGen = 256;         // DecGen of the coefficient phase
constexpr size_t kNoAllocEncGen = 512;         // EncGen of the payload phase
constexpr size_t kNoAllocTiles = 768;          // its two tile offsets
constexpr size_t kNoAllocX = 1024;             // X: n_src x n_recv bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static_assert(sizeof(WorkCounter) <= kNoAllocDecGen - kNoAllocCounter, "WorkCounter slot");
static_assert(sizeof(DecGen) <= kNoAllocEncGen - kNoAllocDecGen, "DecGen slot");
static_assert(sizeof(EncGen) <= kNoAllocTiles - kNoAllocEncGen, "EncGen slot");
static_assert(2 * sizeof(long long) <= kNoAllocX - kNoAllocTiles, "tile offsets slot");

// The descriptors of one call, passed by value to the set-up kernel.
struct NoAllocDescs {
    DecGen dec;
    EncGen enc;
    long long tiles[2];
};

// One thread writes the call's descriptors into the array and clears the
// payload phase's work counter.
__global__ void noalloc_setup_kernel(NoAllocDescs d)
{
    *reinterpret_cast<DecGen *>(g_noalloc_scratch + kNoAllocDecGen) = d.dec;
    *reinterpret_cast<EncGen *>(g_noalloc_scratch + kNoAllocEncGen) = d.enc;
    long long *tiles = reinterpret_cast<long long *>(g_noalloc_scratch + kNoAllocTiles);
    tiles[0] = d.tiles[0];
    tiles[1] = d.tiles[1];
    *reinterpret_cast<WorkCounter *>(g_noalloc_scratch + kNoAllocCounter) = WorkCounter{};
}

// Device address of the scratch array on the current device (looked up once;
// a fixed table, so the lookup itself allocates nothing).
static int scratch_address(unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return GF_ENOTSUP;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GF_ECUDA;
        }
        addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = addr[dev];
    return GF_OK;
}

}  // namespace gf

using namespace gf;

extern "C" int gf_decode_noalloc(int field, int n_src, int n_recv, uint64_t len, const uint8_t *coef,
                                 const uint8_t *payload, uint8_t *out, int32_t *rank, int32_t *used, uint8_t *solved,
                                 gf_stream_t stream)
{
    if (!field_ok(field) || n_src < 0 || n_src > kMaxDecodeN || n_recv < 0 || n_recv > kMaxDecodeR || !rank)
        return GF_EINVAL;
    if (n_src > 0 && len > 0 && !out) return GF_EINVAL;
    if (n_recv > 0 && n_src > 0 && !coef) return GF_EINVAL;
    if (n_recv > 0 && len > 0 && !payload) return GF_EINVAL;
    // the limits: X fits the array, the elimination rows fit one CTA's shared memory
    if ((size_t)n_src * (size_t)n_recv > kNoAllocBytes - kNoAllocX) return GF_EINVAL;
    const int W = (int)align_up((size_t)n_src + (size_t)n_recv, 16);
    const size_t smem = dec_smem_bytes(field, n_src, W, true);
    if (smem > decode_smem_limit()) return GF_EINVAL;

    unsigned char *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != GF_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    DecGen g{};
    g.coef = coef;
    g.payload = payload;
    g.out = out;
    g.rank = rank;
    g.used = used;
    g.solved = solved;
    g.X = scratch + kNoAllocX;
    g.grows = nullptr;
    g.len = len;
    g.field = field;
    g.N = n_src;
    g.R = n_recv;
    g.W = W;

    // payload phase: out = X * payload, an encode of n_src packets from the n_recv received ones
    EncGen e{};
    e.src = payload;
    e.coef = g.X;
    e.out = out;
    e.len = len;
    e.field = field;
    e.n_src = n_recv;
    e.n_coded = n_src;
    e.coef_ld = n_recv;
    e.variant = choose_table_variant(field, n_recv, n_src, len);
    const long long tiles[2] = {0, table_tiles_for(e)};

    // descriptors into the array and the counter cleared, by a kernel whose
    // arguments carry them
    NoAllocDescs d{};
    d.dec = g;
    d.enc = e;
    d.tiles[0] = tiles[0];
    d.tiles[1] = tiles[1];
    noalloc_setup_kernel<<<1, 1, 0, s>>>(d);
    st = cuda_status(cudaGetLastError());
    if (st != GF_OK) return st;
    st = launch_decode_coef_raw(reinterpret_cast<const DecGen *>(scratch + kNoAllocDecGen), 1, smem, s);
    if (st != GF_OK) return st;
    return launch_table_raw(reinterpret_cast<const EncGen *>(scratch + kNoAllocEncGen),
                            reinterpret_cast<const long long *>(scratch + kNoAllocTiles), 1, tiles[1],
                            reinterpret_cast<WorkCounter *>(scratch + kNoAllocCounter), s);
}
