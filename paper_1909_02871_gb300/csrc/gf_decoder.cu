// gf_decoder.cu -- resident decoders: one generation's received packets kept
// in library-owned device memory while they arrive, decoded in batches.
//
// The paper describes the encoder only.  A receiver of random linear network
// coding collects coded packets until their coding vectors reach rank N and
// then solves for the sources; a server doing this for many generations at
// once keeps each partially received generation on the device and decodes
// every generation that got new packets in one launch.  The decode of a poll
// is gf_decode_batched (progressive Gauss-Jordan in arrival order over the
// packets received so far); the rank it reaches is written into a mapped
// host word, read once the attempt's event has completed.
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "gf_decode.h"
#include "gf_runtime.h"

namespace {

struct PollEvent {
    cudaEvent_t ev = nullptr;
    ~PollEvent()
    {
        if (ev) cudaEventDestroy(ev);
    }
};

// Per device: a library-private stream-ordered memory pool that keeps freed
// memory (decoders come and go at request rate; cudaMalloc / cudaFree would
// synchronise the device every time) and a private stream that allocations
// and frees are ordered on.
struct DevicePool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
};

// Rank words: mapped pinned host memory handed out in slots of 64 bytes from
// 16 KB pages (one cudaHostAlloc per 256 decoders, not per decoder).
constexpr size_t kRankSlot = 64, kRankPage = 16384;

std::mutex g_mu;
std::map<int, DevicePool> g_pools;
std::vector<std::pair<char *, char *>> g_rank_free;  // free slots (host, device address)

int device_pool(DevicePool &out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
        DevicePool p;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&p.pool, &props) != cudaSuccess) return GF_ECUDA;
        uint64_t keep = ~0ull;  // never hand freed memory back to the driver on its own
        cudaMemPoolSetAttribute(p.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking) != cudaSuccess) return GF_ECUDA;
        it = g_pools.emplace(dev, p).first;
    }
    out = it->second;
    return GF_OK;
}

int rank_slot(int32_t **host, int32_t **devp)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_rank_free.empty()) {
        char *page = nullptr, *dpage = nullptr;
        if (cudaHostAlloc(reinterpret_cast<void **>(&page), kRankPage, cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess)
            return GF_ENOMEM;
        if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&dpage), page, 0) != cudaSuccess) {
            cudaFreeHost(page);
            return GF_ECUDA;
        }
        for (size_t o = 0; o < kRankPage; o += kRankSlot) g_rank_free.emplace_back(page + o, dpage + o);
    }
    const auto slot = g_rank_free.back();
    g_rank_free.pop_back();
    *host = reinterpret_cast<int32_t *>(slot.first);
    *devp = reinterpret_cast<int32_t *>(slot.second);
    return GF_OK;
}

void release_rank_slot(int32_t *host, int32_t *devp)
{
    std::lock_guard<std::mutex> lock(g_mu);
    g_rank_free.emplace_back(reinterpret_cast<char *>(host), reinterpret_cast<char *>(devp));
}

}  // namespace

struct gf_decoder {
    int field = 0, n_src = 0, max_recv = 0;
    uint64_t len = 0;
    uint8_t *buf = nullptr;  // one allocation: coding vectors | payloads | decoded packets
    uint8_t *coef = nullptr, *payload = nullptr, *out = nullptr;
    int32_t *rank_host = nullptr;  // mapped pinned word written by the decode
    int32_t *rank_dev = nullptr;   // its device address
    int received = 0, tried = 0, last_rank = -1;
    int unit_rows = 0;  // pushed coding vectors that are unit vectors (sources sent uncoded)
    std::shared_ptr<PollEvent> pending;  // the latest attempt, until its result is read
    DevicePool pool;
    // the last use of the buffers on every stream that touched them (push,
    // poll, read): the stream-ordered free waits for all of them
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
};

namespace {

// Unit coding vectors among n rows of n_src coefficients in host memory (a
// systematic sender's uncoded sources); 0 for rows in device memory, which
// the host does not read.
int count_unit_rows(const uint8_t *coef, int n, int n_src)
{
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, coef) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (attr.type != cudaMemoryTypeHost && attr.type != cudaMemoryTypeUnregistered) return 0;
    int units = 0;
    for (int r = 0; r < n; ++r) {
        const uint8_t *row = coef + (size_t)r * n_src;
        int nz = 0, one = 0;
        for (int i = 0; i < n_src && nz < 2; ++i)
            if (row[i]) {
                ++nz;
                one = row[i] == 1;
            }
        units += (nz == 1 && one) ? 1 : 0;
    }
    return units;
}

int note_use(gf_decoder *d, cudaStream_t s)
{
    for (auto &u : d->uses)
        if (u.first == s) return cudaEventRecord(u.second, s) == cudaSuccess ? GF_OK : GF_ECUDA;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return GF_ECUDA;
    d->uses.emplace_back(s, ev);
    return cudaEventRecord(ev, s) == cudaSuccess ? GF_OK : GF_ECUDA;
}

}  // namespace

using gf::align_up;

extern "C" int gf_dec_open(int field, int n_src, int max_recv, uint64_t len, gf_decoder_t **dec)
{
    if (!dec) return GF_EINVAL;
    *dec = nullptr;
    if (!(field == 1 || field == 2 || field == 4 || field == 8) || n_src < 1 || n_src > gf::kMaxDecodeN ||
        max_recv < 1 || max_recv > gf::kMaxDecodeR)
        return GF_EINVAL;
    gf_decoder *d = new (std::nothrow) gf_decoder;
    if (!d) return GF_ENOMEM;
    d->field = field;
    d->n_src = n_src;
    d->max_recv = max_recv;
    d->len = len;
    const size_t c_bytes = align_up((size_t)max_recv * (size_t)n_src, 256);
    const size_t p_bytes = align_up((size_t)max_recv * (size_t)len, 256);
    const size_t o_bytes = align_up((size_t)n_src * (size_t)len, 256);
    int st = device_pool(d->pool);
    if (st != GF_OK) {
        delete d;
        return st;
    }
    // stream-ordered allocation on the pool's stream, complete before return
    if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&d->buf), c_bytes + p_bytes + o_bytes + 256, d->pool.pool,
                                d->pool.stream) != cudaSuccess ||
        cudaStreamSynchronize(d->pool.stream) != cudaSuccess) {
        delete d;
        return GF_ENOMEM;
    }
    d->coef = d->buf;
    d->payload = d->buf + c_bytes;
    d->out = d->buf + c_bytes + p_bytes;
    st = rank_slot(&d->rank_host, &d->rank_dev);
    if (st != GF_OK) {
        cudaFreeAsync(d->buf, d->pool.stream);
        delete d;
        return st;
    }
    *d->rank_host = -1;
    *dec = d;
    return GF_OK;
}

extern "C" int gf_dec_push(gf_decoder_t *d, const uint8_t *coef, const uint8_t *payload, int n, gf_stream_t stream)
{
    if (!d || n < 0) return GF_EINVAL;
    if (n == 0) return GF_OK;
    if (!coef || (d->len > 0 && !payload) || n > d->max_recv - d->received) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    d->unit_rows += count_unit_rows(coef, n, d->n_src);
    if (cudaMemcpyAsync(d->coef + (size_t)d->received * d->n_src, coef, (size_t)n * d->n_src, cudaMemcpyDefault,
                        s) != cudaSuccess)
        return GF_ECUDA;
    if (d->len > 0 && cudaMemcpyAsync(d->payload + (size_t)d->received * d->len, payload, (size_t)n * d->len,
                                      cudaMemcpyDefault, s) != cudaSuccess)
        return GF_ECUDA;
    d->received += n;
    return note_use(d, s);
}

extern "C" int gf_dec_poll(gf_decoder_t *const *decs, int n, gf_stream_t stream, int *n_launched)
{
    if (n_launched) *n_launched = 0;
    if (n < 0 || (n > 0 && !decs)) return GF_EINVAL;
    std::vector<gf_dec_t> gens;
    std::vector<gf_decoder *> tried;
    gens.reserve(n);
    for (int i = 0; i < n; ++i) {
        gf_decoder *d = decs[i];
        if (!d) return GF_EINVAL;
        if (d->received < d->n_src || d->received <= d->tried) continue;
        gf_dec_t g{};
        g.field = d->field;
        g.n_src = d->n_src;
        g.n_recv = d->received;
        g.len = d->len;
        g.coef = d->coef;
        g.payload = d->payload;
        g.out = d->out;
        g.rank = d->rank_dev;
        // at least half of the packets are sources sent uncoded: the payload phase skips the
        // zero multipliers of their unit transform rows
        if (2 * d->unit_rows >= d->received) g.flags = GF_DEC_SYSTEMATIC;
        gens.push_back(g);
        tried.push_back(d);
    }
    if (gens.empty()) return GF_OK;
    int st = gf_decode_batched(gens.data(), (int)gens.size(), stream);
    if (st != GF_OK) return st;
    auto ev = std::make_shared<PollEvent>();
    if (cudaEventCreateWithFlags(&ev->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev->ev, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return GF_ECUDA;
    for (gf_decoder *d : tried) {
        d->tried = d->received;
        d->pending = ev;
        if (note_use(d, reinterpret_cast<cudaStream_t>(stream)) != GF_OK) return GF_ECUDA;
    }
    if (n_launched) *n_launched = (int)tried.size();
    return GF_OK;
}

extern "C" int gf_dec_status(gf_decoder_t *d, int wait, int *rank, int *received, const uint8_t **out)
{
    if (!d) return GF_EINVAL;
    if (d->pending) {
        if (wait) {
            if (cudaEventSynchronize(d->pending->ev) != cudaSuccess) return GF_ECUDA;
        } else {
            const cudaError_t q = cudaEventQuery(d->pending->ev);
            if (q == cudaErrorNotReady) return GF_EBUSY;
            if (q != cudaSuccess) return GF_ECUDA;
        }
        d->last_rank = *reinterpret_cast<volatile int32_t *>(d->rank_host);
        d->pending.reset();
    }
    if (rank) *rank = d->last_rank;
    if (received) *received = d->received;
    if (out) *out = d->out;
    return GF_OK;
}

extern "C" int gf_dec_read(gf_decoder_t *d, uint8_t *dst, gf_stream_t stream)
{
    if (!d) return GF_EINVAL;
    const size_t bytes = (size_t)d->n_src * (size_t)d->len;
    if (bytes == 0) return GF_OK;
    if (!dst) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(dst, d->out, bytes, cudaMemcpyDefault, s) != cudaSuccess) return GF_ECUDA;
    return note_use(d, s);
}

extern "C" int gf_dec_close(gf_decoder_t *d)
{
    if (!d) return GF_OK;
    int st = GF_OK;
    // the rank slot goes back to the free list only once the attempt that
    // writes it is done; the buffers are freed in stream order after every
    // stream that used them
    if (d->pending && cudaEventSynchronize(d->pending->ev) != cudaSuccess) st = GF_ECUDA;
    d->pending.reset();
    for (auto &u : d->uses) {
        if (cudaStreamWaitEvent(d->pool.stream, u.second, 0) != cudaSuccess) st = GF_ECUDA;
        cudaEventDestroy(u.second);
    }
    if (cudaFreeAsync(d->buf, d->pool.stream) != cudaSuccess) st = GF_ECUDA;
    release_rank_slot(d->rank_host, d->rank_dev);
    delete d;
    return st;
}
