// gf_encode.cu -- batched generation encode, table path (Eq. 2:
// out_k = sum_i c_ki * a_i), plus the host side of every batched launch:
// descriptor checks, tile lists, per-stream workspaces and plans.
//
// Table path.  A warp tile is (generation, 32*WPT*4 columns, KPT coded
// packets).  For each source packet a lane loads WPT words of its columns
// once, derives the prmt selectors of those words once, and then, for each
// of the KPT coefficients c_ki, applies c_ki's split tables (gf::ByteMap,
// looked up by value in shared memory) and XORs into KPT x WPT register
// accumulators: 5 integer ops per word and coefficient.  Zero coefficients
// are skipped (the trivial case of section IV).  Warps fetch tiles from a
// self-resetting global counter, so uneven generations (N, K, len, field)
// share one persistent launch.
#include <algorithm>
#include <mutex>
#include <vector>

#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

const TableVariant kTableVariants[kNumTableVariants] = {{4, 16}, {1, 16}, {2, 16}, {4, 8}};

constexpr int kEncThreads = 256;

struct alignas(16) SmemMap {
    ByteMap m;
    uint32_t pad[2];
};

// ---------------------------------------------------------------------------
// word loads/stores of a packet row, any alignment, bytes past len read as 0
// and never written
// ---------------------------------------------------------------------------
template <int WPT>
__device__ __forceinline__ void load_words(const uint8_t *row, unsigned long long col, unsigned long long len,
                                           uint32_t (&w)[WPT])
{
    const uint8_t *p = row + col;
    if (col + 4 * WPT <= len) {
        const uintptr_t a = (uintptr_t)p;
        if (WPT == 4 && (a & 15u) == 0) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
            w[0] = v.x; w[1 % WPT] = v.y; w[2 % WPT] = v.z; w[3 % WPT] = v.w;
            return;
        }
        if (WPT == 2 && (a & 7u) == 0) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
            w[0] = v.x; w[1 % WPT] = v.y;
            return;
        }
        // aligned words straddling the row: each contains at least one byte
        // of [p, p + 4*WPT), so none leaves the allocation
        const uint32_t *q = reinterpret_cast<const uint32_t *>(a & ~(uintptr_t)3);
        const uint32_t sh = (uint32_t)(a & 3u) * 8u;
        if (sh == 0) {
#pragma unroll
            for (int i = 0; i < WPT; ++i) w[i] = __ldg(q + i);
        } else {
            uint32_t prev = __ldg(q);
#pragma unroll
            for (int i = 0; i < WPT; ++i) {
                const uint32_t next = __ldg(q + i + 1);
                w[i] = __funnelshift_r(prev, next, sh);
                prev = next;
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const unsigned long long idx = col + 4 * i + b;
            if (idx < len) v |= (uint32_t)__ldg(row + idx) << (8 * b);
        }
        w[i] = v;
    }
}

template <int WPT>
__device__ __forceinline__ void store_words(uint8_t *row, unsigned long long col, unsigned long long len,
                                            const uint32_t (&w)[WPT])
{
    uint8_t *p = row + col;
    if (col + 4 * WPT <= len) {
        const uintptr_t a = (uintptr_t)p;
        if (WPT == 4 && (a & 15u) == 0) {
            *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1 % WPT], w[2 % WPT], w[3 % WPT]);
            return;
        }
        if (WPT == 2 && (a & 7u) == 0) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1 % WPT]);
            return;
        }
        if ((a & 3u) == 0) {
#pragma unroll
            for (int i = 0; i < WPT; ++i) reinterpret_cast<uint32_t *>(p)[i] = w[i];
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < WPT; ++i)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const unsigned long long idx = col + 4 * i + b;
            if (idx < len) row[idx] = (uint8_t)(w[i] >> (8 * b));
        }
}

template <int WPT, int KPT>
__device__ __forceinline__ void table_tile(const SmemMap *tab, const EncGen &g, int kc, int cc, int lane)
{
    const int N = g.n_src, K = g.n_coded, ld = g.coef_ld;
    const unsigned long long len = g.len;
    const int k0 = kc * KPT;
    const int kn = min(KPT, K - k0);
    const unsigned long long col = (unsigned long long)cc * (32 * WPT * 4) + (unsigned long long)lane * (WPT * 4);
    const SmemMap *ftab = tab + table_base(g.field);
    const uint8_t *coefk = g.coef + (size_t)k0 * ld;

    uint32_t acc[KPT][WPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int i = 0; i < WPT; ++i) acc[k][i] = 0u;

    // the tile's coefficients of source i, four per register (the same for every lane)
    auto load_coef = [&](int i, uint32_t (&c4)[KPT / 4]) {
#pragma unroll
        for (int q = 0; q < KPT / 4; ++q) c4[q] = 0u;
#pragma unroll
        for (int k = 0; k < KPT; ++k)
            if (k < kn) c4[k >> 2] |= (uint32_t)__ldg(coefk + (size_t)k * ld + i) << (8 * (k & 3));
    };
    auto nonzero = [](const uint32_t (&c4)[KPT / 4]) {
        uint32_t any = 0u;
#pragma unroll
        for (int q = 0; q < KPT / 4; ++q) any |= c4[q];
        return any != 0u;
    };
    // acc[k] ^= c_k * (the words w of one source), through the words' prmt selectors
    auto madd = [&](const uint32_t (&c4)[KPT / 4], const uint32_t (&w)[WPT]) {
        Sel s[WPT];
#pragma unroll
        for (int j = 0; j < WPT; ++j) s[j] = make_sel(w[j]);
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const uint32_t ck = (c4[k >> 2] >> (8 * (k & 3))) & 0xFFu;
            if (ck != 0u) {
                const ByteMap m = ftab[ck].m;
#pragma unroll
                for (int j = 0; j < WPT; ++j) acc[k][j] ^= apply(m, s[j]);
            }
        }
    };

    if (KPT * WPT <= 32) {
        // Tiles with registers to spare load ahead: the next source's words and the
        // coefficients of the one after are on their way while this source is applied (a
        // source's words wait for its coefficients, so that a source they all leave out --
        // sparse coding matrices, e.g. the transform of a decode whose received packets are
        // mostly sources sent uncoded -- is not loaded at all)
        uint32_t ca[KPT / 4] = {}, cb[KPT / 4] = {}, w[WPT] = {}, wn[WPT] = {};
        bool za = false;  // a generation without sources reads nothing (its outputs are zero)
        if (N > 0) {
            load_coef(0, ca);
            za = nonzero(ca);
            if (za) load_words<WPT>(g.src, col, len, w);
        }
        if (N > 1) load_coef(1, cb);
        for (int i = 0; i < N; ++i) {
            bool zb = false;
            if (i + 1 < N) {
                zb = nonzero(cb);
                if (zb) load_words<WPT>(g.src + (size_t)(i + 1) * len, col, len, wn);
            }
            uint32_t cc[KPT / 4];
            if (i + 2 < N) load_coef(i + 2, cc);
            if (za) madd(ca, w);
#pragma unroll
            for (int q = 0; q < KPT / 4; ++q) {
                ca[q] = cb[q];
                cb[q] = i + 2 < N ? cc[q] : 0u;
            }
#pragma unroll
            for (int j = 0; j < WPT; ++j) w[j] = wn[j];
            za = zb;
        }
    } else {
        for (int i = 0; i < N; ++i) {
            // the tile's coefficients of source i first: a source they all leave out is not
            // loaded at all (sparse coding matrices, as above)
            uint32_t c4[KPT / 4];
            load_coef(i, c4);
            if (!nonzero(c4)) continue;
            uint32_t w[WPT];
            load_words<WPT>(g.src + (size_t)i * len, col, len, w);
            madd(c4, w);
        }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        if (k < kn) {
            if (g.accumulate) {
                // out ^= the products (the blocked decode's row updates)
                uint32_t old[WPT];
                load_words<WPT>(g.out + (size_t)(k0 + k) * len, col, len, old);
#pragma unroll
                for (int i = 0; i < WPT; ++i) acc[k][i] ^= old[i];
            }
            store_words<WPT>(g.out + (size_t)(k0 + k) * len, col, len, acc[k]);
        }
    }
}

__device__ __forceinline__ int find_gen(const long long *tile_start, int n_gens, long long t)
{
    int lo = 0, hi = n_gens - 1;  // last gen with tile_start <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kEncThreads, 2)
encode_table_kernel(const EncGen *__restrict__ gens, const long long *__restrict__ tile_start, int n_gens,
                    long long total, WorkCounter *ctr)
{
    __shared__ SmemMap tab[kTableEntries];
    for (int e = threadIdx.x; e < kTableEntries; e += blockDim.x) tab[e].m = g_field_tables.map[e];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&ctr->next, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const int gi = find_gen(tile_start, n_gens, t);
        const EncGen g = gens[gi];
        const long long local = t - __ldg(tile_start + gi);
        const int cc = (int)(local / g.k_chunks);
        const int kc = (int)(local % g.k_chunks);
        switch (g.variant) {
        case 0: table_tile<4, 16>(tab, g, kc, cc, lane); break;
        case 1: table_tile<1, 16>(tab, g, kc, cc, lane); break;
        case 2: table_tile<2, 16>(tab, g, kc, cc, lane); break;
        default: table_tile<4, 8>(tab, g, kc, cc, lane); break;
        }
    }
    // the last CTA to finish returns the counters to zero for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&ctr->done, 1ull);
        if (prev == (unsigned long long)gridDim.x - 1ull) {
            ctr->next = 0ull;
            ctr->done = 0ull;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int convert_gen(const gf_gen_t &g, EncGen &e)
{
    if (!field_ok(g.field) || g.n_src < 0 || g.n_coded < 0 || g.reserved != 0) return GF_EINVAL;
    if (g.n_coded > 0 && g.len > 0 && !g.out) return GF_EINVAL;
    if (g.n_coded > 0 && g.n_src > 0 && !g.coef) return GF_EINVAL;
    if (g.n_coded > 0 && g.n_src > 0 && g.len > 0 && !g.src) return GF_EINVAL;
    e = EncGen{};
    e.src = g.src;
    e.coef = g.coef;
    e.out = g.out;
    e.len = g.len;
    e.field = g.field;
    e.n_src = g.n_src;
    e.n_coded = g.n_coded;
    e.coef_ld = g.n_src;
    return GF_OK;
}

static long long table_tiles(EncGen &g)
{
    const TableVariant v = kTableVariants[g.variant];
    const unsigned long long cols = 32ull * v.wpt * 4;
    if (g.n_coded == 0 || g.len == 0) {
        g.col_chunks = g.k_chunks = 0;
        return 0;
    }
    g.col_chunks = (int)((g.len + cols - 1) / cols);
    g.k_chunks = (g.n_coded + v.kpt - 1) / v.kpt;
    return (long long)g.col_chunks * g.k_chunks;
}

void finalize_batch(EncodeBatch &b)
{
    b.tile_start.assign(b.gens.size() + 1, 0);
    b.all_gf256 = true;
    if (b.kind == GF_PATH_BITSLICED) {
        // a bit-sliced work item is (generation, 64 coded packets) over all its
        // column tiles; a batch with fewer items than about two per SM splits
        // each item's column tiles into ranges so that the SMs all get work
        long long items = 0;
        for (const EncGen &g : b.gens) items += (g.n_coded + 63) / 64;
        const long long want = 2LL * sm_count();
        const long long split = items > 0 && items < want ? (want + items - 1) / items : 1;
        b.col_split = false;
        for (EncGen &g : b.gens) {
            const long long ncols = (long long)((g.len + 127) / 128);
            g.col_chunks = (int)std::max(1LL, std::min(split, ncols));
            if (g.col_chunks > 1) b.col_split = true;
        }
    }
    long long t = 0;
    for (size_t i = 0; i < b.gens.size(); ++i) {
        b.tile_start[i] = t;
        if (b.gens[i].field != 8) b.all_gf256 = false;
        long long n;
        if (b.kind == GF_PATH_BITSLICED) n = bitsliced_tiles(b.gens[i], b.gens[i].col_chunks, b.gens[i].k_chunks);
        else n = table_tiles(b.gens[i]);
        t += n;
    }
    b.tile_start[b.gens.size()] = t;
    b.total_tiles = t;
}

size_t batch_bytes(const EncodeBatch &b)
{
    return align_up(b.gens.size() * sizeof(EncGen), 256) + align_up(b.tile_start.size() * sizeof(long long), 256);
}

size_t stage_batch(EncodeBatch &b, char *host, char *dev_base, size_t off)
{
    const size_t g_bytes = b.gens.size() * sizeof(EncGen);
    memcpy(host + off, b.gens.data(), g_bytes);
    b.d_gens = reinterpret_cast<EncGen *>(dev_base + off);
    off += align_up(g_bytes, 256);
    const size_t t_bytes = b.tile_start.size() * sizeof(long long);
    memcpy(host + off, b.tile_start.data(), t_bytes);
    b.d_tile_start = reinterpret_cast<long long *>(dev_base + off);
    off += align_up(t_bytes, 256);
    return off;
}

static int table_grid()
{
    static std::mutex mu;
    static int cached_dev = -1, cached = 0;
    std::lock_guard<std::mutex> lock(mu);
    const int dev = current_device();
    if (dev != cached_dev) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, encode_table_kernel, kEncThreads, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        cached = per_sm * sm_count();
        cached_dev = dev;
    }
    return cached;
}

int launch_batch(const EncodeBatch &b, cudaStream_t stream)
{
    if (b.total_tiles == 0) return GF_OK;
    if (b.kind == GF_PATH_BITSLICED) return launch_bitsliced(b, stream);
    const long long warps = kEncThreads / 32;
    long long grid = (b.total_tiles + warps - 1) / warps;
    grid = std::min<long long>(grid, table_grid());
    encode_table_kernel<<<(unsigned)grid, kEncThreads, 0, stream>>>(b.d_gens, b.d_tile_start, (int)b.gens.size(),
                                                                    b.total_tiles, b.d_counter);
    return cuda_status(cudaGetLastError());
}

// Tile count of one table-path generation (variant already chosen).
long long table_tiles_for(EncGen &g) { return table_tiles(g); }

// Launch the table-path kernel on descriptors already in device memory.
int launch_table_raw(const EncGen *d_gens, const long long *d_tile_start, int n_gens, long long total,
                     WorkCounter *ctr, cudaStream_t stream)
{
    if (total == 0) return GF_OK;
    const long long warps = kEncThreads / 32;
    long long grid = (total + warps - 1) / warps;
    grid = std::min<long long>(grid, table_grid());
    encode_table_kernel<<<(unsigned)grid, kEncThreads, 0, stream>>>(d_gens, d_tile_start, n_gens, total, ctr);
    return cuda_status(cudaGetLastError());
}

int plan_batches(const std::vector<EncGen> &gens, int path, std::vector<EncodeBatch> &out)
{
    out.clear();
    EncodeBatch table, bits;
    table.kind = GF_PATH_TABLE;
    bits.kind = GF_PATH_BITSLICED;
    // A batch of fewer generations than about two per SM cannot fill the GPU
    // through the table path's per-generation tiles; the tensor-core path
    // spreads each generation's column tiles over CTAs, so AUTO takes it.
    const bool small_batch = gens.size() < (size_t)(2 * sm_count());
    for (const EncGen &g0 : gens) {
        EncGen g = g0;
        int p = g0.path_hint ? g0.path_hint : path;
        if (p == GF_PATH_AUTO)
            p = small_batch && bitsliced_available() && bitsliced_supports(g)
                    ? GF_PATH_BITSLICED
                    : choose_path(g.field, g.n_src, g.n_coded, g.len);
        if (p == GF_PATH_BITSLICED) {
            if (!bitsliced_available()) {
                if (path == GF_PATH_BITSLICED) return GF_ENOTSUP;
                p = GF_PATH_TABLE;
            } else if (!bitsliced_supports(g)) {
                p = GF_PATH_TABLE;
            }
        }
        if (p == GF_PATH_BITSLICED) {
            g.variant = 0;
            bits.gens.push_back(g);
        } else if (p == GF_PATH_TABLE) {
            g.variant = choose_table_variant(g.field, g.n_src, g.n_coded, g.len);
            table.gens.push_back(g);
        } else {
            return GF_EINVAL;
        }
    }
    if (!table.gens.empty()) {
        finalize_batch(table);
        out.push_back(std::move(table));
    }
    if (!bits.gens.empty()) {
        // the persistent CTAs take work items in order: the longest items
        // (64-source chunks x column tiles x 32-packet halves) go first so
        // that no long item starts near the end
        auto item_cost = [](const EncGen &g) {
            return (long long)((g.n_src + 63) / 64) * (long long)((g.len + 127) / 128) *
                   (long long)std::min(2, (g.n_coded + 31) / 32);
        };
        std::stable_sort(bits.gens.begin(), bits.gens.end(),
                         [&](const EncGen &a, const EncGen &b) { return item_cost(a) > item_cost(b); });
        finalize_batch(bits);
        out.push_back(std::move(bits));
    }
    return GF_OK;
}

// Stage batches into a workspace (counters at the start of the buffer).
static int run_batches(std::vector<EncodeBatch> &batches, cudaStream_t stream)
{
    if (batches.empty()) return GF_OK;
    Workspace *ws = workspace_for(stream);
    size_t bytes = 0;
    for (auto &b : batches) bytes += batch_bytes(b);
    int st = ws->reserve_host(bytes);
    if (st != GF_OK) return st;
    st = ws->reserve_device(kCounterBytes + bytes, stream);
    if (st != GF_OK) return st;
    char *dev_base = (char *)ws->dev + kCounterBytes;
    size_t off = 0;
    for (size_t i = 0; i < batches.size(); ++i) {
        batches[i].d_counter = reinterpret_cast<WorkCounter *>((char *)ws->dev + 16 * i);
        off = stage_batch(batches[i], (char *)ws->host, dev_base, off);
    }
    st = ws->upload(off, stream);
    if (st != GF_OK) return st;
    for (auto &b : batches) {
        st = launch_batch(b, stream);
        if (st != GF_OK) return st;
    }
    return GF_OK;
}

int encode_batched_impl(const gf_gen_t *gens, int n_gens, int path, cudaStream_t stream)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    if (path < GF_PATH_AUTO || path > GF_PATH_BITSLICED) return GF_EINVAL;
    std::vector<EncGen> eg(n_gens);
    for (int i = 0; i < n_gens; ++i) {
        int st = convert_gen(gens[i], eg[i]);
        if (st != GF_OK) return st;
    }
    std::vector<EncodeBatch> batches;
    int st = plan_batches(eg, path, batches);
    if (st != GF_OK) return st;
    return run_batches(batches, stream);
}

// ---------------------------------------------------------------------------
// coefficient validation
// ---------------------------------------------------------------------------
__global__ void validate_kernel(const uint8_t *coef, size_t n, uint32_t q, int *bad)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (coef[i] >= q) atomicOr(bad, 1);
}

}  // namespace gf

using namespace gf;

extern "C" int gf_encode_batched(const gf_gen_t *gens, int n_gens, gf_stream_t stream)
{
    return encode_batched_impl(gens, n_gens, GF_PATH_AUTO, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gf_encode_batched_ex(const gf_gen_t *gens, int n_gens, int path, gf_stream_t stream)
{
    return encode_batched_impl(gens, n_gens, path, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gf_encode_validate(const gf_gen_t *gens, int n_gens, gf_stream_t stream)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *bad = nullptr;
    if (cudaMallocAsync((void **)&bad, sizeof(int), s) != cudaSuccess) return GF_ENOMEM;
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    int st = GF_OK;
    for (int i = 0; i < n_gens && st == GF_OK; ++i) {
        EncGen e;
        st = convert_gen(gens[i], e);
        if (st != GF_OK) break;
        const size_t n = (size_t)e.n_coded * e.n_src;
        if (n == 0) continue;
        unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
        validate_kernel<<<blocks, 256, 0, s>>>(e.coef, n, 1u << e.field, bad);
        st = cuda_status(cudaGetLastError());
    }
    int h = 0;
    if (cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) st = GF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) st = GF_ECUDA;
    cudaFreeAsync(bad, s);
    if (st == GF_OK && h) st = GF_EINVAL;
    return st;
}

// Recoding (section II: a node forwards combinations of what it received):
// the payloads and the coding vectors are combined with the same fresh
// coefficients, so each recoded generation is two encodes of one batch --
// the coding vectors as n_in "packets" of n_src bytes (one element per byte,
// upper words zero, which the packed arithmetic carries through exactly).
extern "C" int gf_recode_batched(const gf_recode_t *gens, int n_gens, gf_stream_t stream)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    std::vector<gf_gen_t> enc;
    enc.reserve(2 * (size_t)n_gens);
    for (int i = 0; i < n_gens; ++i) {
        const gf_recode_t &r = gens[i];
        if (r.n_src < 0 || r.n_in < 0 || r.n_out < 0) return GF_EINVAL;
        enc.push_back(gf_gen_t{r.field, r.n_in, r.n_out, 0, r.len, r.payload_in, r.mix, r.payload_out});
        enc.push_back(gf_gen_t{r.field, r.n_in, r.n_out, 0, (uint64_t)r.n_src, r.coef_in, r.mix, r.coef_out});
    }
    return encode_batched_impl(enc.data(), (int)enc.size(), GF_PATH_AUTO, reinterpret_cast<cudaStream_t>(stream));
}
