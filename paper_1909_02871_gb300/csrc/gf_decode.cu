// gf_decode.cu -- batched Gauss-Jordan decode.
//
// The paper describes the encoder only; decoding is the inverse linear map.
// Every row operation of a Gauss-Jordan elimination on the augmented rows
// [coding vector | payload] is determined by the coding vectors alone, so
// the library splits it in two phases:
//
//   1. coefficient phase (one CTA per generation, decode_coef_kernel):
//      progressive Gauss-Jordan over the coding vectors, rows in arrival
//      order, each row augmented with its own unit vector to record the
//      transform.  Per received row: eliminate the current pivots (the
//      stored rows are reduced, so this is one parallel vector-matrix
//      product), find the pivot (first nonzero coefficient, warp ballot),
//      drop the row if there is none, normalise it by the pivot's inverse,
//      eliminate its pivot column from every stored row, store it.  It stops
//      at rank N.  Row operations are split-table region madds on 32-bit
//      words in shared memory (gf::ByteMap); in the elimination of the new
//      row each warp sums the products of a share of the stored rows in
//      registers and the warps' sums are combined with shared-memory
//      atomicXor.  Output: X (N x R), where row p of X expresses decoded
//      source p in the received rows (zero if p is not determined), plus
//      rank, rows consumed and per-source flags.
//   2. payload phase: out = X * payload, i.e. an encode (Eq. 2) of N packets
//      from the R received packets, run by the batched encode.
//
// The decoded sources are unique once the rank is N, so this order of
// operations gives exactly the result of eliminating on the payloads row by
// row.
#include <algorithm>
#include <vector>

#include "gf_decode.h"
#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

constexpr int kDecThreads = 1024;

struct alignas(16) DecMap {
    ByteMap m;
    uint32_t pad[2];
};

// Shared-memory bytes needed by a generation when its rows live in shared
// memory (rows_in_smem) or in global memory.
size_t dec_smem_bytes(int field, int N, int W, bool rows_in_smem)
{
    size_t b = 0;
    b += align_up((size_t)(1u << field) * sizeof(DecMap), 16);  // tables
    b += 256;                                                  // inverses
    b += align_up((size_t)N * sizeof(int), 16) * 2;            // pivrow, pcol
    b += align_up((size_t)N, 16) * 2;                          // fsnap, gsnap
    b += (size_t)W;                                            // cur
    if (rows_in_smem) b += (size_t)N * W;
    return b;
}

// cur[j0 + 4 lane .. +3] ^= sum over stored rows t = warp (mod the warp count)
// of f_t * rows[t][same words]: one 16-byte shared load per row and lane, the
// row's byte map loaded once for four words; then one atomicXor per word and
// warp combines the warps (nw, j0 multiples of 4)
__device__ __forceinline__ void eliminate_rows(uint32_t *cur, const uint32_t *rows, const uint8_t *fsnap,
                                               const DecMap *tab, int rank, int nw, int nw_r, int j0, int warp,
                                               int lane)
{
    const int j = j0 + 4 * lane;
    if (j >= nw_r) return;  // lanes past the live words have nothing to add (no warp-wide operations below)
    uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
    for (int t = warp; t < rank; t += kDecThreads / 32) {
        const uint32_t f = fsnap[t];
        if (!f) continue;
        const ByteMap m = tab[f].m;
        const uint4 w = *reinterpret_cast<const uint4 *>(rows + (size_t)t * nw + j);
        a0 ^= apply_word(m, w.x);
        a1 ^= apply_word(m, w.y);
        a2 ^= apply_word(m, w.z);
        a3 ^= apply_word(m, w.w);
    }
    if (a0) atomicXor(&cur[j], a0);
    if (a1) atomicXor(&cur[j + 1], a1);
    if (a2) atomicXor(&cur[j + 2], a2);
    if (a3) atomicXor(&cur[j + 3], a3);
}

__global__ void __launch_bounds__(kDecThreads) decode_coef_kernel(const DecGen *__restrict__ gens)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_rank, s_pivot, s_used;
    __shared__ uint32_t s_inv;

    const DecGen g = gens[blockIdx.x];
    const int N = g.N, R = g.R, W = g.W, n = g.field;
    const int nw = W / 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t q = 1u << n;

    // carve shared memory
    unsigned char *p = smem;
    DecMap *tab = reinterpret_cast<DecMap *>(p);
    p += align_up((size_t)q * sizeof(DecMap), 16);
    uint8_t *invt = p;
    p += 256;
    int *pivrow = reinterpret_cast<int *>(p);  // pivot column -> stored row
    p += align_up((size_t)N * sizeof(int), 16);
    int *pcol = reinterpret_cast<int *>(p);    // stored row -> pivot column
    p += align_up((size_t)N * sizeof(int), 16);
    uint8_t *fsnap = p;
    p += align_up((size_t)N, 16);
    uint8_t *gsnap = p;
    p += align_up((size_t)N, 16);
    uint32_t *cur = reinterpret_cast<uint32_t *>(p);
    p += W;
    uint32_t *rows = g.grows ? reinterpret_cast<uint32_t *>(g.grows) : reinterpret_cast<uint32_t *>(p);
    const uint8_t *curb = reinterpret_cast<const uint8_t *>(cur);

    for (uint32_t c = tid; c < q; c += blockDim.x) {
        tab[c].m = make_bytemap(n, c);
        invt[c] = (uint8_t)finv(n, c);
    }
    for (int i = tid; i < N; i += blockDim.x) pivrow[i] = -1;
    if (tid == 0) {
        s_rank = 0;
        s_used = 0;
    }
    __syncthreads();

    // coefficient bytes of the next arriving row, prefetched a row ahead: the
    // four loads are issued here and only combined into a word when the row
    // is used, a whole row step later, so their latency is hidden (a thread
    // owns coefficient word tid; N <= 4 * kDecThreads)
    uint32_t nb[4];
    auto fetch = [&](int rr) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            nb[b] = (rr < R && 4 * tid + b < N) ? (uint32_t)__ldg(g.coef + (size_t)rr * N + 4 * tid + b) : 0u;
    };
    fetch(0);
    int r = 0;
    for (; r < R; ++r) {
        const int rank = s_rank;
        if (rank >= N) break;
        // 1. the arriving row: [coef | unit vector e_r]
        const uint32_t mine = nb[0] | (nb[1] << 8) | (nb[2] << 16) | (nb[3] << 24);
        fetch(r + 1);
        for (int j = tid; j < nw; j += blockDim.x) {
            uint32_t v = j == tid ? mine : 0u;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * j + b == N + r) v |= 1u << (8 * b);
            cur[j] = v;
        }
        __syncthreads();
        // 2. the arriving row's value in the pivot column of each stored row
        for (int t = tid; t < rank; t += blockDim.x) fsnap[t] = curb[pcol[t]];
        __syncthreads();
        // 3. cur -= sum_t f_t * row(t): stored rows are reduced, so every f_t is
        //    the arriving row's own value in row t's pivot column.  Warp w takes
        //    the stored rows t = w (mod the warp count); each lane accumulates its word
        //    columns (up to four, as many as the row is wide, in independent
        //    registers) and one atomicXor per word and warp combines the warps.
        // Rows received so far carry transform entries only in columns N .. N+r
        // (each row starts as its own unit vector), so every word past
        // column N+r is zero in the stored rows and in the arriving row:
        // the row operations stop at word nw_r.
        const int nw_r = min(nw, (N + r + 1 + 15) / 16 * 4);  // whole 16-byte groups
        if (rank > 0)
            for (int j0 = 0; j0 < nw_r; j0 += 128) eliminate_rows(cur, rows, fsnap, tab, rank, nw, nw_r, j0, warp, lane);
        __syncthreads();
        // 4. pivot: first nonzero coefficient (warp 0, ballot over words)
        if (warp == 0) {
            int piv = -1;
            const int ncw = (N + 3) / 4;
            for (int base = 0; base < ncw && piv < 0; base += 32) {
                const int j = base + lane;
                uint32_t v = 0;
                if (j < ncw) {
                    v = cur[j];
                    const int valid = N - 4 * j;  // bytes of this word inside [0, N)
                    if (valid < 4) v &= (1u << (8 * valid)) - 1u;
                }
                const uint32_t ball = __ballot_sync(0xffffffffu, v != 0);
                if (ball) {
                    const int src = __ffs(ball) - 1;
                    const uint32_t vw = __shfl_sync(0xffffffffu, v, src);
                    piv = 4 * (base + src) + (__ffs(vw) - 1) / 8;
                }
            }
            if (lane == 0) {
                s_pivot = piv;
                if (piv >= 0) s_inv = invt[curb[piv]];
            }
        }
        __syncthreads();
        const int piv = s_pivot;
        if (piv < 0) continue;  // not innovative
        // 5. normalise
        {
            const ByteMap m = tab[s_inv].m;
            for (int j = tid; j < nw_r; j += blockDim.x) cur[j] = apply_word(m, cur[j]);
        }
        // 6. column `piv` of every stored row
        for (int s = tid; s < rank; s += blockDim.x)
            gsnap[s] = reinterpret_cast<const uint8_t *>(rows + (size_t)s * nw)[piv];
        __syncthreads();
        // 7. back-substitution into the stored rows, 8. store the new row.
        //    A thread owns a word column j (its prmt selectors computed once)
        //    and walks a share of the stored rows.
        {
            const int ng = nw_r / 4;                               // 16-byte word groups
            const int per = max(1, kDecThreads / max(ng, 1));      // threads per group
            const int groups = kDecThreads / per;
            const int g_start = tid % groups, part = tid / groups;
            for (int gq = g_start; gq < ng && part < per; gq += groups) {
                const int j = 4 * gq;
                const uint4 cw = *reinterpret_cast<const uint4 *>(cur + j);
                const Sel s0 = make_sel(cw.x), s1 = make_sel(cw.y), s2 = make_sel(cw.z), s3 = make_sel(cw.w);
                for (int s = part; s < rank; s += per) {
                    const uint32_t f = gsnap[s];
                    if (!f) continue;
                    const ByteMap m = tab[f].m;
                    uint4 *rw = reinterpret_cast<uint4 *>(rows + (size_t)s * nw + j);
                    uint4 w = *rw;
                    w.x ^= apply(m, s0);
                    w.y ^= apply(m, s1);
                    w.z ^= apply(m, s2);
                    w.w ^= apply(m, s3);
                    *rw = w;
                }
                if (part == 0) *reinterpret_cast<uint4 *>(rows + (size_t)rank * nw + j) = cw;
            }
            for (int j = nw_r + tid; j < nw; j += blockDim.x) rows[(size_t)rank * nw + j] = 0u;
        }
        __syncthreads();
        if (tid == 0) {
            pivrow[piv] = rank;
            pcol[rank] = piv;
            s_rank = rank + 1;
        }
        __syncthreads();
    }
    if (tid == 0) s_used = r;
    __syncthreads();

    // outputs: X row p = transform part of the row with pivot p if that row
    // reduced to the unit vector e_p, else zero
    for (int pc = warp; pc < N; pc += blockDim.x / 32) {
        const int s = pivrow[pc];
        bool unit = false;
        if (s >= 0) {
            const uint8_t *rb = reinterpret_cast<const uint8_t *>(rows + (size_t)s * nw);
            bool ok = true;
            for (int k = lane; k < N; k += 32)
                if (rb[k] != (k == pc ? 1 : 0)) ok = false;
            unit = __all_sync(0xffffffffu, ok);
        }
        uint8_t *xrow = g.X + (size_t)pc * R;
        const uint8_t *rb = reinterpret_cast<const uint8_t *>(rows + (size_t)(s >= 0 ? s : 0) * nw);
        for (int k = lane; k < R; k += 32) xrow[k] = unit ? rb[N + k] : 0;
        if (lane == 0 && g.solved) g.solved[pc] = unit ? 1 : 0;
    }
    if (tid == 0) {
        if (g.rank) *g.rank = s_rank;
        if (g.used) *g.used = s_used;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static size_t smem_limit()
{
    static int cached = 0;
    if (!cached) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, current_device()) != cudaSuccess ||
            v <= 0)
            v = 48 * 1024;
        cached = v;
    }
    return (size_t)cached - 1024;  // room for the kernel's static shared memory
}

int build_decode(const gf_dec_t *gens, int n_gens, DecodeWork &w)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    w = DecodeWork{};
    w.gens.resize(n_gens);
    std::vector<EncGen> apply(n_gens);
    size_t x_bytes = 0, grow_bytes = 0;
    const size_t limit = smem_limit();
    for (int i = 0; i < n_gens; ++i) {
        const gf_dec_t &d = gens[i];
        if (!field_ok(d.field) || d.n_src < 0 || d.n_src > kMaxDecodeN || d.n_recv < 0 ||
            d.n_recv > kMaxDecodeR || d.reserved != 0)
            return GF_EINVAL;
        if (!d.rank) return GF_EINVAL;
        if (d.n_src > 0 && d.len > 0 && !d.out) return GF_EINVAL;
        if (d.n_recv > 0 && d.n_src > 0 && !d.coef) return GF_EINVAL;
        if (d.n_recv > 0 && d.len > 0 && !d.payload) return GF_EINVAL;
        DecGen &g = w.gens[i];
        g = DecGen{};
        g.coef = d.coef;
        g.payload = d.payload;
        g.out = d.out;
        g.rank = d.rank;
        g.used = d.used;
        g.solved = d.solved;
        g.len = d.len;
        g.field = d.field;
        g.N = d.n_src;
        g.R = d.n_recv;
        g.W = (int)align_up((size_t)d.n_src + (size_t)d.n_recv, 16);
        g.x_off = x_bytes;
        x_bytes += align_up((size_t)g.N * g.R, 256);
        const bool in_smem = dec_smem_bytes(g.field, g.N, g.W, true) <= limit;
        g.grow_off = in_smem ? (size_t)-1 : grow_bytes;
        if (!in_smem) grow_bytes += align_up((size_t)g.N * g.W, 256);
        w.smem = std::max(w.smem, dec_smem_bytes(g.field, g.N, g.W, in_smem));
        EncGen &e = apply[i];
        e = EncGen{};
        e.src = d.payload;
        e.coef = nullptr;  // set once X is placed
        e.out = d.out;
        e.len = d.len;
        e.field = d.field;
        e.n_src = d.n_recv;
        e.n_coded = d.n_src;
        e.coef_ld = d.n_recv;
    }
    w.x_bytes = x_bytes;
    w.grow_bytes = grow_bytes;
    w.apply = std::move(apply);
    return GF_OK;
}

// Place X / global rows at `dev_x`, then build the apply batches.
int place_decode(DecodeWork &w, char *dev_x, char *dev_rows)
{
    for (size_t i = 0; i < w.gens.size(); ++i) {
        DecGen &g = w.gens[i];
        g.X = reinterpret_cast<uint8_t *>(dev_x + g.x_off);
        g.grows = g.grow_off == (size_t)-1 ? nullptr : reinterpret_cast<uint8_t *>(dev_rows + g.grow_off);
        w.apply[i].coef = g.X;
    }
    return plan_batches(w.apply, GF_PATH_AUTO, w.batches);
}

int launch_decode_coef(const DecodeWork &w, const DecGen *d_gens, cudaStream_t stream)
{
    if (w.gens.empty()) return GF_OK;
    if (w.smem > 48 * 1024) {
        if (cudaFuncSetAttribute(decode_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w.smem) !=
            cudaSuccess)
            return GF_ECUDA;
    }
    decode_coef_kernel<<<(unsigned)w.gens.size(), kDecThreads, w.smem, stream>>>(d_gens);
    return cuda_status(cudaGetLastError());
}

// Launch the coefficient phase on descriptors already in device memory.
int launch_decode_coef_raw(const DecGen *d_gens, int n_gens, size_t smem, cudaStream_t stream)
{
    if (n_gens == 0) return GF_OK;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(decode_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return GF_ECUDA;
    }
    decode_coef_kernel<<<(unsigned)n_gens, kDecThreads, smem, stream>>>(d_gens);
    return cuda_status(cudaGetLastError());
}

size_t decode_stage_bytes(const DecodeWork &w)
{
    size_t b = align_up(w.gens.size() * sizeof(DecGen), 256);
    for (const auto &bt : w.batches) b += batch_bytes(bt);
    return b;
}

// Serialise DecGens + apply batches into host at `off`, device pointers
// relative to dev_base; returns the new offset.
size_t stage_decode(DecodeWork &w, char *host, char *dev_base, size_t off, WorkCounter *counters)
{
    const size_t gb = w.gens.size() * sizeof(DecGen);
    // one CTA per generation, scheduled roughly in block order: the most
    // expensive eliminations (N^2 (N + R) row operations) go first so that
    // none of them starts near the end of the launch
    std::vector<DecGen> order(w.gens);
    std::stable_sort(order.begin(), order.end(), [](const DecGen &a, const DecGen &b) {
        return (double)a.N * a.N * (a.N + a.R) > (double)b.N * b.N * (b.N + b.R);
    });
    memcpy(host + off, order.data(), gb);
    w.d_gens = reinterpret_cast<DecGen *>(dev_base + off);
    off += align_up(gb, 256);
    for (size_t i = 0; i < w.batches.size(); ++i) {
        w.batches[i].d_counter = counters + i;
        off = stage_batch(w.batches[i], host, dev_base, off);
    }
    return off;
}

int launch_decode(const DecodeWork &w, cudaStream_t stream)
{
    int st = launch_decode_coef(w, w.d_gens, stream);
    if (st != GF_OK) return st;
    for (const auto &b : w.batches) {
        st = launch_batch(b, stream);
        if (st != GF_OK) return st;
    }
    return GF_OK;
}

static int decode_batched_impl(const gf_dec_t *gens, int n_gens, cudaStream_t stream)
{
    DecodeWork w;
    int st = build_decode(gens, n_gens, w);
    if (st != GF_OK || n_gens == 0) return st;
    Workspace *ws = workspace_for(stream);
    // layout: [counters][x][rows][staged descriptors]
    // (a first pass places X to size the staged part, which does not depend on it)
    const size_t x_total = align_up(w.x_bytes, 256), r_total = align_up(w.grow_bytes, 256);
    st = ws->reserve_device(kCounterBytes + x_total + r_total + (1u << 16), stream);
    if (st != GF_OK) return st;
    // descriptors are staged after X and rows; compute their size with a
    // provisional placement, then reserve and place for real
    st = place_decode(w, (char *)ws->dev + kCounterBytes, (char *)ws->dev + kCounterBytes + x_total);
    if (st != GF_OK) return st;
    const size_t stage = decode_stage_bytes(w);
    st = ws->reserve_device(kCounterBytes + x_total + r_total + stage, stream);
    if (st != GF_OK) return st;
    char *dev_x = (char *)ws->dev + kCounterBytes;
    char *dev_rows = dev_x + x_total;
    st = place_decode(w, dev_x, dev_rows);
    if (st != GF_OK) return st;
    st = ws->reserve_host(x_total + r_total + stage);
    if (st != GF_OK) return st;
    // stage the descriptors at the same offset they occupy on the device
    const size_t off0 = x_total + r_total;
    const size_t end = stage_decode(w, (char *)ws->host, (char *)ws->dev + kCounterBytes, off0,
                                    reinterpret_cast<WorkCounter *>(ws->dev));
    if (cudaMemcpyAsync((char *)ws->dev + kCounterBytes + off0, (char *)ws->host + off0, end - off0,
                        cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return GF_ECUDA;
    if (!ws->staged && cudaEventCreateWithFlags(&ws->staged, cudaEventDisableTiming) != cudaSuccess) return GF_ECUDA;
    if (cudaEventRecord(ws->staged, stream) != cudaSuccess) return GF_ECUDA;
    return launch_decode(w, stream);
}

}  // namespace gf

using namespace gf;

extern "C" int gf_decode_batched(const gf_dec_t *gens, int n_gens, gf_stream_t stream)
{
    return decode_batched_impl(gens, n_gens, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gf_decode_check(const gf_dec_t *gens, int n_gens, gf_stream_t stream)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GF_ECUDA;
    for (int i = 0; i < n_gens; ++i) {
        if (!gens[i].rank) return GF_EINVAL;
        int32_t r = 0;
        if (cudaMemcpy(&r, gens[i].rank, sizeof(r), cudaMemcpyDeviceToHost) != cudaSuccess) return GF_ECUDA;
        if (r < gens[i].n_src) return GF_ERANK;
    }
    return GF_OK;
}
