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
//      transform; a row's pivot is its first nonzero coefficient once the
//      earlier pivots are eliminated, a row without one is dropped, and it
//      stops at rank N.  Rows are taken in batches of kDecBatch: the stored
//      rows are reduced, so eliminating them from every batch row is one
//      parallel product in which each stored word's prmt selectors serve
//      all the batch rows (each warp sums a share of the stored rows in
//      registers, shared-memory atomicXor combines the warps); then the
//      batch is settled row by row in arrival order (pivot by warp ballot,
//      normalisation by the pivot's inverse, the pivot column eliminated
//      from every other batch row at once), and one sweep back-substitutes
//      the batch's new pivots into the stored rows.  The stored rows end in
//      the same reduced form as row-by-row elimination gives (that form is
//      unique), so the outputs do not depend on the batching.  Row
//      operations are split-table region madds on 32-bit words in shared
//      memory (gf::ByteMap).  Output: X (N x R), where row p of X expresses
//      decoded source p in the received rows (zero if p is not determined),
//      plus rank, rows consumed and per-source flags.
//   2. payload phase: out = X * payload, i.e. an encode (Eq. 2) of N packets
//      from the R received packets, run by the batched encode.
//
// The decoded sources are unique once the rank is N, so this order of
// operations gives exactly the result of eliminating on the payloads row by
// row.
#include <algorithm>
#include <mutex>
#include <vector>

#include "gf_decode.h"
#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

constexpr int kDecThreads = 1024;
constexpr int kDecSmallThreads = 256, kDecSmallN = 64;
constexpr int kDecBatch = 4;  // arriving rows eliminated against the stored rows together

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
    b += align_up((size_t)N * kDecBatch, 16) * 2;              // F, G snapshots
    b += (size_t)W * kDecBatch;                                // the batch's rows
    if (rows_in_smem) b += (size_t)N * W;
    return b;
}

// cur[b][j0 + 2 lane .. +1] ^= sum over stored rows t = warp (mod the warp
// count) of F[b][t] * rows[t][same words], for the nb rows b of the batch:
// the prmt selectors of a stored word are computed once and applied with
// each row's coefficient (the point of eliminating rows in batches); then one
// atomicXor per word, row and warp combines the warps (nw_r, j0 even)
__device__ __forceinline__ void eliminate_batch(uint32_t *cur, const uint32_t *rows, const uint8_t *F, int N,
                                                const DecMap *tab, int rank, int nw, int nw_r, int nb, int j0,
                                                int warp, int lane)
{
    const int j = j0 + 2 * lane;
    if (j >= nw_r) return;  // lanes past the live words have nothing to add (no warp-wide operations below)
    uint32_t acc[kDecBatch][2];
#pragma unroll
    for (int b = 0; b < kDecBatch; ++b) acc[b][0] = acc[b][1] = 0u;
    for (int t = warp; t < rank; t += blockDim.x / 32) {
        uint32_t f[kDecBatch];
        uint32_t any = 0u;
#pragma unroll
        for (int b = 0; b < kDecBatch; ++b) {
            f[b] = b < nb ? (uint32_t)F[b * N + t] : 0u;
            any |= f[b];
        }
        if (!any) continue;
        const uint2 w = *reinterpret_cast<const uint2 *>(rows + (size_t)t * nw + j);
        const Sel s0 = make_sel(w.x), s1 = make_sel(w.y);
#pragma unroll
        for (int b = 0; b < kDecBatch; ++b) {
            if (!f[b]) continue;
            const ByteMap m = tab[f[b]].m;
            acc[b][0] ^= apply(m, s0);
            acc[b][1] ^= apply(m, s1);
        }
    }
#pragma unroll
    for (int b = 0; b < kDecBatch; ++b) {
        if (b >= nb) break;
        if (acc[b][0]) atomicXor(&cur[b * nw + j], acc[b][0]);
        if (acc[b][1]) atomicXor(&cur[b * nw + j + 1], acc[b][1]);
    }
}

__global__ void __launch_bounds__(kDecThreads) decode_coef_kernel(const DecGen *__restrict__ gens)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_rank, s_pivot, s_used, s_knew;
    __shared__ uint32_t s_inv;
    __shared__ int s_newb[kDecBatch], s_newc[kDecBatch];  // the batch's pivot rows and their columns
    __shared__ uint8_t s_g[kDecBatch];                    // each batch row's value in the new pivot column

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
    uint8_t *F = p;                            // F[b * N + t]: batch row b in stored row t's pivot column
    p += align_up((size_t)N * kDecBatch, 16);
    uint8_t *G = p;                            // G[t * kDecBatch + k]: stored row t in the k-th new pivot column
    p += align_up((size_t)N * kDecBatch, 16);
    uint32_t *cur = reinterpret_cast<uint32_t *>(p);  // batch row b at cur + b * nw
    p += (size_t)W * kDecBatch;
    uint32_t *rows = g.grows ? reinterpret_cast<uint32_t *>(g.grows) : reinterpret_cast<uint32_t *>(p);
    const uint8_t *curb = reinterpret_cast<const uint8_t *>(cur);
    const uint8_t *rowsb = reinterpret_cast<const uint8_t *>(rows);

    for (uint32_t c = tid; c < q; c += blockDim.x) {
        tab[c].m = g_field_tables.map[table_base(n) + c];
        invt[c] = (uint8_t)g_field_tables.inv[table_base(n) + c];
    }
    for (int i = tid; i < N; i += blockDim.x) pivrow[i] = -1;
    if (tid == 0) {
        s_rank = 0;
        s_used = 0;
    }
    __syncthreads();

    for (int r0 = 0;; r0 += kDecBatch) {
        const int rank = s_rank;  // stored rows before this batch
        if (r0 >= R || rank >= N) break;
        const int nb = min(kDecBatch, R - r0);
        // Rows received so far carry transform entries only in columns N .. N+r0+nb-1 (each row
        // starts as its own unit vector), so every word past that is zero in the stored rows and
        // in the batch: the row operations stop at word nw_r.
        const int nw_r = min(nw, (N + r0 + nb + 15) / 16 * 4);  // whole 16-byte groups
        // 1. the batch's rows: [coef | unit vector e_r] over the live words
        for (int idx = tid; idx < nb * nw_r; idx += blockDim.x) {
            const int b = idx / nw_r, j = idx - b * nw_r;
            uint32_t v = 0u;
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int col = 4 * j + x;
                const uint32_t byte = col < N ? (uint32_t)__ldg(g.coef + (size_t)(r0 + b) * N + col)
                                              : (col == N + r0 + b ? 1u : 0u);
                v |= byte << (8 * x);
            }
            cur[b * nw + j] = v;
        }
        if (tid == 0) s_knew = 0;
        __syncthreads();
        // 2. each batch row's value in the pivot column of each stored row
        for (int idx = tid; idx < nb * rank; idx += blockDim.x) {
            const int b = idx / rank, t = idx - b * rank;
            F[b * N + t] = curb[b * W + pcol[t]];
        }
        __syncthreads();
        // 3. cur[b] -= sum_t F[b][t] * row(t) for every batch row: the stored rows are reduced,
        //    so every F[b][t] is row b's own value in row t's pivot column
        if (rank > 0)
            for (int j0 = 0; j0 < nw_r; j0 += 64) eliminate_batch(cur, rows, F, N, tab, rank, nw, nw_r, nb, j0, warp, lane);
        __syncthreads();
        // 4. Gauss-Jordan within the batch, in arrival order: each new pivot row is normalised and
        //    its pivot column eliminated from every other batch row at once (the earlier pivot
        //    rows stay reduced, the later rows arrive at their turn already reduced)
        if (nw_r <= 32) {
            // rows of at most 32 words: warp 0 alone, lane j holding word j of every batch row in
            // registers (no block barrier per row); the same order and rules as below
            if (warp == 0) {
                uint32_t c[kDecBatch];
#pragma unroll
                for (int o = 0; o < kDecBatch; ++o) c[o] = (o < nb && lane < nw_r) ? cur[o * nw + lane] : 0u;
                int rk = rank, kn = 0, used = s_used;
                const int ncw = (N + 3) / 4;
                // coefficient bytes of the lane's word (columns < N)
                const uint32_t cmask = lane < ncw ? (N - 4 * lane >= 4 ? 0xFFFFFFFFu : (1u << (8 * (N - 4 * lane))) - 1u) : 0u;
#pragma unroll
                for (int b = 0; b < kDecBatch; ++b) {
                    if (b >= nb || rk >= N) break;
                    used = r0 + b + 1;
                    const uint32_t ball = __ballot_sync(0xffffffffu, (c[b] & cmask) != 0u);
                    if (!ball) continue;  // no pivot: the row is not innovative and is dropped
                    const int src = __ffs(ball) - 1;
                    const uint32_t vw = __shfl_sync(0xffffffffu, c[b] & cmask, src);
                    const int byte = (__ffs(vw) - 1) >> 3;
                    const int piv = 4 * src + byte;
                    const uint32_t pv = (vw >> (8 * byte)) & 0xFFu;
                    // the other rows' values in the pivot column, before anything changes
                    uint32_t gv[kDecBatch];
#pragma unroll
                    for (int o = 0; o < kDecBatch; ++o)
                        gv[o] = (__shfl_sync(0xffffffffu, c[o], src) >> (8 * byte)) & 0xFFu;
                    c[b] = apply_word(tab[invt[pv]].m, c[b]);
                    const Sel sel = make_sel(c[b]);
#pragma unroll
                    for (int o = 0; o < kDecBatch; ++o)
                        if (o != b && o < nb && gv[o]) c[o] ^= apply(tab[gv[o]].m, sel);
                    if (lane == 0) {
                        s_newb[kn] = b;
                        s_newc[kn] = piv;
                    }
                    ++kn;
                    ++rk;
                }
#pragma unroll
                for (int o = 0; o < kDecBatch; ++o)
                    if (o < nb && lane < nw_r) cur[o * nw + lane] = c[o];
                if (lane == 0) {
                    s_knew = kn;
                    s_rank = rk;
                    s_used = used;
                }
            }
            __syncthreads();
        } else {
            for (int b = 0; b < nb; ++b) {
                // 4a. pivot: first nonzero coefficient of row b (warp 0, ballot over words); the
                //     other batch rows' values in that column are snapshotted with it
                if (warp == 0) {
                    const uint32_t *row = cur + b * nw;
                    int piv = -1;
                    const int ncw = (N + 3) / 4;
                    for (int base = 0; base < ncw && piv < 0; base += 32) {
                        const int j = base + lane;
                        uint32_t v = 0;
                        if (j < ncw) {
                            v = row[j];
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
                        if (piv >= 0) s_inv = invt[curb[b * W + piv]];
                        s_used = r0 + b + 1;
                    }
                    if (piv >= 0 && lane < nb) s_g[lane] = lane != b ? curb[lane * W + piv] : 0;
                }
                __syncthreads();
                const int piv = s_pivot;
                // 4b. normalise row b and eliminate its pivot column from the other batch rows (a
                //     thread owns a word column of every batch row); a row without a pivot is not
                //     innovative and is dropped
                if (piv >= 0) {
                    const ByteMap m = tab[s_inv].m;
                    for (int j = tid; j < nw_r; j += blockDim.x) {
                        const uint32_t pv = apply_word(m, cur[b * nw + j]);
                        cur[b * nw + j] = pv;
                        const Sel sel = make_sel(pv);
    #pragma unroll
                        for (int o = 0; o < kDecBatch; ++o) {
                            if (o >= nb) break;
                            const uint32_t go = s_g[o];
                            if (o != b && go) cur[o * nw + j] ^= apply(tab[go].m, sel);
                        }
                    }
                }
                if (tid == 0 && piv >= 0) {
                    const int knew = s_knew;
                    s_newb[knew] = b;
                    s_newc[knew] = piv;
                    s_knew = knew + 1;
                    s_rank = s_rank + 1;
                }
                __syncthreads();  // also keeps the pivot shared state of this row until every thread has read it
                if (s_rank >= N) break;
            }
        }
        const int knew = s_knew;
        // 5. back-substitution of the batch's pivots into the stored rows, one sweep: G first
        if (knew > 0 && rank > 0)
            for (int idx = tid; idx < rank * knew; idx += blockDim.x) {
                const int t = idx / knew, k = idx - t * knew;
                G[t * kDecBatch + k] = rowsb[(size_t)t * W + s_newc[k]];
            }
        __syncthreads();
        //    a thread owns a word column j (the prmt selectors of each new pivot row's words
        //    computed once) and walks a share of the stored rows
        if (knew > 0 && rank > 0) {
            const int ng = nw_r / 4;                               // 16-byte word groups
            const int per = max(1, (int)blockDim.x / max(ng, 1));  // threads per group
            const int groups = (int)blockDim.x / per;
            const int g_start = tid % groups, part = tid / groups;
            for (int gq = g_start; gq < ng && part < per; gq += groups) {
                const int j = 4 * gq;
                for (int k = 0; k < knew; ++k) {
                    const uint4 cw = *reinterpret_cast<const uint4 *>(cur + s_newb[k] * nw + j);
                    const Sel s0 = make_sel(cw.x), s1 = make_sel(cw.y), s2 = make_sel(cw.z), s3 = make_sel(cw.w);
                    for (int s = part; s < rank; s += per) {
                        const uint32_t f = G[s * kDecBatch + k];
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
                }
            }
        }
        // 6. store the batch's pivot rows after the stored ones (zero past the live words)
        for (int idx = tid; idx < knew * nw; idx += blockDim.x) {
            const int k = idx / nw, j = idx - k * nw;
            rows[(size_t)(rank + k) * nw + j] = j < nw_r ? cur[s_newb[k] * nw + j] : 0u;
        }
        if (tid < knew) {
            pivrow[s_newc[tid]] = rank + tid;
            pcol[rank + tid] = s_newc[tid];
        }
        __syncthreads();
    }
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

// Largest dynamic shared memory a decode CTA may use on the current device
// (the opt-in limit less room for the kernel's static shared memory).
size_t decode_smem_limit()
{
    static std::mutex mu;
    static int cached[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return 48 * 1024 - 1024;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 48 * 1024;
        cached[dev] = v;
    }
    return (size_t)cached[dev] - 1024;
}

// decode_coef_kernel's dynamic shared-memory limit, raised once per device to
// decode_smem_limit() (the attribute belongs to the function, not to a launch, so
// it is never lowered for a smaller launch).
static int configure_decode_coef()
{
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return GF_ENOTSUP;
    const size_t limit = decode_smem_limit();
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(decode_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) !=
            cudaSuccess) {
            cudaGetLastError();
            return GF_ECUDA;
        }
        done[dev] = true;
    }
    return GF_OK;
}

int build_decode(const gf_dec_t *gens, int n_gens, DecodeWork &w)
{
    if (n_gens < 0 || (n_gens > 0 && !gens)) return GF_EINVAL;
    w = DecodeWork{};
    w.gens.resize(n_gens);
    std::vector<EncGen> apply(n_gens);
    size_t x_bytes = 0, grow_bytes = 0;
    const size_t limit = decode_smem_limit();
    for (int i = 0; i < n_gens; ++i) {
        const gf_dec_t &d = gens[i];
        if (!field_ok(d.field) || d.n_src < 0 || d.n_src > kMaxDecodeN || d.n_recv < 0 ||
            d.n_recv > kMaxDecodeR || (d.flags & ~GF_DEC_SYSTEMATIC) != 0)
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
        g.blk = -1;
        g.grow_off = (size_t)-1;
        if (g.R > 0 && blk_eligible(g.field, g.N, g.R, g.W)) {
            // many sources: the blocked coefficient phase, its scratch in the rows region
            BlkGen b{};
            b.coef = d.coef;
            b.rank_out = d.rank;
            b.used_out = d.used;
            b.solved = d.solved;
            b.field = d.field;
            b.N = g.N;
            b.R = g.R;
            b.W = g.W;
            b.off = grow_bytes;
            grow_bytes += align_up(blk_scratch_bytes(b), 256);
            g.blk = (int)w.blk.size();
            w.blk.push_back(b);
            w.blk_max_w = std::max(w.blk_max_w, g.W);
            w.blk_max_n = std::max(w.blk_max_n, g.N);
        } else {
            const bool in_smem = dec_smem_bytes(g.field, g.N, g.W, true) <= limit;
            if (!in_smem) {
                g.grow_off = grow_bytes;
                grow_bytes += align_up((size_t)g.N * g.W, 256);
            }
            w.smem = std::max(w.smem, dec_smem_bytes(g.field, g.N, g.W, in_smem));
        }
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
        // mostly unit rows in the transform: the table path skips their zero multipliers
        e.path_hint = (d.flags & GF_DEC_SYSTEMATIC) ? GF_PATH_TABLE : 0;
    }
    w.x_bytes = x_bytes;
    w.grow_bytes = grow_bytes;
    w.apply = std::move(apply);
    return GF_OK;
}

// Place X / global rows at `dev_x`, then build the apply batches and the
// blocked generations' row-product batches.
int place_decode(DecodeWork &w, char *dev_x, char *dev_rows)
{
    for (size_t i = 0; i < w.gens.size(); ++i) {
        DecGen &g = w.gens[i];
        g.X = reinterpret_cast<uint8_t *>(dev_x + g.x_off);
        g.grows = g.grow_off == (size_t)-1 ? nullptr : reinterpret_cast<uint8_t *>(dev_rows + g.grow_off);
        w.apply[i].coef = g.X;
        if (g.blk >= 0) {
            BlkGen &b = w.blk[g.blk];
            b.X = g.X;
            blk_place(b, dev_rows + b.off);
        }
    }
    int st = plan_batches(w.apply, GF_PATH_AUTO, w.batches);
    if (st != GF_OK) return st;
    int max_r = 0;
    for (const BlkGen &b : w.blk) max_r = std::max(max_r, b.R);
    const int steps = (max_r + kBlkRows - 1) / kBlkRows;
    w.prod1.assign(steps, {});
    w.prod2.assign(steps, {});
    std::vector<EncGen> p1, p2;
    for (int s = 0; s < steps; ++s) {
        blk_products(w.blk, s, p1, p2);
        if (!p1.empty() && (st = plan_batches(p1, GF_PATH_AUTO, w.prod1[s])) != GF_OK) return st;
        if (!p2.empty() && (st = plan_batches(p2, GF_PATH_AUTO, w.prod2[s])) != GF_OK) return st;
    }
    return GF_OK;
}

int launch_decode_coef(const DecodeWork &w, const DecGen *d_gens, cudaStream_t stream)
{
    if (w.n_coef == 0) return GF_OK;
    const int st = configure_decode_coef();
    if (st != GF_OK) return st;
    decode_coef_kernel<<<(unsigned)w.n_coef, (unsigned)w.coef_threads, w.smem, stream>>>(d_gens);
    return cuda_status(cudaGetLastError());
}

// Launch the coefficient phase on descriptors already in device memory
// (smem <= decode_smem_limit()).
int launch_decode_coef_raw(const DecGen *d_gens, int n_gens, size_t smem, cudaStream_t stream)
{
    if (n_gens == 0) return GF_OK;
    const int st = configure_decode_coef();
    if (st != GF_OK) return st;
    decode_coef_kernel<<<(unsigned)n_gens, kDecThreads, smem, stream>>>(d_gens);
    return cuda_status(cudaGetLastError());
}

size_t decode_stage_bytes(const DecodeWork &w)
{
    size_t b = align_up(w.gens.size() * sizeof(DecGen), 256);
    for (const auto &bt : w.batches) b += batch_bytes(bt);
    b += align_up(w.blk.size() * sizeof(BlkGen), 256);
    for (const auto &step : w.prod1)
        for (const auto &bt : step) b += batch_bytes(bt);
    for (const auto &step : w.prod2)
        for (const auto &bt : step) b += batch_bytes(bt);
    return b;
}

// Work counters a staged decode needs (one per batched launch).
size_t decode_counters(const DecodeWork &w)
{
    size_t n = w.batches.size();
    for (const auto &step : w.prod1) n += step.size();
    for (const auto &step : w.prod2) n += step.size();
    return n;
}

// Serialise DecGens + apply batches into host at `off`, device pointers
// relative to dev_base; returns the new offset.
size_t stage_decode(DecodeWork &w, char *host, char *dev_base, size_t off, WorkCounter *counters)
{
    // one CTA per generation of decode_coef_kernel, scheduled roughly in block order: the most
    // expensive eliminations (N^2 (N + R) row operations) go first so that none of them starts
    // near the end of the launch (blocked generations are not its work)
    std::vector<DecGen> order;
    for (const DecGen &g : w.gens)
        if (g.blk < 0) order.push_back(g);
    std::stable_sort(order.begin(), order.end(), [](const DecGen &a, const DecGen &b) {
        return (double)a.N * a.N * (a.N + a.R) > (double)b.N * b.N * (b.N + b.R);
    });
    w.n_coef = (int)order.size();
    // small generations: a 256-thread CTA (a few words per row operation; fewer warps make the
    // barriers between the row steps cheaper)
    int max_n = 0;
    for (const DecGen &g : order) max_n = std::max(max_n, g.N);
    w.coef_threads = max_n <= kDecSmallN ? kDecSmallThreads : kDecThreads;
    const size_t gb = order.size() * sizeof(DecGen);
    if (gb) memcpy(host + off, order.data(), gb);
    w.d_gens = reinterpret_cast<DecGen *>(dev_base + off);
    off += align_up(w.gens.size() * sizeof(DecGen), 256);
    size_t c = 0;
    for (size_t i = 0; i < w.batches.size(); ++i) {
        w.batches[i].d_counter = counters + c++;
        off = stage_batch(w.batches[i], host, dev_base, off);
    }
    const size_t bb = w.blk.size() * sizeof(BlkGen);
    if (bb) memcpy(host + off, w.blk.data(), bb);
    w.d_blk = reinterpret_cast<BlkGen *>(dev_base + off);
    off += align_up(bb, 256);
    for (auto *prods : {&w.prod1, &w.prod2})
        for (auto &step : *prods)
            for (auto &bt : step) {
                bt.d_counter = counters + c++;
                off = stage_batch(bt, host, dev_base, off);
            }
    return off;
}

int launch_decode(const DecodeWork &w, cudaStream_t stream)
{
    int st = launch_decode_coef(w, w.d_gens, stream);
    if (st != GF_OK) return st;
    if (!w.blk.empty()) {
        const int nb = (int)w.blk.size();
        if ((st = launch_blk_init(w.d_blk, nb, stream)) != GF_OK) return st;
        for (size_t s = 0; s < w.prod1.size(); ++s) {
            if ((st = launch_blk_prepare(w.d_blk, nb, (int)s, stream)) != GF_OK) return st;
            for (const auto &b : w.prod1[s])
                if ((st = launch_batch(b, stream)) != GF_OK) return st;
            if ((st = launch_blk_gj(w.d_blk, nb, (int)s, w.blk_max_w, stream)) != GF_OK) return st;
            for (const auto &b : w.prod2[s])
                if ((st = launch_batch(b, stream)) != GF_OK) return st;
        }
        if ((st = launch_blk_final(w.d_blk, nb, w.blk_max_n, stream)) != GF_OK) return st;
    }
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
    if (decode_counters(w) > kCounterBytes / sizeof(WorkCounter)) return GF_EINVAL;
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
