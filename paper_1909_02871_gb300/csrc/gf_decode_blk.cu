// gf_decode_blk.cu -- coefficient phase of the decode in blocks of 64 rows,
// its row products on the batched encode (and so on the tensor cores).
//
// The coefficient phase is progressive Gauss-Jordan over the received
// coding vectors, each augmented with its own unit vector (the transform).
// For generations with many sources (N >= 64) it runs blockwise: the
// stored rows S are kept reduced (each stored row holds 1 in its pivot
// column and 0 in every other stored row's pivot column), and for each
// block of up to 64 arriving rows:
//
//   1. F[b][t] = block row b's value in stored row t's pivot column;
//   2. cur ^= F . S, which clears every stored pivot column from the block
//      (S is reduced, so one product does it) -- a generation encode (Eq. 2)
//      of the block rows from the stored rows with coefficients F;
//   3. Gauss-Jordan within the block in arrival order (a row without a
//      pivot is dropped; it stops at rank N): new pivot rows, normalised and
//      reduced against each other, appended to S; G[t][k] = stored row t's
//      value in the k-th new pivot column;
//   4. S ^= G . NR (NR = the new pivot rows), which clears the new pivot
//      columns from the older stored rows -- another encode.
//
// Products 2 and 4 are 64-packet encodes that XOR into their output, run by
// the batched encode for every blocked generation of a decode at once.  The
// stored rows end in the same reduced form as row-by-row elimination gives
// (that form is unique), so X, rank, rows used and the solved flags are the
// same as from decode_coef_kernel.  Row operations of step 3 are split-table
// madds on 32-bit words in shared memory (gf::ByteMap).
#include <algorithm>

#include "gf_decode.h"
#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

namespace {

constexpr int kThreads = 1024;
constexpr int kGjThreads = 256;  // threads of the in-block Gauss-Jordan (several generations share an SM)

struct alignas(16) BlkMap {
    ByteMap m;
    uint32_t pad[2];
};

}  // namespace

// Step 1: the block's rows (coefficients | unit vector) into cur, zero rows
// past the block, and F.
__global__ void __launch_bounds__(kThreads) blk_prepare_kernel(const BlkGen *__restrict__ gens, int step)
{
    const BlkGen g = gens[blockIdx.x];
    const int r0 = kBlkRows * step;
    if (r0 >= g.R) return;
    const int N = g.N, W = g.W, nb = min(kBlkRows, g.R - r0);
    const int rank = g.st[0];
    const int nw = W / 4;
    for (int idx = threadIdx.x; idx < kBlkRows * nw; idx += blockDim.x) {
        const int b = idx / nw, j = idx - b * nw;
        uint32_t v = 0u;
        if (b < nb) {
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int col = 4 * j + x;
                const uint32_t byte = col < N ? (uint32_t)__ldg(g.coef + (size_t)(r0 + b) * N + col)
                                              : (col == N + r0 + b ? 1u : 0u);
                v |= byte << (8 * x);
            }
        }
        reinterpret_cast<uint32_t *>(g.cur)[idx] = v;
    }
    // F[b][t] for the stored rows t < rank (pivot columns lie in the coefficient part); zero for
    // the other rows the product reads (t < min(N, r0))
    const int nt = min(N, r0);
    for (int idx = threadIdx.x; idx < nb * nt; idx += blockDim.x) {
        const int b = idx / nt, t = idx - b * nt;
        g.F[(size_t)b * N + t] = t < rank ? __ldg(g.coef + (size_t)(r0 + b) * N + g.pcol[t]) : (uint8_t)0;
    }
}

// Step 3: Gauss-Jordan within the block, appending the new pivot rows to S,
// and G / NR for step 4.
__global__ void __launch_bounds__(kGjThreads) blk_gj_kernel(const BlkGen *__restrict__ gens, int step)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_piv, s_knew, s_rank, s_used;
    __shared__ uint32_t s_inv;
    __shared__ uint8_t s_g[kBlkRows];
    __shared__ int s_newb[kBlkRows], s_newc[kBlkRows];

    const BlkGen g = gens[blockIdx.x];
    const int r0 = kBlkRows * step;
    if (r0 >= g.R) return;
    const int N = g.N, W = g.W, n = g.field, nb = min(kBlkRows, g.R - r0);
    const int nw = W / 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t q = 1u << n;
    const int nt = min(N, r0);  // stored-row bound of the products

    BlkMap *tab = reinterpret_cast<BlkMap *>(smem);
    uint8_t *invt = reinterpret_cast<uint8_t *>(tab + 256);
    uint32_t *cur = reinterpret_cast<uint32_t *>(invt + 256);  // kBlkRows x nw words
    const uint8_t *curb = reinterpret_cast<const uint8_t *>(cur);

    if (tid == 0) {
        s_rank = g.st[0];
        s_used = g.st[1];
        s_knew = 0;
    }
    __syncthreads();
    const int rank0 = s_rank;
    if (rank0 >= N) {
        // rank N reached in an earlier block: no row is consumed; step 4 must change nothing
        for (int idx = tid; idx < nt * kBlkRows; idx += blockDim.x) g.G[idx] = 0;
        return;
    }
    for (uint32_t c = tid; c < q; c += blockDim.x) {
        tab[c].m = g_field_tables.map[table_base(n) + c];
        invt[c] = (uint8_t)g_field_tables.inv[table_base(n) + c];
    }
    // live words: rows so far carry transform entries only up to column N + r0 + nb - 1
    const int nw_r = min(nw, (N + r0 + nb + 15) / 16 * 4);
    for (int idx = tid; idx < nb * nw; idx += blockDim.x) {
        const int b = idx / nw, j = idx - b * nw;
        cur[idx] = j < nw_r ? reinterpret_cast<const uint32_t *>(g.cur)[(size_t)b * nw + j] : 0u;
    }
    __syncthreads();

    // threads share out (word j, a range of rows): per word, `per` threads split the rows, `per` a
    // power of two of at most 32 so that a word's threads lie in one warp; the words are taken
    // `slots` at a time
    int per = 1;
    while (per < 32 && 2 * per * nw_r <= kGjThreads) per *= 2;
    const int slots = kGjThreads / per;
    const int wj0 = tid / per, part = tid - wj0 * per;
    const unsigned gmask = per == 32 ? 0xffffffffu : ((1u << per) - 1u) << ((lane / per) * per);
    for (int b = 0; b < nb; ++b) {
        // pivot: first nonzero coefficient of row b (warp 0, ballot over words); the other
        // rows' values in that column are snapshotted with it
        if (warp == 0) {
            const uint32_t *row = cur + (size_t)b * nw;
            int piv = -1;
            const int ncw = (N + 3) / 4;
            for (int base = 0; base < ncw && piv < 0; base += 32) {
                const int j = base + lane;
                uint32_t v = 0;
                if (j < ncw) {
                    v = row[j];
                    const int valid = N - 4 * j;
                    if (valid < 4) v &= (1u << (8 * valid)) - 1u;
                }
                const uint32_t ball = __ballot_sync(0xffffffffu, v != 0);
                if (ball) {
                    const int src = __ffs(ball) - 1;
                    const uint32_t vw = __shfl_sync(0xffffffffu, v, src);
                    piv = 4 * (base + src) + (__ffs(vw) - 1) / 8;
                }
            }
            if (piv >= 0) {
                for (int o = lane; o < nb; o += 32) s_g[o] = o != b ? curb[(size_t)o * W + piv] : (uint8_t)0;
            }
            if (lane == 0) {
                s_piv = piv;
                if (piv >= 0) s_inv = invt[curb[(size_t)b * W + piv]];
                s_used = r0 + b + 1;
            }
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv >= 0) {
            // normalise row b and eliminate the pivot column from every other row of the block: the
            // threads of a word each normalise it (after all of them have read the old word, one of
            // them stores it) and apply it to their share of the rows (row b itself has g = 0)
            const ByteMap m = tab[s_inv].m;
            for (int wj = wj0; wj < nw_r; wj += slots) {
                const uint32_t pv = apply_word(m, cur[(size_t)b * nw + wj]);
                __syncwarp(gmask);
                if (part == 0) cur[(size_t)b * nw + wj] = pv;
                const Sel sel = make_sel(pv);
                // branch-free (g = 0 maps to zero) and unrolled, so that the rows' loads overlap
#pragma unroll 4
                for (int o = part; o < nb; o += per) cur[(size_t)o * nw + wj] ^= apply(tab[s_g[o]].m, sel);
            }
            if (tid == 0) {
                s_newb[s_knew] = b;
                s_newc[s_knew] = piv;
                s_knew = s_knew + 1;
            }
        }
        __syncthreads();
        if (rank0 + s_knew >= N) break;
    }
    const int knew = s_knew;
    // G[t][k] = stored row t's value in the k-th new pivot column (read before step 4 changes S),
    // zero past the stored rows and the new rows
    for (int idx = tid; idx < nt * kBlkRows; idx += blockDim.x) {
        const int t = idx / kBlkRows, k = idx - t * kBlkRows;
        g.G[idx] = (t < rank0 && k < knew) ? g.S[(size_t)t * W + s_newc[k]] : (uint8_t)0;
    }
    // NR = the new pivot rows (zero rows past them); the same rows appended to S
    for (int idx = tid; idx < kBlkRows * nw; idx += blockDim.x) {
        const int k = idx / nw, j = idx - k * nw;
        const uint32_t v = k < knew ? cur[(size_t)s_newb[k] * nw + j] : 0u;
        reinterpret_cast<uint32_t *>(g.NR)[idx] = v;
        if (k < knew) reinterpret_cast<uint32_t *>(g.S)[(size_t)(rank0 + k) * nw + j] = v;
    }
    if (tid < knew) g.pcol[rank0 + tid] = s_newc[tid];
    if (tid == 0) {
        g.st[0] = rank0 + knew;
        g.st[1] = s_used;
    }
}

__global__ void blk_init_kernel(const BlkGen *__restrict__ gens, int n_gens)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_gens) {
        gens[i].st[0] = 0;
        gens[i].st[1] = 0;
    }
}

// The outputs: X row p = transform part of the stored row with pivot p if
// that row reduced to the unit vector e_p, else zero; rank, rows used, the
// solved flags.
__global__ void __launch_bounds__(kThreads) blk_final_kernel(const BlkGen *__restrict__ gens)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int *pivrow = reinterpret_cast<int *>(smem);
    const BlkGen g = gens[blockIdx.x];
    const int N = g.N, R = g.R, W = g.W;
    const int rank = g.st[0];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < N; i += blockDim.x) pivrow[i] = -1;
    __syncthreads();
    for (int s = tid; s < rank; s += blockDim.x) pivrow[g.pcol[s]] = s;
    __syncthreads();
    for (int pc = warp; pc < N; pc += blockDim.x / 32) {
        const int s = pivrow[pc];
        bool unit = false;
        const uint8_t *rb = g.S + (size_t)(s >= 0 ? s : 0) * W;
        if (s >= 0) {
            bool ok = true;
            for (int k = lane; k < N; k += 32)
                if (rb[k] != (k == pc ? 1 : 0)) ok = false;
            unit = __all_sync(0xffffffffu, ok);
        }
        uint8_t *xrow = g.X + (size_t)pc * R;
        for (int k = lane; k < R; k += 32) xrow[k] = unit ? rb[N + k] : 0;
        if (lane == 0 && g.solved) g.solved[pc] = unit ? 1 : 0;
    }
    if (tid == 0) {
        if (g.rank_out) *g.rank_out = rank;
        if (g.used_out) *g.used_out = g.st[1];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

size_t blk_gj_smem(int W) { return 256 * sizeof(BlkMap) + 256 + (size_t)kBlkRows * W; }

bool blk_eligible(int field, int N, int R, int W)
{
    (void)field;
    (void)R;
    return N >= kBlkMinN && W <= kBlkMaxW && bitsliced_available();
}

size_t blk_scratch_bytes(const BlkGen &g)
{
    const size_t W = (size_t)g.W, N = (size_t)g.N;
    return align_up(N * W, 256) + 2 * align_up((size_t)kBlkRows * W, 256) + align_up((size_t)kBlkRows * N, 256) +
           align_up(N * kBlkRows, 256) + align_up(N * sizeof(int), 256) + 256;
}

void blk_place(BlkGen &g, char *base)
{
    const size_t W = (size_t)g.W, N = (size_t)g.N;
    char *p = base;
    g.S = reinterpret_cast<uint8_t *>(p);
    p += align_up(N * W, 256);
    g.cur = reinterpret_cast<uint8_t *>(p);
    p += align_up((size_t)kBlkRows * W, 256);
    g.NR = reinterpret_cast<uint8_t *>(p);
    p += align_up((size_t)kBlkRows * W, 256);
    g.F = reinterpret_cast<uint8_t *>(p);
    p += align_up((size_t)kBlkRows * N, 256);
    g.G = reinterpret_cast<uint8_t *>(p);
    p += align_up(N * kBlkRows, 256);
    g.pcol = reinterpret_cast<int *>(p);
    p += align_up(N * sizeof(int), 256);
    g.st = reinterpret_cast<int *>(p);
}

// The two products of every step as encode descriptors (generations with
// no stored rows yet, or no rows in the step, take no part).
void blk_products(const std::vector<BlkGen> &gens, int step, std::vector<EncGen> &p1, std::vector<EncGen> &p2)
{
    p1.clear();
    p2.clear();
    const int r0 = kBlkRows * step;
    for (const BlkGen &g : gens) {
        if (r0 >= g.R) continue;
        const int nt = std::min(g.N, r0), nb = std::min(kBlkRows, g.R - r0);
        if (nt == 0) continue;
        EncGen a{};
        a.field = g.field;
        a.len = (unsigned long long)g.W;
        a.accumulate = 1;
        // cur ^= F . S
        a.src = g.S;
        a.coef = g.F;
        a.coef_ld = g.N;
        a.out = g.cur;
        a.n_src = nt;
        a.n_coded = nb;
        p1.push_back(a);
        // S ^= G . NR
        EncGen b = a;
        b.src = g.NR;
        b.coef = g.G;
        b.coef_ld = kBlkRows;
        b.out = g.S;
        b.n_src = nb;
        b.n_coded = nt;
        p2.push_back(b);
    }
}

int blk_configure()
{
    static bool done[kMaxDevices] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return GF_ENOTSUP;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(blk_gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)blk_gj_smem(kBlkMaxW)) != cudaSuccess) {
            cudaGetLastError();
            return GF_ECUDA;
        }
        done[dev] = true;
    }
    return GF_OK;
}

int launch_blk_init(const BlkGen *d, int n, cudaStream_t s)
{
    blk_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(d, n);
    return cuda_status(cudaGetLastError());
}

int launch_blk_prepare(const BlkGen *d, int n, int step, cudaStream_t s)
{
    blk_prepare_kernel<<<n, kThreads, 0, s>>>(d, step);
    return cuda_status(cudaGetLastError());
}

int launch_blk_gj(const BlkGen *d, int n, int step, int max_w, cudaStream_t s)
{
    const int st = blk_configure();
    if (st != GF_OK) return st;
    blk_gj_kernel<<<n, kGjThreads, blk_gj_smem(max_w), s>>>(d, step);
    return cuda_status(cudaGetLastError());
}

int launch_blk_final(const BlkGen *d, int n, int max_n, cudaStream_t s)
{
    blk_final_kernel<<<n, kThreads, (size_t)max_n * sizeof(int), s>>>(d);
    return cuda_status(cudaGetLastError());
}

}  // namespace gf
