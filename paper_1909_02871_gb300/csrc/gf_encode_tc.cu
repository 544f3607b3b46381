// gf_encode_tc.cu -- bit-sliced GF(256) generation encode on the sm_103a
// tensor cores (tcgen05, kind::f8f6f4, FP32 accumulators in TMEM).
//
// The imul algorithm of section IV-B rests on the identity
//     c * a = XOR_j a_j * (c * x^j),        a_j = bit j of a,
// i.e. multiplication by c is the GF(2)-linear map whose 8x8 bit matrix has
// column j = c*x^j.  Eq. 2 over a whole generation therefore becomes one
// binary matrix product:
//     bit r of out_k[l] = sum_{i,j} bit_j(src_i[l]) * bit_r(c_ki * x^j)  (mod 2)
// The tensor core computes the integer sum exactly (0/1 operands, sums below
// 2^24 in FP32) and the parity is the result's lowest bit.  The kernel
// computes the product transposed, one 128-byte column tile at a time:
//     D[l, 8k'+r] = sum_{(i,j)} A[l, 8i+j] * B[8i+j, 8k'+r]
//   A (M = 128 byte positions x K = 8N source bits): written by the producer
//     warps straight into tensor memory with tcgen05.st (one TMEM lane per
//     byte position, 4 FP8 elements per column), no shared-memory traffic;
//   B (K = 8N x N = 128 output bits of 16 coded packets): the coefficients'
//     bit matrices as FP8 0/1, K-major, 128-byte swizzled, resident in shared
//     memory for the whole work item (N <= 64: 64 KB), copied from a 16 KB
//     per-CTA table of the 256 possible 8x8 blocks;
//   D (128 lanes x 128 FP32 columns), double-buffered in TMEM; the epilogue
//     adds 2^23 (so the integer sum sits in the mantissa), takes bit 0 of
//     each of the 8 values of a coded byte and packs them.
// Work item = (generation, 16 coded packets); the CTA loops over all column
// tiles of the item.  Roles, all running concurrently: 2 warps build B for
// the next item into the other of two B buffers (a two-entry item ring in
// shared memory hands the item index to the other roles); 16 producer warps
// fill A (double-buffered in TMEM), prefetching the next tile's source bytes;
// 1 thread issues the MMAs; 8 epilogue warps drain D (double-buffered).  Every mbarrier wait is bounded
// by the global timer; a wait that gives up records GF_ETIMEOUT in the
// library's device status word, the CTA drains its MMAs (bounded), frees
// TMEM and exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

namespace tc {

constexpr int kProducerWarps = 16;  // 4 per TMEM lane quarter, 16 sources each
constexpr int kEpilogueWarps = 8;   // 4 per D half (one per lane quarter)
constexpr int kBWarps = 4;          // coefficient bit matrices (B)
constexpr int kMmaWarp = kProducerWarps + kEpilogueWarps;  // warp 24
constexpr int kBWarp0 = kMmaWarp + 1;                       // warps 25..28
constexpr int kThreads = (kProducerWarps + kEpilogueWarps + 1 + kBWarps) * 32;  // 928
constexpr int kColTile = 128;       // byte positions per tile (MMA M)
constexpr int kCodedPerHalf = 16;   // coded packets per D half (MMA N = 128 output bits)
constexpr int kCodedPerItem = 32;   // coded packets per work item (two D halves)
constexpr int kMaxSrc = 64;         // N limit of this path (A: 128 TMEM columns, B: 128 KB)
constexpr int kSrcPerProducer = 16;
constexpr int kTmemCols = 512;
constexpr int kABufCols = 128;      // A buffers at columns 0 and 128
constexpr int kDCol0 = 256;         // D halves at columns 256 and 384
constexpr uint32_t kOne = 0x38u;    // 1.0 in E4M3
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait
constexpr uint32_t kSuspendNs = 100000;                 // try_wait suspend hint
constexpr long long kSentinel = -1;

// shared memory layout (dynamic, 1024-aligned base)
constexpr int kKBlock = 256 * 128;          // one K-block of B: 256 rows x 128 bytes
constexpr int kBBytes = 4 * kKBlock;        // 128 KB: B of one item (K <= 512)
constexpr int kTabBytes = 256 * 8 * 8;      // 16 KB: 8x8 FP8 block of every coefficient
constexpr int kSmemBytes = kBBytes + kTabBytes + 1024 /*control*/ + 1024 /*alignment slack*/;

struct Ctl {
    unsigned long long a_full[2], a_empty[2], d_full[2], d_empty[2];
    unsigned long long info_full[2], info_empty[2], b_full, b_empty, drain;
    long long ring_item[2];
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the phase did not complete within kWaitNs or the
// CTA is aborting.
__device__ __noinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

// Warp-uniform bounded wait: lane 0 waits, the warp adopts its outcome, so
// the warp-collective tcgen05.ld/st that follow always run with all lanes.
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long *bar, uint32_t parity, volatile int *abort)
{
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();  // lane 0's acquire of the barrier phase covers the whole warp
    return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t b_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

// byte offset of 16-byte chunk m of K-block kb in row n (K-major, 128B swizzle)
__device__ __forceinline__ uint32_t b_chunk_offset(int n, int kb, int m)
{
    return (uint32_t)(kb * (128 * 128) + (n >> 3) * 1024 + (n & 7) * 128 + ((m ^ (n & 7)) << 4));
}

// 8 FP8 values (bytes j = 0..7) of one source byte: 1.0 where bit j is set
__device__ __forceinline__ void spread_bits(uint32_t b, uint32_t &lo, uint32_t &hi)
{
    lo = (((b & 0xFu) * 0x00204081u) & 0x01010101u) * kOne;
    hi = (((b >> 4) * 0x00204081u) & 0x01010101u) * kOne;
}

// parity byte of 8 FP32 sums (columns 8k'..8k'+7 = output bits r = 0..7)
__device__ __forceinline__ uint32_t parity_byte(const uint32_t *v)
{
    uint32_t w[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) w[r] = __float_as_uint(__uint_as_float(v[r]) + 8388608.0f);
    const uint32_t q0 = prmt(prmt(w[0], w[1], 0x0040u), prmt(w[2], w[3], 0x0040u), 0x5410u) & 0x01010101u;
    const uint32_t q1 = prmt(prmt(w[4], w[5], 0x0040u), prmt(w[6], w[7], 0x0040u), 0x5410u) & 0x01010101u;
    return ((q0 * 0x01020408u) >> 24) | (((q1 * 0x01020408u) >> 24) << 4);
}

__device__ __forceinline__ int locate(const long long *tile_start, int n_gens, long long item)
{
    int lo = 0, hi = n_gens - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// this producer thread's 16 source bytes of column `col` (0 outside the generation)
__device__ __forceinline__ void load_sources(const EncGen &g, int ibase, unsigned long long col,
                                             uint32_t (&b)[kSrcPerProducer])
{
    const unsigned long long len = g.len;
    const uint8_t *p = g.src + (size_t)ibase * len + col;
    if (col < len && ibase + kSrcPerProducer <= g.n_src) {
#pragma unroll
        for (int t = 0; t < kSrcPerProducer; ++t) b[t] = (uint32_t)__ldg(p + (size_t)t * len);
    } else {
#pragma unroll
        for (int t = 0; t < kSrcPerProducer; ++t)
            b[t] = (col < len && ibase + t < g.n_src) ? (uint32_t)__ldg(p + (size_t)t * len) : 0u;
    }
}

// Shared-memory offset of 16-byte chunk m of K-block kb in B row n (K-major,
// 128-byte swizzle: 8-row atoms of 1024 bytes, chunk index XOR row % 8).
__device__ __forceinline__ uint32_t b_chunk(int n, int kb, int m)
{
    return (uint32_t)(kb * kKBlock + (n >> 3) * 1024 + (n & 7) * 128 + ((m ^ (n & 7)) << 4));
}

__global__ void __launch_bounds__(kThreads, 1)
encode_bitsliced_kernel(const EncGen *__restrict__ gens, const long long *__restrict__ tile_start, int n_gens,
                        long long total, WorkCounter *ctr, int *status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Bs = smem;
    unsigned long long *tab = reinterpret_cast<unsigned long long *>(smem + kBBytes);  // [c][r]
    Ctl *ctl = reinterpret_cast<Ctl *>(smem + kBBytes + kTabBytes);
    volatile int *abort_flag = &ctl->abort;
    volatile long long *ring = ctl->ring_item;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the 8x8 FP8 block of every coefficient: row r, byte j = bit r of c*x^j
    for (int e = tid; e < 256 * 8; e += blockDim.x) {
        const uint32_t c = (uint32_t)e >> 3, r = (uint32_t)e & 7u;
        uint32_t p = c;
        unsigned long long row = 0;
        for (int j = 0; j < 8; ++j) {
            if ((p >> r) & 1u) row |= (unsigned long long)kOne << (8 * j);
            p = xtime(8, p);
        }
        tab[e] = row;
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->a_full[b], kProducerWarps * 32);
            mbar_init(&ctl->a_empty[b], 1);
            mbar_init(&ctl->d_full[b], 1);
            mbar_init(&ctl->d_empty[b], (kEpilogueWarps / 2) * 32);
            mbar_init(&ctl->info_full[b], 1);
            mbar_init(&ctl->info_empty[b], kProducerWarps + kEpilogueWarps + 1);
        }
        mbar_init(&ctl->b_full, kBWarps * 32);
        mbar_init(&ctl->b_empty, 1);
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp >= kBWarp0) {
        // ------------- B builder: publishes the next item, then its bit matrices -------------
        const int bt = tid - kBWarp0 * 32;
        const int m = bt & 7;            // 16-byte chunk in a K-block: sources 2m, 2m+1
        const int kb = (bt >> 3) & 3;    // K-block: sources 16kb .. 16kb+15
        const int kq = bt >> 5;          // coded packets 8kq .. 8kq+7 of the item
        for (uint32_t seq = 0;; ++seq) {
            const uint32_t e = seq & 1u, use = seq >> 1;
            if (bt == 0) {
                const bool ok = mbar_wait(&ctl->info_empty[e], (use & 1u) ^ 1u, abort_flag);
                long long it = ok ? (long long)atomicAdd(&ctr->next, 1ull) : kSentinel;
                if (it >= total) it = kSentinel;
                if (!ok) ctl->abort = 1;
                ring[e] = it;
                mbar_arrive(&ctl->info_full[e]);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kBWarps * 32) : "memory");
            const long long item = ring[e];
            if (item == kSentinel) break;
            const int gi = locate(tile_start, n_gens, item);
            const EncGen g = gens[gi];
            const int k0 = (int)(item - __ldg(tile_start + gi)) * kCodedPerItem + kq * 8;
            const int N = g.n_src, K = g.n_coded, ld = g.coef_ld;
            const int nkb = (N + 15) / 16;
            const int i0 = 16 * kb + 2 * m, i1 = i0 + 1;
            uint32_t c0[8], c1[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = k0 + t;
                c0[t] = (kb < nkb && k < K && i0 < N) ? (uint32_t)__ldg(g.coef + (size_t)k * ld + i0) : 0u;
                c1[t] = (kb < nkb && k < K && i1 < N) ? (uint32_t)__ldg(g.coef + (size_t)k * ld + i1) : 0u;
            }
            // B is single-buffered: wait until the MMAs of the previous item are done
            bool ok = true;
            if (bt == 0) ok = mbar_wait(&ctl->b_empty, (seq & 1u) ^ 1u, abort_flag);
            if (bt == 0 && !ok) ctl->abort = 1;
            asm volatile("bar.sync 1, %0;" ::"r"(kBWarps * 32) : "memory");
            if (kb < nkb) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kp = kq * 8 + t;
                    const bool live = k0 + t < K;
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const unsigned long long v0 = live ? tab[c0[t] * 8 + r] : 0ull;
                        const unsigned long long v1 = live ? tab[c1[t] * 8 + r] : 0ull;
                        uint4 q;
                        q.x = (uint32_t)v0;
                        q.y = (uint32_t)(v0 >> 32);
                        q.z = (uint32_t)v1;
                        q.w = (uint32_t)(v1 >> 32);
                        *reinterpret_cast<uint4 *>(Bs + b_chunk(8 * kp + r, kb, m)) = q;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&ctl->b_full);
            if (*abort_flag) break;
        }
    } else if (warp < kProducerWarps) {
        // ---------------- producers: A = source bit planes -> TMEM ----------------
        const int quarter = warp & 3;          // TMEM lane quarter
        const int part = warp >> 2;            // which 16 sources of the 64
        const int pos = quarter * 32 + lane;   // byte position within the column tile
        uint32_t fills = 0;
        for (uint32_t seq = 0;; ++seq) {
            const uint32_t e = seq & 1u, use = seq >> 1;
            if (!mbar_wait_warp(&ctl->info_full[e], use & 1u, abort_flag)) {
                ctl->abort = 1;
                break;
            }
            const long long item = ring[e];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->info_empty[e]);
            if (item < 0) break;
            const int gi = locate(tile_start, n_gens, item);
            const EncGen g = gens[gi];
            const int ncols = (int)((g.len + kColTile - 1) / kColTile);
            const int ibase = part * kSrcPerProducer;
            uint32_t bx[kSrcPerProducer], by[kSrcPerProducer];
            load_sources(g, ibase, (unsigned long long)pos, bx);
            bool ok = true;
            for (int ct = 0; ct < ncols && ok; ct += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = ct + h;
                    if (c >= ncols) break;
                    uint32_t(&cur)[kSrcPerProducer] = h == 0 ? bx : by;
                    uint32_t(&nxt)[kSrcPerProducer] = h == 0 ? by : bx;
                    if (c + 1 < ncols) load_sources(g, ibase, (unsigned long long)(c + 1) * kColTile + pos, nxt);
                    const uint32_t buf = fills & 1u, fu = fills >> 1;
                    if (!mbar_wait_warp(&ctl->a_empty[buf], (fu & 1u) ^ 1u, abort_flag)) {
                        ctl->abort = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t acol = tmem + ((uint32_t)(quarter * 32) << 16) + buf * kABufCols + part * 32;
#pragma unroll
                    for (int grp = 0; grp < 2; ++grp) {
                        uint32_t v[16];
#pragma unroll
                        for (int t = 0; t < 8; ++t) spread_bits(cur[grp * 8 + t], v[2 * t], v[2 * t + 1]);
                        tmem_st16(acol + grp * 16, v);
                    }
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&ctl->a_full[buf]);
                    ++fills;
                }
            }
            if (!ok) break;
        }
    } else if (warp < kProducerWarps + kEpilogueWarps) {
        // ---------------- epilogue: D half -> parity bytes -> global ----------------
        const int quarter = warp & 3;
        const int half = (warp - kProducerWarps) >> 2;  // D half = coded packets 16*half .. +15
        const int pos = quarter * 32 + lane;
        uint32_t tiles = 0;
        for (uint32_t seq = 0;; ++seq) {
            const uint32_t e = seq & 1u, use = seq >> 1;
            if (!mbar_wait_warp(&ctl->info_full[e], use & 1u, abort_flag)) {
                ctl->abort = 1;
                break;
            }
            const long long item = ring[e];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->info_empty[e]);
            if (item < 0) break;
            const int gi = locate(tile_start, n_gens, item);
            const EncGen g = gens[gi];
            const int k0 = (int)(item - __ldg(tile_start + gi)) * kCodedPerItem + half * kCodedPerHalf;
            const int K = g.n_coded;
            const unsigned long long len = g.len;
            const int ncols = (int)((len + kColTile - 1) / kColTile);
            bool ok = true;
            for (int ct = 0; ct < ncols; ++ct) {
                if (!mbar_wait_warp(&ctl->d_full[half], tiles & 1u, abort_flag)) {
                    ctl->abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = tmem + ((uint32_t)(quarter * 32) << 16) + kDCol0 + half * 128;
                const unsigned long long col = (unsigned long long)ct * kColTile + pos;
                uint8_t *o = g.out + (size_t)k0 * len + col;
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    uint32_t outb[8];
#pragma unroll
                    for (int g2 = 0; g2 < 2; ++g2) {
                        uint32_t v[32];
                        tmem_ld32(dcol + (pr * 2 + g2) * 32, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int t = 0; t < 4; ++t) outb[g2 * 4 + t] = parity_byte(v + 8 * t);
                    }
                    if (pr == 1) {
                        tc_fence_before();
                        mbar_arrive(&ctl->d_empty[half]);
                    }
                    if (col < len) {
#pragma unroll
                        for (int kp = 0; kp < 8; ++kp)
                            if (k0 + pr * 8 + kp < K) o[(size_t)(pr * 8 + kp) * len] = (uint8_t)outb[kp];
                    }
                }
                ++tiles;
            }
            if (!ok) break;
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer (warp kMmaWarp, one thread) ----------------
        uint32_t fills = 0, tiles = 0;
        for (uint32_t seq = 0;; ++seq) {
            const uint32_t e = seq & 1u, use = seq >> 1;
            if (!mbar_wait(&ctl->info_full[e], use & 1u, abort_flag)) {
                ctl->abort = 1;
                break;
            }
            const long long item = ring[e];
            mbar_arrive(&ctl->info_empty[e]);
            if (item < 0) break;
            const int gi = locate(tile_start, n_gens, item);
            const EncGen g = gens[gi];
            const int ncols = (int)((g.len + kColTile - 1) / kColTile);
            const int ksteps = (g.n_src + 3) / 4;  // 4 sources = 32 FP8 per MMA
            const int k_item = g.n_coded - (int)(item - __ldg(tile_start + gi)) * kCodedPerItem;
            const int halves = k_item > kCodedPerHalf ? 2 : 1;
            bool ok = mbar_wait(&ctl->b_full, seq & 1u, abort_flag);
            tc_fence_after();
            const uint32_t b_base = smem_u32(Bs);
            for (int ct = 0; ct < ncols && ok; ++ct) {
                const uint32_t buf = fills & 1u, fu = fills >> 1;
                if (!mbar_wait(&ctl->a_full[buf], fu & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int h = 0; h < halves; ++h) {
                    if (!mbar_wait(&ctl->d_empty[h], (tiles & 1u) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + kDCol0 + h * 128;
                    for (int s = 0; s < ksteps; ++s) {
                        const int kglob = s * 32;  // byte offset in K
                        const uint32_t baddr =
                            b_base + (uint32_t)((kglob >> 7) * kKBlock + h * (128 * 128) + (kglob & 127));
                        tc_mma(dt, tmem + buf * kABufCols + s * 8, b_desc(baddr), kIdesc, s > 0 ? 1u : 0u);
                    }
                    tc_commit(&ctl->d_full[h]);
                }
                if (!ok) break;
                if (halves == 1) {
                    // keep both halves' phases in step: the idle half completes an empty phase
                    if (!mbar_wait(&ctl->d_empty[1], (tiles & 1u) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_commit(&ctl->d_full[1]);
                }
                tc_commit(&ctl->a_empty[buf]);
                ++fills;
                ++tiles;
            }
            tc_commit(&ctl->b_empty);
            if (!ok) {
                ctl->abort = 1;
                break;
            }
        }
    }

    __syncthreads();
    // drain: wait (bounded) for every MMA this CTA issued, then free TMEM
    if (warp == kMmaWarp) {
        if (lane == 0) {
            tc_commit(&ctl->drain);
            const unsigned long long t0 = now_ns();
            while (!mbar_try(&ctl->drain, 0) && now_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
    if (tid == 0 && ctl->abort) atomicExch(status, GF_ETIMEOUT);
    // the last CTA to finish returns the counters to zero for the next launch
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&ctr->done, 1ull);
        if (prev == (unsigned long long)gridDim.x - 1ull) {
            ctr->next = 0ull;
            ctr->done = 0ull;
            __threadfence();
        }
    }
}

}  // namespace tc

bool bitsliced_available()
{
    static std::mutex mu;
    static int cached_dev = -1;
    static bool ok = false;
    std::lock_guard<std::mutex> lock(mu);
    const int dev = current_device();
    if (dev != cached_dev) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        ok = (major == 10 && minor == 3);
        cached_dev = dev;
    }
    return ok;
}

bool bitsliced_supports(const EncGen &g)
{
    return g.field == 8 && g.n_src > 0 && g.n_src <= tc::kMaxSrc && g.n_coded > 0 && g.len > 0;
}

long long bitsliced_tiles(const EncGen &g, int &col_chunks, int &k_chunks)
{
    if (!bitsliced_supports(g)) {
        col_chunks = k_chunks = 0;
        return 0;
    }
    col_chunks = 1;
    k_chunks = (g.n_coded + tc::kCodedPerItem - 1) / tc::kCodedPerItem;
    return k_chunks;
}

int launch_bitsliced(const EncodeBatch &b, cudaStream_t stream)
{
    static std::mutex mu;
    static int configured_dev = -1;
    {
        std::lock_guard<std::mutex> lock(mu);
        const int dev = current_device();
        if (dev != configured_dev) {
            if (cudaFuncSetAttribute(tc::encode_bitsliced_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tc::kSmemBytes) != cudaSuccess)
                return GF_ECUDA;
            configured_dev = dev;
        }
    }
    int *status = device_status_word();
    if (!status) return GF_ENOMEM;
    const long long grid = std::min<long long>(b.total_tiles, sm_count());
    tc::encode_bitsliced_kernel<<<(unsigned)grid, tc::kThreads, tc::kSmemBytes, stream>>>(
        b.d_gens, b.d_tile_start, (int)b.gens.size(), b.total_tiles, b.d_counter, status);
    return cuda_status(cudaGetLastError());
}

}  // namespace gf
