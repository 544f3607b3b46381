// gf_encode_tc.cu -- bit-sliced GF(256) generation encode on the sm_103a
// tensor cores (tcgen05, kind::f8f6f4, FP32 accumulators in TMEM).
//
// The imul algorithm of section IV-B rests on the identity
//     c * a = XOR_j a_j * (c * x^j),        a_j = bit j of a,
// i.e. multiplication by c is the GF(2)-linear map whose 8x8 bit matrix has
// column j = c*x^j.  Eq. 2 over a whole generation therefore becomes one
// binary matrix product:
//     bit r of out_k[l] = sum_{i,j} bit_j(src_i[l]) * bit_r(c_ki * x^j)  (mod 2)
// The tensor core computes the integer sum exactly (0/1 operands, sums of
// at most 512 terms, exact in the FP16 accumulator) and the parity is the
// result's lowest bit.  The kernel computes the product transposed, one
// 128-byte column tile at a time:
//     D[l, 8k'+r] = sum_{(i,j)} A[l, 8i+j] * B[8i+j, 8k'+r]
//   A (M = 128 byte positions x K = 8N source bits): written by the producer
//     warps straight into tensor memory with tcgen05.st (one TMEM lane per
//     byte position, 4 FP8 elements per column), no shared-memory traffic;
//   B (K = 8N x N = 256 output bits of 32 coded packets): the coefficients'
//     bit matrices as FP8 0/1, K-major, 128-byte swizzled, resident in shared
//     memory for the whole work item (N <= 64: 128 KB), copied from a 16 KB
//     per-CTA table of the 256 possible 8x8 blocks;
//   D (128 lanes x 256 FP16 columns): one N = 256 MMA stream per tile (full
//     FP8 rate); the epilogue reads two columns per register
//     (tcgen05.ld .pack::16b), adds 1024 so the integer sum sits in the
//     mantissa, takes bit 0 of each of the 8 values of a coded byte and packs
//     them.
// Work item = (generation, 32 coded packets); the CTA loops over all column
// tiles of the item.  Roles, all running concurrently: 2 warps publish the
// next item in a two-entry ring and build its B; 8 producer warps stage
// their source rows in shared memory with cp.async two tiles ahead and fill
// A (double-buffered in TMEM, via a 2 KB table of pre-spread FP8 words);
// 1 thread issues the MMAs; 16 epilogue warps drain D.  Every handshake
// arrives once per warp (after __syncwarp), never once per thread.  Every
// mbarrier wait is bounded by the global timer; a wait that gives up
// records GF_ETIMEOUT in the library's device status word, the CTA drains
// its MMAs (bounded), frees TMEM and exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gf_encode.h"
#include "gf_internal.cuh"

namespace gf {

namespace tc {

constexpr int kProducerWarps = 8;   // 2 per TMEM lane quarter, 32 sources each
constexpr int kEpilogueWarps = 16;  // 4 per lane quarter, 8 coded packets each
constexpr int kBWarps = 4;          // coefficient bit matrices (B)
constexpr int kMmaWarp = kProducerWarps + kEpilogueWarps;  // warp 24
constexpr int kBWarp0 = kMmaWarp + 1;                       // warps 25..28
constexpr int kThreads = (kProducerWarps + kEpilogueWarps + 1 + kBWarps) * 32;  // 928
constexpr int kColTile = 128;       // byte positions per tile (MMA M)
constexpr int kCodedPerItem = 32;   // coded packets per work item (MMA N = 256 output bits)
constexpr int kMaxSrc = 64;         // N limit of this path (A: 128 TMEM columns, B: 128 KB)
constexpr int kSrcPerProducer = 32;
constexpr int kStages = 3;          // source staging depth (tiles) per producer warp
constexpr int kStageBytes = kSrcPerProducer * 32;  // 32 sources x 32 byte positions
constexpr int kTmemCols = 512;
constexpr int kABufCols = 128;      // A buffers at columns 0 and 128
constexpr int kDCol0 = 256;         // D: 256 columns from column 256
constexpr uint32_t kOne = 0x38u;    // 1.0 in E4M3
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait
constexpr uint32_t kSuspendNs = 100000;                 // try_wait suspend hint
constexpr long long kSentinel = -1;

// shared memory layout (dynamic, 1024-aligned base)
constexpr int kKBlock = 256 * 128;          // one K-block of B: 256 rows x 128 bytes
constexpr int kBBytes = 4 * kKBlock;        // 128 KB: B of one item (K <= 512)
constexpr int kTabBytes = 256 * 8 * 8;      // 16 KB: 8x8 FP8 block of every coefficient
constexpr int kStageAll = kProducerWarps * kStages * kStageBytes;  // 24 KB source staging
constexpr int kSpreadBytes = 256 * 8;       // 2 KB: the 8 FP8 bit values of every source byte
constexpr int kSmemBytes = kBBytes + kTabBytes + kStageAll + kSpreadBytes + 1024 /*control*/ + 1024 /*slack*/;

struct Ctl {
    unsigned long long a_full[2], a_empty[2], d_full, d_empty;
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

// 32 lanes x 32 columns of 16-bit values, two adjacent columns per register
__device__ __forceinline__ void tmem_ld16_pack(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.pack::16b.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
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

// Instruction descriptor, kind::f8f6f4: D = F16 (integer sums <= 512 are
// exact), A = B = E4M3, both K-major, N = 256, M = 128.  An F16 accumulator
// still takes one tensor-memory column per element (low 16 bits).  (N = 256 runs at the full FP8 rate whatever the commit
// cadence; two N = 128 streams with commits between them run about a third
// slower.)
constexpr uint32_t kIdesc = (0u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(256 >> 3) << 17) |
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

// parity byte of 8 FP16 sums packed two per word (word j = output bits 2j,
// 2j+1): adding 1024 puts the integer sum in the mantissa, so bit 0 of each
// half is the parity
__device__ __forceinline__ uint32_t parity_byte_h(const uint32_t *v)
{
    uint32_t h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) asm("add.rn.f16x2 %0, %1, %2;" : "=r"(h[j]) : "r"(v[j]), "r"(0x64006400u));
    const uint32_t q0 = prmt(h[0], h[1], 0x6420u) & 0x01010101u;
    const uint32_t q1 = prmt(h[2], h[3], 0x6420u) & 0x01010101u;
    return ((q0 * 0x01020408u) >> 24) | (((q1 * 0x01020408u) >> 24) << 4);
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

// this producer thread's 32 source bytes of column `col` straight from
// global memory (generations whose rows are not 4-byte aligned)
__device__ __forceinline__ void load_direct(const EncGen &g, int ibase, unsigned long long col, uint32_t (&b)[8],
                                            int grp)
{
    const unsigned long long len = g.len;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int i = ibase + grp * 8 + t;
        b[t] = (col < len && i < g.n_src) ? (uint32_t)__ldg(g.src + (size_t)i * len + col) : 0u;
    }
}

// Stage this warp's 32 sources x 32 byte positions of column tile `ct` into
// shared memory with 4-byte cp.async (rows 4-byte aligned); bytes outside
// the generation are zero-filled.
__device__ __forceinline__ void stage_tile(const EncGen &g, int ibase, int quarter, int ct, unsigned char *stage,
                                           int lane)
{
    const unsigned long long len = g.len;
    const unsigned long long c0 = (unsigned long long)ct * kColTile + quarter * 32;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int w = lane + 32 * j;      // word of the 32 x 32-byte block
        const int row = w >> 3, wc = w & 7;
        const int i = ibase + row;
        const unsigned long long col = c0 + 4 * wc;
        uint32_t bytes = 0;
        const uint8_t *src = g.src;
        if (i < g.n_src && col < len) {
            bytes = (uint32_t)min(4ull, len - col);
            src = g.src + (size_t)i * len + col;
        }
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(stage + row * 32 + 4 * wc)),
                     "l"(src), "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
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
    unsigned long long *tab = reinterpret_cast<unsigned long long *>(smem + kBBytes);  // [r][c]
    unsigned char *staging = smem + kBBytes + kTabBytes;
    uint2 *spread = reinterpret_cast<uint2 *>(smem + kBBytes + kTabBytes + kStageAll);  // [source byte]
    Ctl *ctl = reinterpret_cast<Ctl *>(smem + kBBytes + kTabBytes + kStageAll + kSpreadBytes);
    volatile int *abort_flag = &ctl->abort;
    volatile long long *ring = ctl->ring_item;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the 8x8 FP8 block of every coefficient: row r, byte j = bit r of c*x^j,
    // stored [r][c] so that lanes looking up different coefficients for the
    // same row spread over all shared-memory banks
    for (int e = tid; e < 256 * 8; e += blockDim.x) {
        const uint32_t c = (uint32_t)e & 255u, r = (uint32_t)e >> 8;
        uint32_t p = c;
        unsigned long long row = 0;
        for (int j = 0; j < 8; ++j) {
            if ((p >> r) & 1u) row |= (unsigned long long)kOne << (8 * j);
            p = xtime(8, p);
        }
        tab[e] = row;
    }
    for (int b = tid; b < 256; b += blockDim.x) {
        uint2 v;
        spread_bits((uint32_t)b, v.x, v.y);
        spread[b] = v;
    }
    if (tid == 0) {
        mbar_init(&ctl->d_full, 1);
        mbar_init(&ctl->d_empty, kEpilogueWarps);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->a_full[b], kProducerWarps);
            mbar_init(&ctl->a_empty[b], 1);
            mbar_init(&ctl->info_full[b], 1);
            mbar_init(&ctl->info_empty[b], kProducerWarps + kEpilogueWarps + 1);
        }
        mbar_init(&ctl->b_full, 1);
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
        const int kq0 = bt >> 5;         // coded-packet octet kq0 (0..3)
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
            const int kbase = (int)(item - __ldg(tile_start + gi)) * kCodedPerItem;
            const int N = g.n_src, K = g.n_coded, ld = g.coef_ld;
            const int nkb = (N + 15) / 16;
            const int i0 = 16 * kb + 2 * m, i1 = i0 + 1;
            uint32_t cc[8];  // coefficient pair (c[k][i0], c[k][i1]) packed in 16 bits
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = kbase + kq0 * 8 + t;
                const uint32_t a = (kb < nkb && k < K && i0 < N) ? (uint32_t)__ldg(g.coef + (size_t)k * ld + i0) : 0u;
                const uint32_t b = (kb < nkb && k < K && i1 < N) ? (uint32_t)__ldg(g.coef + (size_t)k * ld + i1) : 0u;
                cc[t] = a | (b << 8);
            }
            // B is single-buffered: wait until the MMAs of the previous item are done
            bool ok = true;
            if (bt == 0) ok = mbar_wait(&ctl->b_empty, (seq & 1u) ^ 1u, abort_flag);
            if (bt == 0 && !ok) ctl->abort = 1;
            asm volatile("bar.sync 1, %0;" ::"r"(kBWarps * 32) : "memory");
            if (kb < nkb) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kp = kq0 * 8 + t;
                    const bool live = kbase + kp < K;
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const unsigned long long v0 = live ? tab[r * 256 + (cc[t] & 0xFFu)] : 0ull;
                        const unsigned long long v1 = live ? tab[r * 256 + (cc[t] >> 8)] : 0ull;
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
            asm volatile("bar.sync 1, %0;" ::"r"(kBWarps * 32) : "memory");
            if (bt == 0) mbar_arrive(&ctl->b_full);
            if (*abort_flag) break;
        }
    } else if (warp < kProducerWarps) {
        // ---------------- producers: A = source bit planes -> TMEM ----------------
        const int quarter = warp & 3;          // TMEM lane quarter
        const int part = warp >> 2;            // which 32 sources of the 64
        const int pos = quarter * 32 + lane;   // byte position within the column tile
        const int ibase = part * kSrcPerProducer;
        unsigned char *stage = staging + warp * (kStages * kStageBytes);
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
            const bool staged = ((((uintptr_t)g.src) | (uintptr_t)g.len) & 3u) == 0;
            if (staged) {
                // always kStages-1 groups in flight before the loop (empty ones past the row end)
                for (int p = 0; p < kStages - 1; ++p) {
                    if (p < ncols) stage_tile(g, ibase, quarter, p, stage + p * kStageBytes, lane);
                    else asm volatile("cp.async.commit_group;" ::: "memory");
                }
            }
            bool ok = true;
            for (int ct = 0; ct < ncols; ++ct) {
                if (staged) {
                    __syncwarp();  // every lane is done reading the stage about to be refilled
                    if (ct + kStages - 1 < ncols)
                        stage_tile(g, ibase, quarter, ct + kStages - 1, stage + ((ct + kStages - 1) % kStages) * kStageBytes,
                                   lane);
                    else
                        asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
                    __syncwarp();
                }
                const uint32_t buf = fills & 1u, fu = fills >> 1;
                if (!mbar_wait_warp(&ctl->a_empty[buf], (fu & 1u) ^ 1u, abort_flag)) {
                    ctl->abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acol = tmem + ((uint32_t)(quarter * 32) << 16) + buf * kABufCols + part * 64;
                const unsigned char *sb = stage + (ct % kStages) * kStageBytes + lane;
#pragma unroll
                for (int grp = 0; grp < 4; ++grp) {
                    uint32_t b[8];
                    if (staged) {
#pragma unroll
                        for (int t = 0; t < 8; ++t) b[t] = sb[(grp * 8 + t) * 32];
                    } else {
                        load_direct(g, ibase, (unsigned long long)ct * kColTile + pos, b, grp);
                    }
                    uint32_t v[16];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const uint2 w = spread[b[t]];
                        v[2 * t] = w.x;
                        v[2 * t + 1] = w.y;
                    }
                    tmem_st16(acol + grp * 16, v);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->a_full[buf]);
                ++fills;
            }
            if (staged) asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (!ok) break;
        }
    } else if (warp < kProducerWarps + kEpilogueWarps) {
        // ---------------- epilogue: 64 D columns -> parity bytes -> global ----------------
        const int quarter = warp & 3;
        const int oct = (warp - kProducerWarps) >> 2;   // 8-packet group of the item: 0..3
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
            const int k0 = (int)(item - __ldg(tile_start + gi)) * kCodedPerItem + oct * 8;
            const int K = g.n_coded;
            const unsigned long long len = g.len;
            const int ncols = (int)((len + kColTile - 1) / kColTile);
            bool ok = true;
            for (int ct = 0; ct < ncols; ++ct) {
                if (!mbar_wait_warp(&ctl->d_full, tiles & 1u, abort_flag)) {
                    ctl->abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = tmem + ((uint32_t)(quarter * 32) << 16) + kDCol0 + oct * 64;
                uint32_t va[16], vb[16];
                tmem_ld16_pack(dcol, va);
                tmem_ld16_pack(dcol + 32, vb);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->d_empty);  // D is free as soon as it is in registers
                uint32_t outb[8];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    outb[t] = parity_byte_h(va + 4 * t);
                    outb[4 + t] = parity_byte_h(vb + 4 * t);
                }
                const unsigned long long col = (unsigned long long)ct * kColTile + pos;
                if (col < len) {
                    uint8_t *o = g.out + (size_t)k0 * len + col;
#pragma unroll
                    for (int kp = 0; kp < 8; ++kp)
                        if (k0 + kp < K) o[(size_t)kp * len] = (uint8_t)outb[kp];
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
            bool ok = mbar_wait(&ctl->b_full, seq & 1u, abort_flag);
            tc_fence_after();
            const uint64_t bdesc0 = b_desc(smem_u32(Bs));
            for (int ct = 0; ct < ncols && ok; ++ct) {
                const uint32_t buf = fills & 1u, fu = fills >> 1;
                if (!mbar_wait(&ctl->a_full[buf], fu & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                if (!mbar_wait(&ctl->d_empty, (tiles & 1u) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // descriptors advance by the byte offset >> 4 (no carry out of the 14-bit field:
                // B lies below 256 KB of shared memory)
                const uint32_t dt = tmem + kDCol0;
                const uint32_t at = tmem + buf * kABufCols;
                tc_mma(dt, at, bdesc0, kIdesc, 0u);
#pragma unroll
                for (int s = 1; s < 16; ++s) {
                    if (s < ksteps)
                        tc_mma(dt, at + s * 8, bdesc0 + (uint64_t)((((s * 32) >> 7) * kKBlock + ((s * 32) & 127)) >> 4),
                               kIdesc, 1u);
                }
                tc_commit(&ctl->d_full);
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
