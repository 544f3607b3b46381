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
//     memory for the whole work item, copied from a 16 KB per-CTA table of
//     the 256 possible 8x8 blocks;
//   D (128 lanes x 128 FP32 columns), double-buffered in TMEM; the epilogue
//     adds 2^23 (so the integer sum sits in the mantissa), takes bit 0 of
//     each of the 8 values of a coded byte and packs them.
// Work item = (generation, 16 coded packets); the CTA loops over all column
// tiles of the item.  Roles: 8 producer warps (A), 4 epilogue warps (D),
// 1 warp that owns TMEM and issues the MMAs.  Every mbarrier wait is bounded
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

constexpr int kProducerWarps = 8;
constexpr int kEpilogueWarps = 4;
constexpr int kThreads = (kProducerWarps + kEpilogueWarps + 1) * 32;  // 416
constexpr int kMmaWarp = kProducerWarps + kEpilogueWarps;               // warp 12
constexpr int kColTile = 128;       // byte positions per tile (MMA M)
constexpr int kCodedPerItem = 16;   // coded packets per item (MMA N = 128 output bits)
constexpr int kMaxSrc = 128;        // N limit of this path (B resident: 8N x 128 bytes)
constexpr int kChunkSrc = 64;       // sources per A fill (128 TMEM columns)
constexpr int kTmemCols = 512;
constexpr int kABufCols = 128;
constexpr int kDCol0 = 256;         // D buffers at columns 256 and 384
constexpr uint32_t kOne = 0x38u;    // 1.0 in E4M3
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait

// shared memory layout (dynamic, 1024-aligned base)
constexpr int kBBytes = kMaxSrc * 8 * 128;  // 128 KB: B, 8 K-blocks of 16 KB
constexpr int kTabBytes = 256 * 8 * 8;      // 16 KB: 8x8 FP8 block of every coefficient
constexpr int kSmemBytes = kBBytes + kTabBytes + 1024 /*barriers etc*/ + 1024 /*alignment slack*/;

struct Ctl {
    unsigned long long a_full[2], a_empty[2], d_full[2], d_empty[2], drain;
    uint32_t tmem_base;
    int abort;
    long long item;
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
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
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

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

// byte offset of (row n, K byte k) inside B (K-major, 128B swizzle, K-blocks of 128 bytes)
__device__ __forceinline__ uint32_t b_offset(int n, int k)
{
    const int kb = k >> 7, kk = k & 127;
    return (uint32_t)(kb * (128 * 128) + (n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 4) ^ (n & 7)) << 4) | (kk & 15)));
}

// 8 FP8 values (bytes j = 0..7) of one source byte: 1.0 where bit j is set
__device__ __forceinline__ void spread_bits(uint32_t b, uint32_t &lo, uint32_t &hi)
{
    lo = (((b & 0xFu) * 0x00204081u) & 0x01010101u) * kOne;
    hi = ((((b >> 4) & 0xFu) * 0x00204081u) & 0x01010101u) * kOne;
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
            mbar_init(&ctl->d_empty[b], kEpilogueWarps * 32);
        }
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

    // per-role pipeline counters (every role walks the same sequence)
    uint32_t fills = 0, tiles = 0;

    for (;;) {
        if (tid == 0) ctl->item = (long long)atomicAdd(&ctr->next, 1ull);
        __syncthreads();
        const long long item = ctl->item;
        if (item >= total || *abort_flag) break;
        // locate the generation
        int lo = 0, hi = n_gens - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(tile_start + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const EncGen g = gens[lo];
        const int kc = (int)(item - __ldg(tile_start + lo));
        const int N = g.n_src, K = g.n_coded, ld = g.coef_ld;
        const unsigned long long len = g.len;
        const int k0 = kc * kCodedPerItem;
        const int nchunks = (N + kChunkSrc - 1) / kChunkSrc;
        const int ncols = (int)((len + kColTile - 1) / kColTile);
        const int kbytes = ((N + 15) / 16) * 128;  // B K extent, whole K-blocks

        // B: rows n = 8k'+r, K bytes 8i+j; zero outside the generation
        for (int e = tid; e < 128 * (kbytes / 16); e += blockDim.x) {
            const int n = e / (kbytes / 16);
            const int chunk = e - n * (kbytes / 16);  // 16-byte chunk = sources 2*chunk, 2*chunk+1
            const int kp = n >> 3, r = n & 7, k = k0 + kp;
            const int i0 = 2 * chunk, i1 = i0 + 1;
            unsigned long long v0 = 0, v1 = 0;
            if (k < K) {
                if (i0 < N) v0 = tab[__ldg(g.coef + (size_t)k * ld + i0) * 8 + r];
                if (i1 < N) v1 = tab[__ldg(g.coef + (size_t)k * ld + i1) * 8 + r];
            }
            uint4 q;
            q.x = (uint32_t)v0;
            q.y = (uint32_t)(v0 >> 32);
            q.z = (uint32_t)v1;
            q.w = (uint32_t)(v1 >> 32);
            *reinterpret_cast<uint4 *>(Bs + b_offset(n, 16 * chunk)) = q;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        if (warp < kProducerWarps) {
            // ---------------- producers: A = source bit planes -> TMEM ----------------
            const int half = warp >> 2;      // which 32 sources of a 64-source chunk
            const int lrow = (warp & 3) * 32;  // TMEM lane quarter
            const int pos = lrow + lane;       // byte position within the column tile
            for (int ct = 0; ct < ncols && !*abort_flag; ++ct) {
                const unsigned long long col = (unsigned long long)ct * kColTile + pos;
                const bool in = col < len;
                for (int ch = 0; ch < nchunks; ++ch) {
                    const uint32_t buf = fills & 1u, use = fills >> 1;
                    // gather this thread's 32 source bytes first (loads in flight together)
                    uint32_t bytes[32];
                    const int ibase = ch * kChunkSrc + half * 32;
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const int i = ibase + t;
                        bytes[t] = (in && i < N) ? (uint32_t)__ldg(g.src + (size_t)i * len + col) : 0u;
                    }
                    if (!mbar_wait_warp(&ctl->a_empty[buf], (use & 1u) ^ 1u, abort_flag)) {
                        ctl->abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t acol = tmem + ((uint32_t)lrow << 16) + buf * kABufCols + half * 64;
#pragma unroll
                    for (int grp = 0; grp < 4; ++grp) {
                        uint32_t v[16];
#pragma unroll
                        for (int t = 0; t < 8; ++t) spread_bits(bytes[grp * 8 + t], v[2 * t], v[2 * t + 1]);
                        tmem_st16(acol + grp * 16, v);
                    }
                    tmem_wait_st();
                    tc_fence_before();
                    mbar_arrive(&ctl->a_full[buf]);
                    ++fills;
                }
            }
        } else if (warp < kProducerWarps + kEpilogueWarps) {
            // ---------------- epilogue: D -> parity bytes -> global ----------------
            const int q = warp - kProducerWarps;  // TMEM lane quarter (warp % 4)
            const int pos = q * 32 + lane;
            for (int ct = 0; ct < ncols && !*abort_flag; ++ct) {
                const uint32_t buf = tiles & 1u, use = tiles >> 1;
                if (!mbar_wait_warp(&ctl->d_full[buf], use & 1u, abort_flag)) {
                    ctl->abort = 1;
                    break;
                }
                tc_fence_after();
                const unsigned long long col = (unsigned long long)ct * kColTile + pos;
                const uint32_t dcol = tmem + ((uint32_t)(q * 32) << 16) + kDCol0 + buf * 128;
                uint32_t outb[16];
#pragma unroll
                for (int grp = 0; grp < 8; ++grp) {
                    uint32_t v[16];
                    tmem_ld16(dcol + grp * 16, v);
                    tmem_wait_ld();
                    outb[2 * grp] = parity_byte(v);
                    outb[2 * grp + 1] = parity_byte(v + 8);
                }
                tc_fence_before();
                mbar_arrive(&ctl->d_empty[buf]);
                if (col < len) {
#pragma unroll
                    for (int kp = 0; kp < kCodedPerItem; ++kp)
                        if (k0 + kp < K) g.out[(size_t)(k0 + kp) * len + col] = (uint8_t)outb[kp];
                }
                ++tiles;
            }
        } else if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t b_base = smem_u32(Bs);
            for (int ct = 0; ct < ncols && !*abort_flag; ++ct) {
                const uint32_t dbuf = tiles & 1u, duse = tiles >> 1;
                if (!mbar_wait(&ctl->d_empty[dbuf], (duse & 1u) ^ 1u, abort_flag)) {
                    ctl->abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + kDCol0 + dbuf * 128;
                bool ok = true;
                for (int ch = 0; ch < nchunks; ++ch) {
                    const uint32_t buf = fills & 1u, use = fills >> 1;
                    if (!mbar_wait(&ctl->a_full[buf], use & 1u, abort_flag)) {
                        ctl->abort = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int nsrc = min(kChunkSrc, N - ch * kChunkSrc);
                    const int ksteps = (nsrc + 3) / 4;  // 4 sources = 32 FP8 per MMA
                    for (int s = 0; s < ksteps; ++s) {
                        const int kglob = ch * kChunkSrc * 8 + s * 32;  // byte offset in K
                        const uint32_t baddr = b_base + (uint32_t)((kglob >> 7) * (128 * 128) + (kglob & 127));
                        tc_mma(dt, tmem + buf * kABufCols + s * 8, b_desc(baddr), kIdesc,
                               (ch > 0 || s > 0) ? 1u : 0u);
                    }
                    tc_commit(&ctl->a_empty[buf]);
                    ++fills;
                }
                if (!ok) break;
                tc_commit(&ctl->d_full[dbuf]);
                ++tiles;
            }
        }
        __syncthreads();  // item done: D drained, B may be rewritten
    }

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
