// gf_region.cu -- region multiply-accumulate / multiply over GF(2^n)
// (the madd operation of section II; Algorithms 1 and 2 of section IV are
// its CPU SIMD forms).
//
// The hot loop is HBM-bound: madd moves 3 bytes per region byte (read src,
// read dst, write dst), mul 2.  Each thread streams 16-byte vectors, UNROLL
// of them in flight, and maps every 4-byte word through the coefficient's
// split tables held in registers (gf::ByteMap, ~17 integer ops per word).
// Trivial coefficients (section IV: c = 0, c = 1) become no-op / XOR / copy /
// zero fill without table lookups.
#include "gf_internal.cuh"

namespace gf {

enum RegionOp { OP_MADD = 0, OP_MUL = 1, OP_XOR = 2, OP_COPY = 3, OP_ZERO = 4 };

template <int OP>
__device__ __forceinline__ uint32_t op_word(const ByteMap &m, uint32_t s, uint32_t d)
{
    if (OP == OP_MADD) return d ^ apply_word(m, s);
    if (OP == OP_MUL) return apply_word(m, s);
    if (OP == OP_XOR) return d ^ s;
    if (OP == OP_COPY) return s;
    return 0u;
}

template <int OP>
__device__ __forceinline__ void op_byte(const ByteMap &m, uint8_t *dst, const uint8_t *src, size_t i)
{
    const uint32_t s = (OP == OP_ZERO) ? 0u : src[i];
    const uint32_t d = (OP == OP_MADD || OP == OP_XOR) ? dst[i] : 0u;
    dst[i] = (uint8_t)op_word<OP>(m, s, d);
}

constexpr int kRegionThreads = 256;
constexpr int kUnroll = 4;

// dst and src share their alignment modulo 16: bytes [0, head) and
// [head + 16*n16, len) go byte by byte (global threads 0..31), the rest as
// 16-byte vectors.
template <int OP>
__global__ void __launch_bounds__(kRegionThreads)
region_vec_kernel(uint8_t *dst, const uint8_t *src, size_t len, size_t head, size_t n16,
                  int field, uint32_t c)
{
    const ByteMap m = make_bytemap(field, c);
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;

    if (tid < 32) {
        for (size_t i = tid; i < head; i += 32) op_byte<OP>(m, dst, src, i);
        for (size_t i = head + 16 * n16 + tid; i < len; i += 32) op_byte<OP>(m, dst, src, i);
    }

    uint4 *dv = reinterpret_cast<uint4 *>(dst + head);
    const uint4 *sv = reinterpret_cast<const uint4 *>(src + head);
    for (size_t base = tid; base < n16; base += nthreads * kUnroll) {
        uint4 s[kUnroll], d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t i = base + (size_t)u * nthreads;
            if (i < n16) {
                if (OP != OP_ZERO) s[u] = sv[i];
                if (OP == OP_MADD || OP == OP_XOR) d[u] = dv[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t i = base + (size_t)u * nthreads;
            if (i < n16) {
                uint4 r;
                r.x = op_word<OP>(m, s[u].x, d[u].x);
                r.y = op_word<OP>(m, s[u].y, d[u].y);
                r.z = op_word<OP>(m, s[u].z, d[u].z);
                r.w = op_word<OP>(m, s[u].w, d[u].w);
                dv[i] = r;
            }
        }
    }
}

// dst and src differ in alignment modulo 16.  dst is walked in aligned
// 4-byte words; each source word is assembled from the two aligned source
// words it straddles (funnel shift).  The unaligned head of dst and the last
// word plus tail go byte by byte, so no load leaves the source region.
template <int OP>
__global__ void __launch_bounds__(kRegionThreads)
region_word_kernel(uint8_t *dst, const uint8_t *src, size_t len, size_t head, size_t nwords,
                   int field, uint32_t c)
{
    const ByteMap m = make_bytemap(field, c);
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;

    if (tid < 32) {
        for (size_t i = tid; i < head; i += 32) op_byte<OP>(m, dst, src, i);
        for (size_t i = head + 4 * nwords + tid; i < len; i += 32) op_byte<OP>(m, dst, src, i);
    }

    uint32_t *dw = reinterpret_cast<uint32_t *>(dst + head);
    const uint8_t *s0 = src + head;
    const uint32_t shift = (uint32_t)((uintptr_t)s0 & 3u) * 8u;
    const uint32_t *sw = reinterpret_cast<const uint32_t *>((uintptr_t)s0 & ~(uintptr_t)3);
    for (size_t base = tid; base < nwords; base += nthreads * kUnroll) {
        uint32_t s[kUnroll], d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t i = base + (size_t)u * nthreads;
            if (i < nwords) {
                if (OP != OP_ZERO) {
                    if (shift == 0) s[u] = sw[i];
                    else s[u] = __funnelshift_r(sw[i], sw[i + 1], shift);
                }
                if (OP == OP_MADD || OP == OP_XOR) d[u] = dw[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t i = base + (size_t)u * nthreads;
            if (i < nwords) dw[i] = op_word<OP>(m, s[u], d[u]);
        }
    }
}

template <int OP>
static int launch_region(uint8_t *dst, const uint8_t *src, size_t len, int field, uint32_t c,
                         cudaStream_t stream)
{
    // up to 256 blocks per SM (about two vectors per thread for a 1 GiB region): with 8 per SM each
    // thread strode through the region some 50 times and mul reached 0.85-0.92 of the measured
    // copy bandwidth; with 256 madd and mul reach 1.01-1.05 of it
    const size_t max_blocks = (size_t)sm_count() * 256;
    const uintptr_t da = (uintptr_t)dst, sa = (uintptr_t)src;
    if (OP == OP_ZERO || ((da ^ sa) & 15u) == 0) {
        size_t head = (16 - (da & 15u)) & 15u;
        if (head > len) head = len;
        const size_t n16 = (len - head) / 16;
        size_t blocks = (n16 + (size_t)kRegionThreads * kUnroll - 1) / ((size_t)kRegionThreads * kUnroll);
        if (blocks < 1) blocks = 1;
        if (blocks > max_blocks) blocks = max_blocks;
        region_vec_kernel<OP><<<(unsigned)blocks, kRegionThreads, 0, stream>>>(dst, src, len, head, n16,
                                                                                 field, c);
    } else {
        size_t head = (4 - (da & 3u)) & 3u;
        if (head > len) head = len;
        // keep the last full word out of the funnel path: its second source
        // word could lie past the end of the source region
        size_t nwords = (len - head) / 4;
        if (nwords > 0) nwords -= 1;
        size_t blocks = (nwords + (size_t)kRegionThreads * kUnroll - 1) / ((size_t)kRegionThreads * kUnroll);
        if (blocks < 1) blocks = 1;
        if (blocks > max_blocks) blocks = max_blocks;
        region_word_kernel<OP><<<(unsigned)blocks, kRegionThreads, 0, stream>>>(dst, src, len, head,
                                                                                  nwords, field, c);
    }
    return cuda_status(cudaGetLastError());
}

static int check_region(int field, uint8_t *dst, const uint8_t *src, uint32_t coef, size_t len)
{
    if (!field_ok(field) || coef >= (1u << field)) return GF_EINVAL;
    if (len == 0) return GF_OK;
    if (!dst || !src) return GF_EINVAL;
    const uintptr_t d = (uintptr_t)dst, s = (uintptr_t)src;
    if (d != s && d < s + len && s < d + len) return GF_EOVERLAP;
    return GF_OK;
}

}  // namespace gf

using namespace gf;

extern "C" int gf_region_madd(int field, uint8_t *dst, const uint8_t *src, uint8_t coef, size_t len,
                              gf_stream_t stream)
{
    int st = check_region(field, dst, src, coef, len);
    if (st != GF_OK || len == 0 || coef == 0) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (coef == 1) return launch_region<OP_XOR>(dst, src, len, field, 1, s);
    return launch_region<OP_MADD>(dst, src, len, field, coef, s);
}

extern "C" int gf_region_mul(int field, uint8_t *dst, const uint8_t *src, uint8_t coef, size_t len,
                             gf_stream_t stream)
{
    int st = check_region(field, dst, src, coef, len);
    if (st != GF_OK || len == 0) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (coef == 0) return launch_region<OP_ZERO>(dst, src, len, field, 0, s);
    if (coef == 1) {
        if (dst == src) return GF_OK;
        return launch_region<OP_COPY>(dst, src, len, field, 1, s);
    }
    return launch_region<OP_MUL>(dst, src, len, field, coef, s);
}
