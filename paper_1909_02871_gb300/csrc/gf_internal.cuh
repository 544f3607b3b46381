// gf_internal.cuh -- device field arithmetic and host helpers shared by the
// CUDA translation units of the library (not part of the public ABI).
//
// Field GF(2^n), n in {1,2,4,8}, polynomial basis, reduction polynomials
// x^2+x+1, x^4+x+1, x^8+x^4+x^3+x^2+1 (section II of the paper names none;
// these are the library's reading).  A byte holds 8/n words.
//
// Multiplying every word of a byte by a constant c is a GF(2)-linear map of
// the byte's 8 bits.  The library represents it by the images of the 8 unit
// bytes (bit i set), e_i = c * x^(i mod n) placed in word i / n -- the
// "powers of c" that the imul algorithm multiplies bit planes with
// (section IV-B) -- and evaluates it four bytes at a time with the split
// nibble tables of the shuffle algorithm (section IV-A): PTX prmt plays the
// part of the byte shuffle.  prmt selects from 8 bytes, so each nibble
// lookup covers the nibble's low three bits (8 entries, two registers) and
// the nibble's top bit is added by linearity from a sign-replicated mask.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gf.h"

namespace gf {

// ------------------------------------------------------------------------
// scalar field arithmetic (device and host)
// ------------------------------------------------------------------------

__host__ __device__ constexpr uint32_t field_poly(int n)
{
    return n == 2 ? 0x7u : n == 4 ? 0x13u : n == 8 ? 0x11Du : 0x3u;
}

// v * x in GF(2^n), v < 2^n
__host__ __device__ constexpr uint32_t xtime(int n, uint32_t v)
{
    v <<= 1;
    if (v >> n) v ^= field_poly(n);
    return v;
}

// a * b in GF(2^n) by shift-and-add over the bits of b
__host__ __device__ constexpr uint32_t fmul(int n, uint32_t a, uint32_t b)
{
    uint32_t r = 0;
    for (int i = 0; i < n; ++i) {
        if ((b >> i) & 1u) r ^= a;
        a = xtime(n, a);
    }
    return r;
}

// a^-1 = a^(q-2) in GF(q) (0 maps to 0)
__host__ __device__ constexpr uint32_t finv(int n, uint32_t a)
{
    uint32_t q = 1u << n, r = 1, e = q - 2;
    if (a == 0) return 0;
    while (e) {
        if (e & 1u) r = fmul(n, r, a);
        a = fmul(n, a, a);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------------
// byte maps: multiplication of every word of a byte by c, 4 bytes at a time
// ------------------------------------------------------------------------

struct ByteMap {
    uint32_t lo0, lo1;  // images of the 8 values of bits 0..2, packed 4 per register
    uint32_t hi0, hi1;  // images of the 8 values of bits 4..6
    uint32_t k3, k7;    // images of bit 3 and bit 7, replicated in all 4 bytes
};

// Image of the unit byte (1 << i) under "multiply every word by c".
__host__ __device__ constexpr uint32_t unit_image(int n, uint32_t c, int i)
{
    const int word = i / n, bit = i % n;
    uint32_t v = c;
    for (int k = 0; k < bit; ++k) v = xtime(n, v);
    return (v << (word * n)) & 0xFFu;
}

__host__ __device__ constexpr ByteMap make_bytemap(int n, uint32_t c)
{
    uint32_t e[8] = {};
    for (int i = 0; i < 8; ++i) e[i] = unit_image(n, c, i);
    ByteMap m{};
    m.lo0 = (e[0] << 8) | (e[1] << 16) | ((e[0] ^ e[1]) << 24);
    m.lo1 = m.lo0 ^ (e[2] * 0x01010101u);
    m.hi0 = (e[4] << 8) | (e[5] << 16) | ((e[4] ^ e[5]) << 24);
    m.hi1 = m.hi0 ^ (e[6] * 0x01010101u);
    m.k3 = e[3] * 0x01010101u;
    m.k7 = e[7] * 0x01010101u;
    return m;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Per-word selectors, shared by every coefficient applied to the same word.
struct Sel {
    uint32_t lo, hi;  // prmt selectors: bits 0..2 / 4..6 of each byte, one nibble per byte
    uint32_t m3, m7;  // 0xFF in the bytes whose bit 3 / bit 7 is set
};

__device__ __forceinline__ Sel make_sel(uint32_t w)
{
    Sel s;
    const uint32_t l = w & 0x07070707u;
    const uint32_t h = (w >> 4) & 0x07070707u;
    s.lo = prmt(l | (l >> 4), 0u, 0x0020u);
    s.hi = prmt(h | (h >> 4), 0u, 0x0020u);
    s.m3 = prmt(w << 4, 0u, 0xBA98u);  // selector nibbles 8..B: replicate each byte's sign bit
    s.m7 = prmt(w, 0u, 0xBA98u);
    return s;
}

__device__ __forceinline__ uint32_t apply(const ByteMap &m, const Sel &s)
{
    uint32_t r = prmt(m.lo0, m.lo1, s.lo) ^ prmt(m.hi0, m.hi1, s.hi);
    r ^= s.m3 & m.k3;
    r ^= s.m7 & m.k7;
    return r;
}

__device__ __forceinline__ uint32_t apply_word(const ByteMap &m, uint32_t w)
{
    return apply(m, make_sel(w));
}

// Byte maps of every coefficient of every field, in shared memory:
// GF(2): 2 entries, GF(4): 4, GF(16): 16, GF(256): 256.
constexpr int kTableEntries = 2 + 4 + 16 + 256;

__host__ __device__ constexpr int table_base(int n)
{
    return n == 1 ? 0 : n == 2 ? 2 : n == 4 ? 6 : 22;
}

// The byte maps and inverses of every coefficient of every field, computed
// by the compiler (the kernels copy what they need into shared memory
// instead of deriving it per CTA: a 1024-thread CTA spent about 19,000
// clocks building 256 maps and inverses).  Entry table_base(n) + c.
struct FieldTables {
    ByteMap map[kTableEntries];
    uint32_t inv[kTableEntries];
};

__host__ __device__ constexpr FieldTables make_field_tables()
{
    FieldTables t{};
    const int fields[4] = {1, 2, 4, 8};
    for (int f = 0; f < 4; ++f) {
        const int n = fields[f];
        for (uint32_t c = 0; c < (1u << n); ++c) {
            t.map[table_base(n) + c] = make_bytemap(n, c);
            t.inv[table_base(n) + c] = finv(n, c);
        }
    }
    return t;
}

// every nonzero coefficient times its inverse is 1, in every field
__host__ __device__ constexpr bool field_tables_consistent(const FieldTables &t)
{
    const int fields[4] = {1, 2, 4, 8};
    for (int f = 0; f < 4; ++f) {
        const int n = fields[f];
        for (uint32_t c = 1; c < (1u << n); ++c)
            if (fmul(n, c, t.inv[table_base(n) + c]) != 1u) return false;
    }
    return true;
}

static __device__ const FieldTables g_field_tables = make_field_tables();
static_assert(field_tables_consistent(make_field_tables()), "field inverses");

// Fill `tab` (kTableEntries ByteMaps) cooperatively by the whole block.
__device__ __forceinline__ void fill_tables(ByteMap *tab)
{
    for (int e = threadIdx.x; e < kTableEntries; e += blockDim.x) tab[e] = g_field_tables.map[e];
}

// ------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------
inline bool field_ok(int n) { return n == 1 || n == 2 || n == 4 || n == 8; }

constexpr int kMaxDevices = 64;        // per-device tables of the host side

int sm_count();                        // SMs of the current device (cached)
int current_device();
int cuda_status(cudaError_t e);        // GF_OK or GF_ECUDA (clears sticky-free errors)

}  // namespace gf
