/*
 * gf_oracle.c -- plain, slow CPU oracle for GF(2^n) random linear network
 * coding (Guenther, Appel, Carle, "Galois Field Arithmetics for Linear Network
 * Coding using AVX 512 Instruction Set Extensions", arXiv:1909.02871).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness authority the CUDA
 * library is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the library never does.  It
 * shares no code, header, table or constant generator with the CUDA path:
 * every value here is computed from the definitions below, one element at a
 * time, with no blocking, fusion or reordering beyond what the paper states.
 *
 * Conventions, all from section II of the paper, with the readings taken
 * where the paper is silent:
 *   - the field is GF(q), q = 2^n, n in {1, 2, 4, 8}; a word of n bits is a
 *     polynomial over GF(2) whose bit i is the coefficient of x^i;
 *   - addition is bitwise XOR (section II, after Eq. 2);
 *   - multiplication is the polynomial product reduced by a field-specific
 *     polynomial (section II).  The paper names none; this oracle reads them
 *     as x^2+x+1 (GF(4)), x^4+x+1 (GF(16)) and x^8+x^4+x^3+x^2+1 (GF(256),
 *     the RAID-6 polynomial of Anvin's construction that the paper cites for
 *     the shuffle algorithm).  GF(2) needs no reduction (products have
 *     degree 0);
 *   - a packet of l bits holds l/n words (section II); a byte holds 8/n
 *     words, word j in bits [j*n, (j+1)*n) -- GF(16) words are nibbles;
 *   - coefficients are stored one field element per byte.
 *
 * Parity status: every function here is pinned by the CPU tests against
 * properties the paper and the mathematics fix (field axioms checked
 * exhaustively, multiplication by x as shift-and-reduce, the GF(4) field
 * derived by brute force from the axioms, the paper's two madd algorithms
 * restated independently, encode/decode round trips, brute-force rank on
 * tiny matrices and the full-rank probability of random matrices).  The
 * planted-mistake tests compile altered copies of this file (a wrong
 * polynomial, a dropped reduction step, a misplaced word, a transposed
 * matrix, a missing elimination step, ...) and check that each one fails
 * at least one of those pins.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Field definition (section II)                                       */
/* ------------------------------------------------------------------ */

/* Returns 1 if n names one of the four fields of section II. */
int gfo_field_ok(int n) { return n == 1 || n == 2 || n == 4 || n == 8; }

/* Reduction polynomial of GF(2^n), bit i = coefficient of x^i (reading). */
unsigned gfo_poly(int n)
{
    switch (n) {
    case 1: return 0x3;   /* x + 1: never used, products have degree 0 */
    case 2: return 0x7;   /* x^2 + x + 1 */
    case 4: return 0x13;  /* x^4 + x + 1 */
    case 8: return 0x11D; /* x^8 + x^4 + x^3 + x^2 + 1 */
    default: return 0;
    }
}

/* Product of two field elements: schoolbook carry-less multiplication of
 * the two polynomials, then reduction modulo gfo_poly(n) by long division
 * from degree 2n-2 down to degree n (section II). */
unsigned gfo_mul(int n, unsigned a, unsigned b)
{
    unsigned p = gfo_poly(n);
    unsigned prod = 0;
    int i, d;
    for (i = 0; i < n; i++)
        if ((b >> i) & 1u)
            prod ^= a << i;
    for (d = 2 * n - 2; d >= n; d--)
        if ((prod >> d) & 1u)
            prod ^= p << (d - n);
    return prod;
}

/* Multiplicative inverse by exhaustive search; 0 has none and maps to 0. */
unsigned gfo_inv(int n, unsigned a)
{
    unsigned q = 1u << n, b;
    if (a == 0)
        return 0;
    for (b = 1; b < q; b++)
        if (gfo_mul(n, a, b) == 1)
            return b;
    return 0;
}

/* Full multiplication table, out[a*q + b] = a*b. */
void gfo_mul_table(int n, uint8_t *out)
{
    unsigned q = 1u << n, a, b;
    for (a = 0; a < q; a++)
        for (b = 0; b < q; b++)
            out[a * q + b] = (uint8_t)gfo_mul(n, a, b);
}

/* ------------------------------------------------------------------ */
/* Region operations (section II, the madd operation b := b + c*a)     */
/* ------------------------------------------------------------------ */

/* dst := dst + c*src over GF(2^n), word by word. */
void gfo_region_madd(int n, uint8_t *dst, const uint8_t *src, unsigned c, size_t len)
{
    unsigned mask = (1u << n) - 1u;
    int words = 8 / n, j;
    size_t k;
    for (k = 0; k < len; k++) {
        unsigned byte = src[k], acc = dst[k];
        for (j = 0; j < words; j++) {
            unsigned w = (byte >> (j * n)) & mask;
            acc ^= gfo_mul(n, c, w) << (j * n);
        }
        dst[k] = (uint8_t)acc;
    }
}

/* dst := c*src over GF(2^n), word by word (dst may equal src). */
void gfo_region_mul(int n, uint8_t *dst, const uint8_t *src, unsigned c, size_t len)
{
    unsigned mask = (1u << n) - 1u;
    int words = 8 / n, j;
    size_t k;
    for (k = 0; k < len; k++) {
        unsigned byte = src[k], res = 0;
        for (j = 0; j < words; j++) {
            unsigned w = (byte >> (j * n)) & mask;
            res |= gfo_mul(n, c, w) << (j * n);
        }
        dst[k] = (uint8_t)res;
    }
}

/* The shuffle algorithm (section IV-A, Algorithm 1), restated on bytes:
 * each byte is split into its low and high nibble; tl[v] holds c times the
 * words packed in a low nibble v, th[v] c times the words of a high nibble v;
 * the product byte is tl[lo] ^ th[hi], XORed into dst.  Written here as an
 * independent route to the same madd, for the tests. */
void gfo_madd_shuffle(int n, uint8_t *dst, const uint8_t *src, unsigned c, size_t len)
{
    uint8_t tl[16], th[16];
    unsigned v;
    size_t k;
    for (v = 0; v < 16; v++) {
        uint8_t lo = (uint8_t)v, hi = (uint8_t)(v << 4);
        gfo_region_mul(n, &tl[v], &lo, c, 1);
        gfo_region_mul(n, &th[v], &hi, c, 1);
    }
    for (k = 0; k < len; k++)
        dst[k] ^= (uint8_t)(tl[src[k] & 15u] ^ th[src[k] >> 4]);
}

/* The imul algorithm (section IV-B, Algorithm 2), restated on 32-bit words:
 * for each bit position i of a word, mask bit i of every word, shift it down
 * to the word's lowest bit and multiply it (an ordinary integer product) by
 * p[i] = c * x^i; the words are n bits apart and p[i] < 2^n, so the partial
 * products never overlap and their XOR is c times every word.  The tail that
 * does not fill a 32-bit word is handled byte by byte the same way. */
void gfo_madd_imul(int n, uint8_t *dst, const uint8_t *src, unsigned c, size_t len)
{
    uint32_t p[8], low = 0;
    int i, j;
    size_t k;
    for (i = 0; i < n; i++)
        p[i] = gfo_mul(n, c, 1u << i);      /* c * x^i, reduced */
    for (j = 0; j < 32; j += n)
        low |= 1u << j;                      /* bit 0 of every word */
    for (k = 0; k + 4 <= len; k += 4) {
        uint32_t a = (uint32_t)src[k] | ((uint32_t)src[k + 1] << 8) |
                     ((uint32_t)src[k + 2] << 16) | ((uint32_t)src[k + 3] << 24);
        uint32_t r = 0;
        for (i = 0; i < n; i++)
            r ^= ((a & (low << i)) >> i) * p[i];
        dst[k] ^= (uint8_t)r;
        dst[k + 1] ^= (uint8_t)(r >> 8);
        dst[k + 2] ^= (uint8_t)(r >> 16);
        dst[k + 3] ^= (uint8_t)(r >> 24);
    }
    for (; k < len; k++) {
        uint32_t a = src[k], r = 0;
        for (i = 0; i < n; i++)
            r ^= ((a & ((low & 0xFFu) << i)) >> i) * p[i];
        dst[k] ^= (uint8_t)r;
    }
}

/* ------------------------------------------------------------------ */
/* Generation encode (section II, Eq. 1 and Eq. 2)                    */
/* ------------------------------------------------------------------ */

/* Encode K coded packets from the N source packets of one generation:
 * out_k = sum_i coef[k][i] * src_i (Eq. 2), each built in an accumulator
 * that starts at zero and receives one madd per source packet (the working
 * set of section V-A: N sources plus one accumulator). */
void gfo_encode(int n, int N, int K, size_t len, const uint8_t *src,
                const uint8_t *coef, uint8_t *out)
{
    int k, i;
    for (k = 0; k < K; k++) {
        uint8_t *acc = out + (size_t)k * len;
        memset(acc, 0, len);
        for (i = 0; i < N; i++)
            gfo_region_madd(n, acc, src + (size_t)i * len, coef[(size_t)k * N + i], len);
    }
}

/* ------------------------------------------------------------------ */
/* Decode: Gauss-Jordan elimination (not in the paper; reading)        */
/* ------------------------------------------------------------------ */

/* Progressive Gauss-Jordan decode of one generation over GF(2^n).
 *
 * Received rows arrive in order r = 0..R-1; row r is the augmented vector
 * [coef[r][0..N-1] | payload[r][0..len-1]].  For each arriving row:
 *   1. eliminate every existing pivot column from it (row -= f * pivot row);
 *   2. its pivot is its lowest-index nonzero coefficient; a row that reduced
 *      to zero is not innovative and is dropped;
 *   3. normalise it by the inverse of its pivot coefficient;
 *   4. eliminate its pivot column from every stored row (back-substitution).
 * Processing stops as soon as the rank reaches N (later rows are not needed).
 *
 * Outputs: out[p] (N rows of len bytes) is the decoded source p when the
 * stored row with pivot p has reduced to the unit vector e_p (solved[p] = 1);
 * otherwise out[p] is zero and solved[p] = 0.  *used receives the number of
 * received rows consumed.  Returns the rank, or -1 on allocation failure. */
int gfo_decode(int n, int N, int R, size_t len, const uint8_t *coef,
               const uint8_t *payload, uint8_t *out, uint8_t *solved, int *used)
{
    size_t width = (size_t)N + len;
    uint8_t *rows = (uint8_t *)malloc((size_t)(N > 0 ? N : 1) * (width > 0 ? width : 1));
    uint8_t *cur = (uint8_t *)malloc(width > 0 ? width : 1);
    int *row_of_pivot = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int rank = 0, r, s, p, col;
    if (!rows || !cur || !row_of_pivot) {
        free(rows); free(cur); free(row_of_pivot);
        return -1;
    }
    for (p = 0; p < N; p++)
        row_of_pivot[p] = -1;
    for (r = 0; r < R && rank < N; r++) {
        int pivot = -1;
        unsigned f;
        memcpy(cur, coef + (size_t)r * N, (size_t)N);
        if (len)
            memcpy(cur + N, payload + (size_t)r * len, len);
        /* 1. eliminate existing pivots */
        for (p = 0; p < N; p++) {
            s = row_of_pivot[p];
            if (s < 0 || cur[p] == 0)
                continue;
            f = cur[p];
            for (col = 0; col < N; col++)
                cur[col] ^= (uint8_t)gfo_mul(n, f, rows[(size_t)s * width + col]);
            gfo_region_madd(n, cur + N, rows + (size_t)s * width + N, f, len);
        }
        /* 2. pivot = lowest nonzero coefficient */
        for (col = 0; col < N; col++)
            if (cur[col] != 0) { pivot = col; break; }
        if (pivot < 0)
            continue;
        /* 3. normalise */
        f = gfo_inv(n, cur[pivot]);
        for (col = 0; col < N; col++)
            cur[col] = (uint8_t)gfo_mul(n, f, cur[col]);
        gfo_region_mul(n, cur + N, cur + N, f, len);
        /* 4. back-substitute into the stored rows */
        for (p = 0; p < N; p++) {
            uint8_t *row;
            s = row_of_pivot[p];
            if (s < 0)
                continue;
            row = rows + (size_t)s * width;
            f = row[pivot];
            if (f == 0)
                continue;
            for (col = 0; col < N; col++)
                row[col] ^= (uint8_t)gfo_mul(n, f, cur[col]);
            gfo_region_madd(n, row + N, cur + N, f, len);
        }
        memcpy(rows + (size_t)rank * width, cur, width);
        row_of_pivot[pivot] = rank;
        rank++;
    }
    if (used)
        *used = r;
    for (p = 0; p < N; p++) {
        int unit = 0;
        s = row_of_pivot[p];
        if (s >= 0) {
            unit = 1;
            for (col = 0; col < N; col++)
                if (rows[(size_t)s * width + col] != (col == p ? 1 : 0)) { unit = 0; break; }
        }
        if (len && unit)
            memcpy(out + (size_t)p * len, rows + (size_t)s * width + N, len);
        else if (len)
            memset(out + (size_t)p * len, 0, len);
        if (solved)
            solved[p] = (uint8_t)unit;
    }
    free(rows); free(cur); free(row_of_pivot);
    return rank;
}

/* Rank of an R x N coefficient matrix, by the same elimination with an empty
 * payload and no early stop. */
int gfo_rank(int n, int R, int N, const uint8_t *coef)
{
    uint8_t *out = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    uint8_t *solved = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    int used = 0, rank;
    if (!out || !solved) { free(out); free(solved); return -1; }
    rank = gfo_decode(n, N, R, 0, coef, NULL, out, solved, &used);
    free(out); free(solved);
    return rank;
}

/* ------------------------------------------------------------------ */
/* Recoding at an intermediate node (section II: a node forwards linear */
/* combinations of the packets it has received)                        */
/* ------------------------------------------------------------------ */

/* A node holding R coded packets (coding vectors coef_in, R x N; payloads
 * payload_in, R x len) sends K2 new ones, each a linear combination of the
 * packets it holds with fresh coefficients mix (K2 x R):
 *   payload_out_k = sum_r mix[k][r] * payload_in_r        (Eq. 2 again)
 *   coef_out_k[i] = sum_r mix[k][r] * coef_in[r][i]       (field products)
 * so that coef_out expresses the new packets in the original sources. */
void gfo_recode(int n, int N, int R, int K2, size_t len, const uint8_t *coef_in,
                const uint8_t *payload_in, const uint8_t *mix, uint8_t *coef_out,
                uint8_t *payload_out)
{
    int k, r, i;
    for (k = 0; k < K2; k++)
        for (i = 0; i < N; i++) {
            unsigned acc = 0;
            for (r = 0; r < R; r++)
                acc ^= gfo_mul(n, mix[(size_t)k * R + r], coef_in[(size_t)r * N + i]);
            coef_out[(size_t)k * N + i] = (uint8_t)acc;
        }
    gfo_encode(n, R, K2, len, payload_in, mix, payload_out);
}
