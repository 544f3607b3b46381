"""The bit-sliced formulation of Eq. 2, checked on the CPU against the oracle.

The tensor-core encode rests on the identity of section IV-B,
c * a = XOR_j a_j * (c * x^j): multiplication by c is a GF(2)-linear map, an
8 x 8 bit matrix on a byte (block-diagonal with n x n blocks for GF(2^n),
n < 8, since a byte holds 8/n words multiplied by the same c).  Eq. 2 then
becomes one binary matrix product whose integer sums are reduced mod 2, and
the kernel computes those sums in FP32 above a bias of 2^23, reading the
parity from the low mantissa bits.  These tests restate that arithmetic with
numpy (no CUDA) and compare it with the oracle's encode, so the formulation
itself is pinned independently of the kernel."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import synth

FIELDS = (1, 2, 4, 8)


def bit_matrix(n, c):
    """8 x 8 matrix over GF(2): entry [r][j] = bit r of the product byte when
    the input byte is the unit byte with bit j set (words of n bits)."""
    M = np.zeros((8, 8), dtype=np.int64)
    for j in range(8):
        word, bit = divmod(j, n)
        prod = oracle.mul(n, c, 1 << bit) << (word * n)  # c * x^bit, in the same word
        for r in range(8):
            M[r, j] = (prod >> r) & 1
    return M


def bits(a):
    """Bit planes of a byte array: shape (..., 8), plane j = bit j."""
    return (a[..., None] >> np.arange(8)) & 1


@pytest.mark.parametrize("n", FIELDS)
def test_bit_matrix_is_the_product(n):
    q = 1 << n
    for c in range(q):
        M = bit_matrix(n, c)
        for a in range(256):
            prod = oracle.region_mul(n, np.array([a], dtype=np.uint8), c)[0]
            assert np.array_equal((M @ bits(np.array(a))) % 2, bits(np.array(prod)))


@pytest.mark.parametrize("n", (1, 2, 4))
def test_small_fields_are_block_diagonal(n):
    for c in range(1 << n):
        M = bit_matrix(n, c)
        for r in range(8):
            for j in range(8):
                if r // n != j // n:
                    assert M[r, j] == 0


@pytest.mark.parametrize("n", FIELDS)
def test_encode_as_one_binary_matrix_product(n):
    g = synth.choice(31, n)
    N, K, L = 70, 37, 53  # more than one 64-source chunk, ragged everywhere
    src = synth.random_bytes(g, (N, L))
    coef = synth.coefficients(g, n, (K, N), nonzero=False)
    # A: (8N x L) source bit planes; B: (8K x 8N) block matrix of the coefficients' bit matrices
    A = bits(src).transpose(0, 2, 1).reshape(8 * N, L)
    B = np.zeros((8 * K, 8 * N), dtype=np.int64)
    mats = {c: bit_matrix(n, c) for c in range(1 << n)}
    for k in range(K):
        for i in range(N):
            B[8 * k:8 * k + 8, 8 * i:8 * i + 8] = mats[int(coef[k, i])]
    S = B @ A  # integer sums, at most 8N terms each
    assert S.max() <= 8 * N
    # the sums of the 64-source chunks, reduced separately and XORed, give the same parities
    chunks = [B[:, 8 * i0:8 * min(N, i0 + 64)] @ A[8 * i0:8 * min(N, i0 + 64)] for i0 in range(0, N, 64)]
    par = np.zeros_like(S)
    for part in chunks:
        par ^= part & 1
    assert np.array_equal(par, S & 1)
    out_bits = (S & 1).reshape(K, 8, L)
    out = (out_bits << np.arange(8)[None, :, None]).sum(axis=1).astype(np.uint8)
    assert np.array_equal(out, oracle.encode(n, src, coef))


def test_fp32_sums_above_the_bias_are_exact():
    """A 64-source chunk sums at most 512 products of 0/1 values; added to 2^23
    in FP32 in any order the result stays an integer below 2^24, so the low
    16 bits of its encoding are the sum and bit 0 is the parity."""
    g = synth.choice(32, 0)
    for _ in range(200):
        terms = g.integers(0, 2, size=512).astype(np.float32)
        order = g.permutation(512)
        acc = np.float32(2.0 ** 23)
        for t in terms[order]:
            acc = np.float32(acc + t)
        exact = int(terms.sum())
        low16 = int(np.array(acc, dtype=np.float32).view(np.uint32)) & 0xFFFF
        assert low16 == exact and (low16 & 1) == (exact & 1)
    # the largest chunk sum: every product 1
    acc = np.float32(2.0 ** 23)
    for _ in range(512):
        acc = np.float32(acc + np.float32(1.0))
    assert int(np.array(acc, dtype=np.float32).view(np.uint32)) & 0xFFFF == 512


def test_two_packets_per_fp32_column_are_exact():
    """Two coded packets share one FP32 accumulator column: the products of
    packet p's bit matrix are summed with weight 1 and those of packet p + 16
    with weight 2^10 (a block scale), above the 2^23 bias.  Each sum is at
    most 512 < 2^10, so the total stays an integer below 2^24 (exact in FP32
    whatever the order of the K = 64 partial sums), bit 0 is the parity of
    the first sum and bit 10 that of the second, both in the low 16 bits."""
    g = synth.choice(33, 0)
    for trial in range(300):
        lo = g.integers(0, 2, size=512)
        hi = g.integers(0, 2, size=512)
        if trial == 0:
            lo[:] = 1
            hi[:] = 1
        # one partial sum per K = 64 MMA, weight 1 for the first eight, 2^10 for the next eight
        parts = [np.float32(lo[64 * s:64 * s + 64].sum()) for s in range(8)]
        parts += [np.float32(1024.0) * np.float32(hi[64 * s:64 * s + 64].sum()) for s in range(8)]
        acc = np.float32(2.0 ** 23)
        for s in g.permutation(16):
            acc = np.float32(acc + parts[s])
        word = int(np.array(acc, dtype=np.float32).view(np.uint32))
        assert word - 0x4B000000 == int(lo.sum()) + 1024 * int(hi.sum())
        assert (word & 1) == (lo.sum() & 1) and ((word >> 10) & 1) == (hi.sum() & 1)
        assert ((word & 0xFFFF) >> 10) & 1 == (hi.sum() & 1)


@pytest.mark.parametrize("n", FIELDS)
def test_encode_with_two_packets_per_column(n):
    """Eq. 2 for a pass of 32 coded packets computed as 128 accumulator
    columns (column 8p + r: bit r of packets p and p + 16), each the FP32
    value 2^23 + S_lo + 2^10 S_hi, with the parities read from bits 0 and 10;
    64-source chunks XORed as the kernel does."""
    g = synth.choice(34, n)
    N, K, L = 100, 29, 41  # two source chunks, a pass with 13 packets in its second 16
    src = synth.random_bytes(g, (N, L))
    coef = synth.coefficients(g, n, (K, N), nonzero=False)
    mats = {c: bit_matrix(n, c) for c in range(1 << n)}
    A = bits(src).transpose(0, 2, 1).reshape(8 * N, L)
    out_bits = np.zeros((32, 8, L), dtype=np.int64)
    for i0 in range(0, N, 64):
        i1 = min(N, i0 + 64)
        Ac = A[8 * i0:8 * i1]
        B = np.zeros((2, 128, 8 * (i1 - i0)), dtype=np.int64)  # [lo/hi][column][K]
        for kp in range(32):
            if kp >= K:
                continue
            half, slot = divmod(kp, 16)
            for i in range(i0, i1):
                B[half, 8 * slot:8 * slot + 8, 8 * (i - i0):8 * (i - i0) + 8] = mats[int(coef[kp, i])]
        D = (np.float32(2.0 ** 23) + (B[0] @ Ac).astype(np.float32)
             + np.float32(1024.0) * (B[1] @ Ac).astype(np.float32)).astype(np.float32)
        word = D.view(np.uint32).astype(np.int64) & 0xFFFF
        for kp in range(32):
            half, slot = divmod(kp, 16)
            out_bits[kp] ^= (word[8 * slot:8 * slot + 8] >> (10 * half)) & 1
    out = (out_bits[:K] << np.arange(8)[None, :, None]).sum(axis=1).astype(np.uint8)
    assert np.array_equal(out, oracle.encode(n, src, coef))


def test_permuted_bit_order_of_the_kernel():
    """The kernel orders the 8 bits of a source byte as (0, 4, 1, 5, 2, 6, 3, 7)
    along K, on both sides: the source side spreads a byte with two halving
    steps, the coefficient side keeps the unit images p_j (the image of the
    unit byte with bit j set) as two nibble planes (nibble t of Z.x / Z.y is
    the low / high nibble of p_(t%2*4 + t/2)) and builds row r of a block
    with one shift and one mask.  Restated here bit for bit, the nibble-wise
    dot product of row r with the spread byte a has the parity of bit r of
    c*a, for every coefficient, byte and field."""
    order = [0, 4, 1, 5, 2, 6, 3, 7]

    def spread(b):
        x = (b | (b << 14)) & 0x00330033
        x = (x | (x << 7)) & 0x11111111
        return (x << 1) & 0xFFFFFFFF

    def planes(imgs):
        zx = zy = 0
        for t in range(8):
            p = imgs[(t & 1) * 4 + (t >> 1)]
            zx |= (p & 0xF) << (4 * t)
            zy |= (p >> 4) << (4 * t)
        return zx, zy

    def block_row(zx, zy, r):
        return (((zx if r < 4 else zy) >> (r & 3)) & 0x11111111) << 1

    for b in range(256):
        w = spread(b)
        for k in range(8):
            assert ((w >> (4 * k)) & 0xF) == (2 if (b >> order[k]) & 1 else 0)
    for n in FIELDS:
        for c in range(1 << n):
            imgs = [int(oracle.region_mul(n, np.array([1 << j], np.uint8), c)[0]) for j in range(8)]
            zx, zy = planes(imgs)
            rows = [block_row(zx, zy, r) for r in range(8)]
            for a in range(256):
                wa = spread(a)
                prod = int(oracle.region_mul(n, np.array([a], np.uint8), c)[0])
                for r in range(8):
                    dot = sum(((rows[r] >> (4 * k)) & 0xF) * ((wa >> (4 * k)) & 0xF) for k in range(8)) // 4
                    assert dot % 2 == (prod >> r) & 1, (n, c, a, r)


def test_quad_byte_transpose_of_the_epilogue():
    """The epilogue stores rows of 4-byte aligned words after a byte
    transpose within each quad of lanes: lane j of a quad starts with byte t
    of its word = packet t at position j, exchanges with lane j^1 (byte
    selectors 0x6240 / 0x3715 for even / odd lanes) and then with lane j^2
    (0x5410 / 0x3276), and ends with byte i = packet j at position i.
    Restated with prmt's byte selection, for random words."""
    def prmt(a, b, sel):
        pool = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
        return sum(pool[(sel >> (4 * i)) & 7] << (8 * i) for i in range(4))

    g = np.random.default_rng(5)
    for _ in range(200):
        m = g.integers(0, 256, (4, 32))                       # m[packet][position]
        w = [sum(int(m[t][j]) << (8 * t) for t in range(4)) for j in range(32)]
        z = [prmt(w[j], w[j ^ 1], 0x3715 if j & 1 else 0x6240) for j in range(32)]
        v = [prmt(z[j], z[j ^ 2], 0x3276 if j & 2 else 0x5410) for j in range(32)]
        for j in range(32):
            q, jj = j >> 2, j & 3
            assert v[j] == sum(int(m[jj][4 * q + i]) << (8 * i) for i in range(4))
