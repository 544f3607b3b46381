"""Pins of the oracle's region operations (madd b := b + c*a, section II).

The oracle's word-by-word region madd is compared with the paper's two
independent algorithms restated from section IV (shuffle: split nibble
tables, Algorithm 1; imul: masked bit planes times c*x^i with integer
multiplies, Algorithm 2), with the trivial cases of section IV (c = 0 is a
no-op, c = 1 a plain XOR), with GF(2) reducing to bitwise logic, and with
the linearity identities of a vector space over GF(q).
"""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import synth

FIELDS = (1, 2, 4, 8)


@pytest.mark.parametrize("n", FIELDS)
def test_madd_agrees_with_shuffle_and_imul_every_byte_every_coef(n):
    q = 1 << n
    src = np.arange(256, dtype=np.uint8)
    dst = synth.random_bytes(synth.choice(1, n), 256)
    for c in range(q):
        ref = oracle.region_madd(n, dst, src, c)
        assert np.array_equal(ref, oracle.madd_shuffle(n, dst, src, c)), c
        assert np.array_equal(ref, oracle.madd_imul(n, dst, src, c)), c


@pytest.mark.parametrize("n", FIELDS)
@pytest.mark.parametrize("length", [0, 1, 3, 4, 5, 15, 16, 17, 63, 64, 1000, 1500])
def test_madd_agrees_with_imul_ragged(n, length):
    g = synth.choice(2, n, length)
    src, dst = synth.random_bytes(g, length), synth.random_bytes(g, length)
    c = int(g.integers(0, 1 << n))
    assert np.array_equal(oracle.region_madd(n, dst, src, c), oracle.madd_imul(n, dst, src, c))


@pytest.mark.parametrize("n", FIELDS)
def test_trivial_coefficients(n):
    g = synth.choice(3, n)
    src, dst = synth.random_bytes(g, 777), synth.random_bytes(g, 777)
    assert np.array_equal(oracle.region_madd(n, dst, src, 0), dst)
    assert np.array_equal(oracle.region_madd(n, dst, src, 1), dst ^ src)
    assert np.array_equal(oracle.region_mul(n, src, 0), np.zeros_like(src))
    assert np.array_equal(oracle.region_mul(n, src, 1), src)


def test_gf2_is_bitwise():
    g = synth.choice(4)
    src, dst = synth.random_bytes(g, 4096), synth.random_bytes(g, 4096)
    # every bit is a word; c * bit = c AND bit
    for c in (0, 1):
        mask = np.uint8(0xFF if c else 0)
        assert np.array_equal(oracle.region_madd(1, dst, src, c), dst ^ (src & mask))


@pytest.mark.parametrize("n", [2, 4, 8])
def test_region_mul_applies_scalar_to_each_word(n):
    """Unpack every word, multiply with the (axiom-pinned) scalar product,
    repack: equals the region result."""
    g = synth.choice(5, n)
    src = synth.random_bytes(g, 512)
    mask = (1 << n) - 1
    for c in range(1, 1 << n, max(1, (1 << n) // 16)):
        res = oracle.region_mul(n, src, c)
        expect = np.zeros_like(src)
        for j in range(8 // n):
            words = (src >> (j * n)) & mask
            prod = np.array([oracle.mul(n, c, int(w)) for w in words], dtype=np.uint8)
            expect |= (prod << (j * n)).astype(np.uint8)
        assert np.array_equal(res, expect)


def _rotate_words(x: np.ndarray, n: int) -> np.ndarray:
    """Rotate the words of every byte by one word position."""
    return (((x.astype(np.uint16) << n) | (x.astype(np.uint16) >> (8 - n))) & 0xFF).astype(np.uint8)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_word_order_invariance(n):
    """Every word of a region is multiplied by the same c, so permuting words
    inside bytes commutes with the region operation."""
    g = synth.choice(6, n)
    src, dst = synth.random_bytes(g, 300), synth.random_bytes(g, 300)
    for c in range(1 << n):
        lhs = _rotate_words(oracle.region_madd(n, dst, src, c), n)
        rhs = oracle.region_madd(n, _rotate_words(dst, n), _rotate_words(src, n), c)
        assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("n", FIELDS)
def test_linearity(n):
    g = synth.choice(7, n)
    src, dst = synth.random_bytes(g, 999), synth.random_bytes(g, 999)
    q = 1 << n
    for _ in range(8):
        c1, c2 = int(g.integers(0, q)), int(g.integers(0, q))
        # madd(c1) then madd(c2) == madd(c1 + c2)
        two = oracle.region_madd(n, oracle.region_madd(n, dst, src, c1), src, c2)
        assert np.array_equal(two, oracle.region_madd(n, dst, src, c1 ^ c2))
        # mul(c2) o mul(c1) == mul(c1 * c2)
        assert np.array_equal(oracle.region_mul(n, oracle.region_mul(n, src, c1), c2),
                              oracle.region_mul(n, src, oracle.mul(n, c1, c2)))
        if c1:
            back = oracle.region_mul(n, oracle.region_mul(n, src, c1), oracle.inv(n, c1))
            assert np.array_equal(back, src)
