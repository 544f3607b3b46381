"""Pins of the oracle's field arithmetic (section II of the paper).

The oracle multiplies by schoolbook carry-less product plus long-division
reduction.  These tests check it against facts that do not come from that
code: the field axioms over every pair/triple, multiplication by x as
shift-and-reduce (which, with distributivity and associativity, determines
the whole multiplication), GF(4) derived by brute force from the axioms
alone, and hand-derived powers of x from the textbook tables.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
READING_POLY = {2: 0x7, 4: 0x13, 8: 0x11D}


def _golden_ints(name):
    vals, extra = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].isdigit():
                vals.extend(int(p) for p in parts)
            else:
                extra[parts[0]] = int(parts[1])
    return vals, extra


def test_reading_polynomials():
    for n, p in READING_POLY.items():
        assert oracle.poly(n) == p


def test_gf2_is_and():
    for a, b in itertools.product(range(2), repeat=2):
        assert oracle.mul(1, a, b) == (a & b)


def test_gf4_is_the_unique_field_from_axioms():
    """Enumerate every commutative table on {0,1,2,3} with 0 absorbing and 1
    neutral (entries 2*2, 2*3, 3*3 free: 64 candidates); exactly one of them
    makes ({0..3}, XOR, *) a field, and it must be the oracle's."""
    survivors = []
    for t22, t23, t33 in itertools.product(range(4), repeat=3):
        T = np.zeros((4, 4), dtype=np.int64)
        T[1, :] = T[:, 1] = np.arange(4)
        T[0, :] = T[:, 0] = 0
        T[2, 2], T[2, 3], T[3, 2], T[3, 3] = t22, t23, t23, t33
        ok = True
        for a, b, c in itertools.product(range(4), repeat=3):
            if T[a, T[b, c]] != T[T[a, b], c] or T[a, b ^ c] != (T[a, b] ^ T[a, c]):
                ok = False
                break
        if ok and all(any(T[a, b] == 1 for b in range(4)) for a in range(1, 4)):
            survivors.append(T)
    assert len(survivors) == 1
    assert np.array_equal(survivors[0], oracle.mul_table(2).astype(np.int64))


@pytest.mark.parametrize("n", [2, 4, 8])
def test_mul_by_x_is_shift_and_reduce(n):
    """x * a = (a << 1) reduced once by the field polynomial."""
    q = 1 << n
    for a in range(q):
        expect = a << 1
        if expect & q:
            expect ^= READING_POLY[n]
        assert oracle.mul(n, 2, a) == expect


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_field_axioms_exhaustive(n):
    q = 1 << n
    T = oracle.mul_table(n).astype(np.int64)
    a = np.arange(q)
    # identities
    assert np.array_equal(T[0], np.zeros(q)) and np.array_equal(T[:, 0], np.zeros(q))
    assert np.array_equal(T[1], a) and np.array_equal(T[:, 1], a)
    # commutativity (all pairs)
    assert np.array_equal(T, T.T)
    # nonzero rows form a Latin square (no zero divisors, every product reachable)
    for x in range(1, q):
        assert sorted(T[x, 1:].tolist()) == list(range(1, q))
    # associativity and distributivity over XOR, all triples
    A, B, C = np.meshgrid(a, a, a, indexing="ij")
    assert np.array_equal(T[T[A, B], C], T[A, T[B, C]])
    assert np.array_equal(T[A, B ^ C], T[A, B] ^ T[A, C])


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_inverse_unique(n):
    q = 1 << n
    T = oracle.mul_table(n)
    for x in range(1, q):
        inverses = [y for y in range(1, q) if T[x, y] == 1]
        assert len(inverses) == 1
        assert oracle.inv(n, x) == inverses[0]
    assert oracle.inv(n, 0) == 0


@pytest.mark.parametrize("n", [2, 4, 8])
def test_x_is_primitive(n):
    """The reading polynomials are primitive: x has order 2^n - 1."""
    q = 1 << n
    v, order = 2, 1
    while v != 1:
        v = oracle.mul(n, v, 2)
        order += 1
        assert order < q
    assert order == q - 1


@pytest.mark.parametrize("n", [2, 4, 8])
def test_frobenius_is_additive(n):
    """(a + b)^2 = a^2 + b^2 in characteristic 2."""
    q = 1 << n
    for a in range(q):
        for b in range(0, q, max(1, q // 32)):
            s = a ^ b
            assert oracle.mul(n, s, s) == oracle.mul(n, a, a) ^ oracle.mul(n, b, b)


def test_gf16_powers_golden():
    vals, _ = _golden_ints("gf16_powers_of_x.txt")
    v = 1
    for i, expect in enumerate(vals):
        assert v == expect, f"x^{i}"
        v = oracle.mul(4, v, 2)


def test_gf256_powers_golden():
    vals, extra = _golden_ints("gf256_powers_of_x.txt")
    v = 1
    for i, expect in enumerate(vals):
        assert v == expect, f"x^{i}"
        v = oracle.mul(8, v, 2)
    assert oracle.inv(8, 2) == extra["inverse_of_x"]
    assert oracle.mul(8, 0x80, 0x02) == 0x1D
    assert oracle.mul(4, 0x8, 0x2) == 0x3
