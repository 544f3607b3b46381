"""Pins of the oracle's encode (Eq. 2) and Gauss-Jordan decode.

Encode is checked with identity and permutation matrices, linearity in the
coding matrix and composition (coding coded packets, i.e. recoding, equals
coding with the product matrix).  Decode is checked by round trips, by
rank-deficient cases worked out by hand, by brute-force rank on tiny
matrices (the row space is enumerated: |span| = q^rank) and by the
full-rank probability of random square matrices over GF(q),
prod_{i=1..N} (1 - q^-i) (the linear-dependence effect behind the paper's
remark on GF(2), cf. Cooper), within a binomial confidence bound.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import synth

FIELDS = (1, 2, 4, 8)


def _matmul(n, A, B):
    """Matrix product over GF(2^n) from the (axiom-pinned) scalar table."""
    T = oracle.mul_table(n)
    out = np.zeros((A.shape[0], B.shape[1]), dtype=np.uint8)
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            acc = 0
            for k in range(A.shape[1]):
                acc ^= int(T[A[i, k], B[k, j]])
            out[i, j] = acc
    return out


@pytest.mark.parametrize("n", FIELDS)
def test_encode_identity_and_permutation(n):
    g = synth.choice(10, n)
    src = synth.random_bytes(g, (6, 333))
    assert np.array_equal(oracle.encode(n, src, np.eye(6, dtype=np.uint8)), src)
    perm = g.permutation(6)
    P = np.eye(6, dtype=np.uint8)[perm]
    assert np.array_equal(oracle.encode(n, src, P), src[perm])


@pytest.mark.parametrize("n", FIELDS)
def test_encode_linear_in_coefficients(n):
    g = synth.choice(11, n)
    src = synth.random_bytes(g, (5, 200))
    B1 = synth.coefficients(g, n, (4, 5), nonzero=False)
    B2 = synth.coefficients(g, n, (4, 5), nonzero=False)
    assert np.array_equal(oracle.encode(n, src, B1 ^ B2),
                          oracle.encode(n, src, B1) ^ oracle.encode(n, src, B2))


@pytest.mark.parametrize("n", FIELDS)
def test_recoding_equals_product_matrix(n):
    g = synth.choice(12, n)
    src = synth.random_bytes(g, (5, 128))
    B1 = synth.coefficients(g, n, (7, 5), nonzero=False)
    B2 = synth.coefficients(g, n, (3, 7), nonzero=False)
    twice = oracle.encode(n, oracle.encode(n, src, B1), B2)
    assert np.array_equal(twice, oracle.encode(n, src, _matmul(n, B2, B1)))


@pytest.mark.parametrize("n", FIELDS)
def test_encode_single_row_is_sum_of_madds(n):
    g = synth.choice(13, n)
    src = synth.random_bytes(g, (9, 257))
    c = synth.coefficients(g, n, (1, 9), nonzero=False)
    acc = np.zeros(257, dtype=np.uint8)
    for i in range(9):
        acc = oracle.madd_imul(n, acc, src[i], int(c[0, i]))
    assert np.array_equal(oracle.encode(n, src, c)[0], acc)


@pytest.mark.parametrize("n", FIELDS)
def test_round_trip_single_generation(n):
    gen = synth.generation(n)
    coded = oracle.encode(n, gen.src, gen.coef_stream)
    out, solved, rank, used = oracle.decode(n, gen.coef_stream, coded)
    assert rank == 16 and solved.all()
    assert np.array_equal(out, gen.src)
    assert 16 <= used <= gen.coef_stream.shape[0]
    # rows after `used` are never needed
    out2, _, rank2, _ = oracle.decode(n, gen.coef_stream[:used], coded[:used])
    assert rank2 == 16 and np.array_equal(out2, gen.src)


def test_rank_deficient_by_hand():
    # GF(256): rows [1,1,0] and [0,0,5] span a 2-dim space of GF(256)^3;
    # only source 2 is determined (its row reduces to e_2).
    coef = np.array([[1, 1, 0], [0, 0, 5]], dtype=np.uint8)
    payload = np.array([[7, 9], [3, 4]], dtype=np.uint8)
    out, solved, rank, used = oracle.decode(8, coef, payload)
    assert rank == 2 and used == 2
    assert solved.tolist() == [False, False, True]
    inv5 = oracle.inv(8, 5)
    assert out[2].tolist() == [oracle.mul(8, inv5, 3), oracle.mul(8, inv5, 4)]
    assert out[0].tolist() == [0, 0] and out[1].tolist() == [0, 0]
    # a repeated row is not innovative
    coef = np.array([[2, 0], [2, 0], [0, 1]], dtype=np.uint8)
    payload = np.array([[2], [2], [9]], dtype=np.uint8)
    out, solved, rank, used = oracle.decode(8, coef, payload)
    assert rank == 2 and used == 3 and solved.all()
    assert out[:, 0].tolist() == [1, 9]


@pytest.mark.parametrize("n", FIELDS)
def test_used_counts_rows_until_rank_n(n):
    """The decoder stops once the rank reaches N: `used` is the position of
    the row that completed the rank, whatever follows it (rows by hand)."""
    # two unit rows complete the rank of a 2-source generation; the third row is never consumed
    coef = np.array([[1, 0], [0, 1], [1, 1]], dtype=np.uint8)
    payload = np.array([[5], [6], [0]], dtype=np.uint8)  # the last row is inconsistent on purpose
    out, solved, rank, used = oracle.decode(n, coef, payload)
    assert (rank, used) == (2, 2) and solved.all()
    assert out[:, 0].tolist() == [5, 6]  # unit rows: the payload bytes themselves, in every field
    # a repeated row in between is consumed but not innovative
    coef = np.array([[1, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.uint8)
    out, solved, rank, used = oracle.decode(n, coef, np.zeros((6, 0), dtype=np.uint8))
    assert (rank, used) == (3, 4)
    # a stream that never reaches rank N consumes every row
    coef = np.array([[1, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.uint8)
    out, solved, rank, used = oracle.decode(n, coef, np.zeros((3, 0), dtype=np.uint8))
    assert (rank, used) == (2, 3) and solved.tolist() == [False, False, True]


def _brute_rank(n, M):
    """log_q of the number of distinct vectors in the row space."""
    q = 1 << n
    T = oracle.mul_table(n)
    R, N = M.shape
    span = set()
    for combo in itertools.product(range(q), repeat=R):
        v = np.zeros(N, dtype=np.uint8)
        for r, c in enumerate(combo):
            v ^= T[c, M[r]]
        span.add(v.tobytes())
    return round(math.log(len(span), q))


@pytest.mark.parametrize("n", [1, 2])
def test_rank_matches_brute_force(n):
    g = synth.choice(14, n)
    for _ in range(60):
        R, N = int(g.integers(1, 5)), int(g.integers(1, 5))
        M = synth.coefficients(g, n, (R, N), nonzero=False)
        # make some rows dependent on purpose
        if R >= 2 and g.random() < 0.4:
            M[R - 1] = M[0]
        assert oracle.rank(n, M) == _brute_rank(n, M)


@pytest.mark.parametrize("n,N,trials", [(1, 8, 3000), (2, 6, 3000), (1, 3, 3000)])
def test_full_rank_probability(n, N, trials):
    q = 1 << n
    p = 1.0
    for i in range(1, N + 1):
        p *= 1.0 - q ** (-i)
    g = synth.choice(15, n, N)
    full = sum(oracle.rank(n, synth.coefficients(g, n, (N, N), nonzero=False)) == N
               for _ in range(trials))
    sigma = math.sqrt(trials * p * (1 - p))
    assert abs(full - trials * p) < 4.5 * sigma, (full, trials * p)


@pytest.mark.parametrize("n", FIELDS)
def test_uneven_generation_round_trip(n):
    batch = synth.uneven_batch(n_gens=3, n_min=4, n_max=20, len_min=10, len_max=300,
                               fields=(n,), index=n)
    for ge in batch.gens:
        coded = oracle.encode(n, ge.src, ge.coef_stream)
        keep = ~ge.erased
        out, solved, rank, used = oracle.decode(n, ge.coef_stream[keep], coded[keep])
        assert rank == ge.n_src and solved.all()
        assert np.array_equal(out, ge.src)


# ---------------------------------------------------------------------------
# recoding at an intermediate node (oracle.recode)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", FIELDS)
def test_recode_identity_mix_forwards_packets(n):
    g = synth.choice(20, n)
    coef = synth.coefficients(g, n, (6, 4), nonzero=False)
    pay = synth.random_bytes(g, (6, 99))
    c2, p2 = oracle.recode(n, coef, pay, np.eye(6, dtype=np.uint8))
    assert np.array_equal(c2, coef) and np.array_equal(p2, pay)


@pytest.mark.parametrize("n", FIELDS)
def test_recoded_packets_decode_to_the_sources(n):
    """Sources -> coded at the sender -> recoded at a relay -> decoded with the
    composed coding vectors: the relay's vectors must describe its packets in
    the original sources (a wrong composition fails the decode)."""
    g = synth.choice(21, n)
    N, L = 8, 300
    src = synth.random_bytes(g, (N, L))
    for attempt in range(20):
        C = synth.coefficients(g, n, (N + 6, N), nonzero=False)
        M = synth.coefficients(g, n, (N + 10, N + 6), nonzero=False)
        c2, p2 = oracle.recode(n, C, oracle.encode(n, src, C), M)
        if oracle.rank(n, c2) == N:
            break
    out, solved, rank, _ = oracle.decode(n, c2, p2)
    assert rank == N and solved.all()
    assert np.array_equal(out, src)


@pytest.mark.parametrize("n", FIELDS)
def test_recode_payload_is_encode_and_vectors_are_product(n):
    g = synth.choice(22, n)
    C = synth.coefficients(g, n, (5, 7), nonzero=False)
    pay = synth.random_bytes(g, (5, 64))
    M = synth.coefficients(g, n, (3, 5), nonzero=False)
    c2, p2 = oracle.recode(n, C, pay, M)
    assert np.array_equal(p2, oracle.encode(n, pay, M))
    assert np.array_equal(c2, _matmul(n, M, C))


def test_recode_gf2_is_xor_of_selected_rows():
    """GF(2): a mix row selects packets; the new packet and vector are the
    bitwise XOR of the selected ones (no field multiplication involved)."""
    g = synth.choice(23)
    C = synth.coefficients(g, 1, (9, 6), nonzero=False)
    pay = synth.random_bytes(g, (9, 50))
    M = synth.coefficients(g, 1, (4, 9), nonzero=False)
    c2, p2 = oracle.recode(1, C, pay, M)
    for k in range(4):
        sel = np.nonzero(M[k])[0]
        want_c = np.bitwise_xor.reduce(C[sel], axis=0) if sel.size else np.zeros(6, np.uint8)
        want_p = np.bitwise_xor.reduce(pay[sel], axis=0) if sel.size else np.zeros(50, np.uint8)
        assert np.array_equal(c2[k], want_c) and np.array_equal(p2[k], want_p)
