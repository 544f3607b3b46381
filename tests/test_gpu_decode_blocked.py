"""The blocked coefficient phase of the decode (generations of at least 64
sources: blocks of 64 arriving rows, each cleared of the stored pivots by a
row product on the batched encode, Gauss-Jordan within the block, then the
new pivots cleared from the stored rows by a second product) against the
oracle's progressive Gauss-Jordan: decoded packets, rank, rows consumed and
per-source flags, bit-exact, in every field; rank reached inside a block,
rank deficiency, repeated and zero rows, the widest rows the blocked phase
takes, and a batch mixing blocked and one-CTA generations."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import synth

import oracle_pool
from gpu_util import dev
from test_gpu_decode import _decode

pytestmark = pytest.mark.gpu
FIELDS = (1, 2, 4, 8)


def _expect(item):
    field, coef, payload = item
    return oracle.decode(field, coef, payload)


def _compare(items, got):
    refs = oracle_pool.pmap(_expect, items)
    for (field, coef, payload), (out, solved, rank, used), (r_out, r_solved, r_rank, r_used) in zip(items, got, refs):
        assert rank == r_rank and used == r_used, (field, coef.shape, rank, r_rank, used, r_used)
        assert np.array_equal(solved, r_solved)
        assert np.array_equal(out, r_out)


@pytest.mark.parametrize("field", FIELDS)
def test_blocked_shapes(field):
    dev()
    g = synth.choice(72, field)
    items = []
    for N, R, L in ((64, 64, 100), (64, 65, 7), (128, 130, 1), (200, 200, 333), (255, 320, 64), (255, 1793, 16),
                    (130, 64, 40), (300, 310, 128)):
        src = synth.random_bytes(g, (N, L))
        coef = synth.coefficients(g, field, (R, N), nonzero=False)
        items.append((field, coef, oracle.encode(field, src, coef)))
    _compare(items, _decode(items))


@pytest.mark.parametrize("field", [2, 8])
def test_blocked_degenerate_rows(field):
    """Repeated rows, zero rows and a dependent row inside and across blocks;
    rows arriving after rank N; too few rows for rank N."""
    dev()
    g = synth.choice(73, field)
    N, L = 140, 50
    src = synth.random_bytes(g, (N, L))
    coef = synth.coefficients(g, field, (230, N), nonzero=False)
    coef[10] = coef[3]          # repeated within block 0
    coef[70] = coef[5]          # repeated across blocks
    coef[71] = 0                # zero row
    coef[100] = coef[0] ^ coef[1] if field == 1 else oracle.region_madd(field, coef[0], coef[1], 1)
    coef[64:80] = coef[0:16]    # a run of repeats starting a block
    items = [(field, coef, oracle.encode(field, src, coef)),
             (field, coef[:120].copy(), oracle.encode(field, src, coef[:120]))]  # rank < N
    got = _decode(items)
    _compare(items, got)
    assert got[1][2] < N and got[0][2] == N


def test_blocked_and_one_cta_generations_in_one_call():
    dev()
    batch = synth.uneven_batch(n_gens=40, n_min=8, n_max=255, len_min=64, len_max=3000, index=74)
    items = []
    for ge in batch.gens:
        keep = ~ge.erased
        coef = np.ascontiguousarray(ge.coef_stream[keep])
        items.append((ge.field, coef, oracle.encode(ge.field, ge.src, coef)))
    assert any(c.shape[1] >= 64 for _, c, _ in items) and any(c.shape[1] < 64 for _, c, _ in items)
    got = _decode(items)
    _compare(items, got)
    for r, ge in zip(got, batch.gens):
        assert r[2] == ge.n_src and np.array_equal(r[0], ge.src)
