"""GPU parity of the batched Gauss-Jordan decode against the oracle's
progressive Gauss-Jordan: decoded packets, rank, rows consumed and the
per-source flags, bit-exact, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FIELDS = (1, 2, 4, 8)


def _decode(items):
    """items: list of (field, coef R x N, payload R x L) -> list of (out, solved, rank, used)."""
    keep, decs, res = [], [], []
    for field, coef, payload in items:
        R, N = coef.shape
        L = payload.shape[1]
        c = to_dev(coef.reshape(-1)) if coef.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        p = to_dev(payload.reshape(-1)) if payload.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        o = torch.full((max(N * L, 1),), 0x5A, dtype=torch.uint8, device=dev())
        rank = torch.full((1,), -7, dtype=torch.int32, device=dev())
        used = torch.full((1,), -7, dtype=torch.int32, device=dev())
        solved = torch.full((max(N, 1),), 9, dtype=torch.uint8, device=dev())
        keep += [c, p, o, rank, used, solved]
        decs.append((field, N, R, L, c, p, o, rank, used, solved))
        res.append((o, solved, rank, used, N, L))
    gf.gf_decode_batched(decs)
    torch.cuda.synchronize()
    return [(to_host(o)[:N * L].reshape(N, L), to_host(s)[:N].astype(bool), int(r.item()), int(u.item()))
            for o, s, r, u, N, L in res]


def _check(field, coef, payload, got):
    ref_out, ref_solved, ref_rank, ref_used = oracle.decode(field, coef, payload)
    out, solved, rank, used = got
    assert rank == ref_rank and used == ref_used
    assert np.array_equal(solved, ref_solved)
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("field", FIELDS)
def test_single_generation_round_trip(field):
    gen = synth.generation(field)
    coded = oracle.encode(field, gen.src, gen.coef_stream)
    (got,) = _decode([(field, gen.coef_stream, coded)])
    _check(field, gen.coef_stream, coded, got)
    assert got[2] == 16 and np.array_equal(got[0], gen.src)


@pytest.mark.parametrize("field", FIELDS)
def test_gpu_encode_then_gpu_decode(field):
    gen = synth.generation(field, index=5)
    K = gen.coef_stream.shape[0]
    src, coef = to_dev(gen.src), to_dev(gen.coef_stream)
    coded = torch.empty((K, gen.length), dtype=torch.uint8, device=dev())
    gf.gf_encode_batched([(field, 16, K, gen.length, src, coef, coded)])
    out = torch.empty_like(src)
    rank = torch.zeros(1, dtype=torch.int32, device=dev())
    gf.gf_decode_batched([(field, 16, K, gen.length, coef, coded, out, rank, None, None)])
    assert int(rank.item()) == 16
    assert np.array_equal(to_host(out), gen.src)


@pytest.mark.parametrize("field", FIELDS)
def test_rank_deficient_and_degenerate(field):
    g = synth.choice(70, field)
    q = 1 << field
    items = []
    # fewer rows than sources
    items.append((field, synth.coefficients(g, field, (5, 9), nonzero=False), synth.random_bytes(g, (5, 33))))
    # repeated and zero rows
    c = synth.coefficients(g, field, (8, 6), nonzero=False)
    c[3] = c[1]
    c[5] = 0
    items.append((field, c, synth.random_bytes(g, (8, 50))))
    # a row dependent on two others
    c = synth.coefficients(g, field, (7, 7), nonzero=False)
    if q > 2:
        c[6] = oracle.region_madd(field, c[0], c[1], 1 + int(g.integers(0, q - 1)))
    else:
        c[6] = c[0] ^ c[1]
    items.append((field, c, synth.random_bytes(g, (7, 19))))
    # empty cases
    items.append((field, np.zeros((0, 4), np.uint8), np.zeros((0, 10), np.uint8)))
    items.append((field, np.zeros((3, 0), np.uint8), np.zeros((3, 10), np.uint8)))
    items.append((field, synth.coefficients(g, field, (4, 4), nonzero=False), np.zeros((4, 0), np.uint8)))
    # identity and permutation
    items.append((field, np.eye(6, dtype=np.uint8)[g.permutation(6)], synth.random_bytes(g, (6, 77))))
    got = _decode(items)
    for (fld, coef, payload), r in zip(items, got):
        _check(fld, coef, payload, r)


def test_uneven_batch_one_call():
    batch = synth.uneven_batch(n_gens=24, n_min=8, n_max=64, len_min=64, len_max=2000, index=1)
    items = []
    for ge in batch.gens:
        coded = oracle.encode(ge.field, ge.src, ge.coef_stream)
        keep = ~ge.erased
        items.append((ge.field, ge.coef_stream[keep], coded[keep]))
    got = _decode(items)
    for (field, coef, payload), r, ge in zip(items, got, batch.gens):
        _check(field, coef, payload, r)
        assert r[2] == ge.n_src and np.array_equal(r[0], ge.src)


@pytest.mark.parametrize("field", [2, 8])
@pytest.mark.parametrize("N", [40, 63])
def test_rows_crossing_the_register_settling_width(field, N):
    """Rows of at most 32 words (N + rows so far <= 128 bytes) are settled by
    one warp in registers, wider ones block-wide: zero and repeated rows
    first keep the rank low while the rows grow past 128 bytes, so one
    generation takes both forms, in one launch with a generation that takes
    only the first."""
    g = synth.choice(72, field, N)
    src = synth.random_bytes(g, (N, 40))
    base = synth.coefficients(g, field, (6, N), nonzero=True)
    rows = [np.zeros((20, N), np.uint8), base[g.integers(0, 6, 70)],
            synth.coefficients(g, field, (N + 10, N), nonzero=False)]
    coef = np.ascontiguousarray(np.concatenate(rows))
    small = synth.coefficients(g, field, (12, 10), nonzero=True)
    items = [(field, coef, oracle.encode(field, src, coef)),
             (field, small, oracle.encode(field, synth.random_bytes(g, (10, 40)), small))]
    got = _decode(items)
    for (fld, c, payload), r in zip(items, got):
        _check(fld, c, payload, r)
    assert got[0][2] == N and np.array_equal(got[0][0], src)


@pytest.mark.parametrize("field", [1, 8])
@pytest.mark.parametrize("N,R", [(255, 300), (400, 420), (400, 1700)])
def test_large_generations(field, N, R):
    """N = 255 and N = 400 take the blocked coefficient phase; N = 400 with
    1700 rows (rows wider than the blocked phase takes) keeps the one-CTA
    elimination with its rows in global memory."""
    g = synth.choice(71, field, N)
    src = synth.random_bytes(g, (N, 32))
    coef = synth.coefficients(g, field, (R, N), nonzero=True)
    coded = oracle.encode(field, src, coef)
    (got,) = _decode([(field, coef, coded)])
    _check(field, coef, coded, got)


def test_decode_plan_and_check():
    gen = synth.generation(8, index=9)
    coded = oracle.encode(8, gen.src, gen.coef_stream)
    R = gen.coef_stream.shape[0]
    c, p = to_dev(gen.coef_stream), to_dev(coded)
    out = torch.zeros((16, gen.length), dtype=torch.uint8, device=dev())
    rank = torch.zeros(1, dtype=torch.int32, device=dev())
    decs = [(8, 16, R, gen.length, c, p, out, rank, None, None)]
    plan = gf.Plan.decode(decs)
    plan.launch()
    assert gf.gf_decode_check(decs) == gf.GF_OK
    assert np.array_equal(to_host(out), gen.src)
    # too few rows: rank-deficient
    decs2 = [(8, 16, 10, gen.length, c, p, out, rank, None, None)]
    gf.gf_decode_batched(decs2)
    assert gf.gf_decode_check(decs2) == gf.GF_ERANK
    plan.close()
