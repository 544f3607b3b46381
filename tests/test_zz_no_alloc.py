"""gf_decode_noalloc: the decode entry point for callers that cannot let a
call allocate device memory (a packet data path that must not wait on the
CUDA allocator, or a process whose device memory all belongs to its own
pool); its scratch is a fixed device array inside the library.  Checked
through the C ABI against the oracle's Gauss-Jordan decode and against
gf_decode_batched, bit-exact (the tolerance of every decode test), on calls
in a row that share the array, at its documented size limit, just past it,
and on empty inputs.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _case(field, n_src, n_recv, length, index):
    g = synth.choice(90, field, n_src, n_recv, length, index)
    src = synth.random_bytes(g, (n_src, length))
    coef = synth.coefficients(g, field, (n_recv, n_src), nonzero=False)
    payload = oracle.encode(field, src, coef)
    return src, coef, payload


def _outputs(n_src, length):
    return (torch.full((max(n_src * length, 1),), 0x77, dtype=torch.uint8, device=dev()),
            torch.full((1,), -3, dtype=torch.int32, device=dev()),
            torch.full((1,), -3, dtype=torch.int32, device=dev()),
            torch.full((max(n_src, 1),), 9, dtype=torch.uint8, device=dev()))


def _inputs(coef, payload):
    c = to_dev(coef.reshape(-1)) if coef.size else torch.zeros(1, dtype=torch.uint8, device=dev())
    p = to_dev(payload.reshape(-1)) if payload.size else torch.zeros(1, dtype=torch.uint8, device=dev())
    return c, p


def _batched(field, N, R, L, coef, payload):
    c, p = _inputs(coef, payload)
    out, rank, used, solved = _outputs(N, L)
    gf.gf_decode_batched([(field, N, R, L, c, p, out, rank, used, solved)])
    torch.cuda.synchronize()
    return to_host(out)[:N * L], int(rank.item()), int(used.item()), to_host(solved)[:N]


def _expect(field, coef, payload, N, L):
    out, solved, rank, used = oracle.decode(field, coef.reshape(-1, N) if N else coef, payload.reshape(-1, L)
                                            if L else payload, n_src=N if N else None)
    return out.reshape(-1), rank, used, solved.astype(np.uint8)


def _same(got, want):
    return (np.array_equal(got[0], want[0]) and got[1] == want[1] and got[2] == want[2]
            and np.array_equal(got[3], want[3]))


def test_noalloc_matches_oracle_two_calls_in_a_row():
    # the second and third calls reuse the array the first one filled
    cases = [(8, 40, 47, 1500, 0), (4, 17, 17, 333, 1), (2, 9, 30, 64, 2)]
    keep, expect = [], []
    for field, N, R, L, idx in cases:
        src, coef, payload = _case(field, N, R, L, idx)
        want = _expect(field, coef, payload, N, L)
        assert _same(_batched(field, N, R, L, coef, payload), want)
        expect.append(want)
        keep.append((field, N, R, L, *_inputs(coef, payload), *_outputs(N, L)))
    for field, N, R, L, c, p, out, rank, used, solved in keep:
        assert gf.gf_decode_noalloc(field, N, R, L, c, p, out, rank, used, solved) == gf.GF_OK
    torch.cuda.synchronize()
    for (field, N, R, L, c, p, out, rank, used, solved), want in zip(keep, expect):
        got = (to_host(out)[:N * L], int(rank.item()), int(used.item()), to_host(solved)[:N])
        assert _same(got, want), (field, N, R, L)
    # the first case decodes its sources completely
    assert expect[0][1] == 40


def test_noalloc_at_its_documented_limit():
    """n_src = 255 with n_recv = 560 (GF(256)): the largest case the header
    names; its elimination rows need the opt-in shared memory."""
    field, N, R, L = 8, 255, 560, 96
    src, coef, payload = _case(field, N, R, L, 3)
    want = _expect(field, coef, payload, N, L)
    assert want[1] == N and np.array_equal(want[0], src.reshape(-1))
    c, p = _inputs(coef, payload)
    for _ in range(2):
        out, rank, used, solved = _outputs(N, L)
        assert gf.gf_decode_noalloc(field, N, R, L, c, p, out, rank, used, solved) == gf.GF_OK
        torch.cuda.synchronize()
        got = (to_host(out)[:N * L], int(rank.item()), int(used.item()), to_host(solved)[:N])
        assert _same(got, want)


def test_noalloc_empty_inputs_match_batched():
    """len = 0 (no payload launch), n_recv = 0 (rank 0, zero outputs) and
    n_src = 0, compared with gf_decode_batched and the oracle."""
    for field, N, R, L in ((8, 12, 20, 0), (4, 7, 0, 50), (8, 0, 5, 40)):
        src, coef, payload = _case(field, N, R, L, 4)
        want = _batched(field, N, R, L, coef, payload)
        if N:
            assert _same(want, _expect(field, coef, payload, N, L))
        c, p = _inputs(coef, payload)
        out, rank, used, solved = _outputs(N, L)
        assert gf.gf_decode_noalloc(field, N, R, L, c, p, out, rank, used, solved) == gf.GF_OK
        torch.cuda.synchronize()
        got = (to_host(out)[:N * L], int(rank.item()), int(used.item()), to_host(solved)[:N])
        assert _same(got, want), (field, N, R, L)


def test_noalloc_rejects_sizes_beyond_its_array():
    out, rank, used, solved = _outputs(4, 4)
    # n_src * n_recv above the fixed scratch
    assert gf.gf_decode_noalloc(8, 600, 600, 4, out, out, out, rank) == gf.GF_EINVAL
    # just past the documented limit: 255 x 600 fits the array but its rows do not fit one CTA
    assert gf.gf_decode_noalloc(8, 255, 600, 4, out, out, out, rank) == gf.GF_EINVAL
    # rows that do not fit one CTA's shared memory
    assert gf.gf_decode_noalloc(8, 1000, 200, 4, out, out, out, rank) == gf.GF_EINVAL
    assert gf.gf_decode_noalloc(3, 4, 4, 4, out, out, out, rank) == gf.GF_EINVAL
