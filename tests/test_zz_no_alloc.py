"""gf_decode_noalloc: the decode entry point for callers that cannot let a
call allocate device memory (its scratch is a fixed device array inside the
library).  Checked through the C ABI against gf_decode_batched, bit-exact (the
tolerance of every decode test), on two calls in a row that share the array.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
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
    return coef, payload


def _outputs(n_src, length):
    return (torch.full((max(n_src * length, 1),), 0x77, dtype=torch.uint8, device=dev()),
            torch.full((1,), -3, dtype=torch.int32, device=dev()),
            torch.full((1,), -3, dtype=torch.int32, device=dev()),
            torch.full((max(n_src, 1),), 9, dtype=torch.uint8, device=dev()))


def _reference(field, coef, payload):
    R, N = coef.shape
    L = payload.shape[1]
    c, p = to_dev(coef.reshape(-1)), to_dev(payload.reshape(-1))
    out, rank, used, solved = _outputs(N, L)
    gf.gf_decode_batched([(field, N, R, L, c, p, out, rank, used, solved)])
    torch.cuda.synchronize()
    return (to_host(out)[:N * L], int(rank.item()), int(used.item()), to_host(solved)[:N])


def test_noalloc_matches_batched_decode_two_calls_in_a_row():
    cases = [(8, 40, 47, 1500, 0), (4, 17, 17, 333, 1)]  # the second one reuses the array
    refs, keep = [], []
    for field, N, R, L, idx in cases:
        coef, payload = _case(field, N, R, L, idx)
        refs.append(_reference(field, coef, payload))
        keep.append((field, N, R, L, to_dev(coef.reshape(-1)), to_dev(payload.reshape(-1)), *_outputs(N, L)))
    for field, N, R, L, c, p, out, rank, used, solved in keep:
        assert gf.gf_decode_noalloc(field, N, R, L, c, p, out, rank, used, solved) == gf.GF_OK
    torch.cuda.synchronize()
    for (field, N, R, L, c, p, out, rank, used, solved), ref in zip(keep, refs):
        assert np.array_equal(to_host(out)[:N * L], ref[0])
        assert int(rank.item()) == ref[1] and int(used.item()) == ref[2]
        assert np.array_equal(to_host(solved)[:N], ref[3])
    # the first case decodes its sources completely
    assert refs[0][1] == 40


def test_noalloc_rejects_sizes_beyond_its_array():
    out, rank, used, solved = _outputs(4, 4)
    # n_src * n_recv above the fixed scratch
    assert gf.gf_decode_noalloc(8, 600, 600, 4, out, out, out, rank) == gf.GF_EINVAL
    # rows that do not fit one CTA's shared memory
    assert gf.gf_decode_noalloc(8, 1000, 200, 4, out, out, out, rank) == gf.GF_EINVAL
    assert gf.gf_decode_noalloc(3, 4, 4, 4, out, out, out, rank) == gf.GF_EINVAL
