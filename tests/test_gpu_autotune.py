"""The encode autotuner on the GPU: for a shape bucket it times the
bit-sliced path and every table-path tile shape, records the fastest, and
GF_PATH_AUTO then encodes with that choice, bit-exact against the oracle.
Two buckets: the uniform batch's shape (64 x 64 x 1500 B, GF(256), where the
tensor-core path wins) and small GF(2) generations (8 sources, 8 coded
packets of 128 B, where a table tile wins)."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

import oracle_pool
from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("field,N,K,L,G,expect", [(8, 64, 64, 1500, 1024, gf.PATH_BITSLICED),
                                                  (1, 8, 8, 128, 2048, gf.PATH_TABLE)])
def test_autotuner_records_fastest_and_auto_uses_it(field, N, K, L, G, expect):
    dev()
    gf.gf_autotune_clear()
    try:
        path, variant = gf.gf_autotune_encode(field, N, K, L, G)
        timings = gf.gf_autotune_last()
        assert len(timings) == 5  # the bit-sliced path and four table tile shapes
        assert {(p, v) for p, v, _ in timings} == {(gf.PATH_BITSLICED, 0)} | {(gf.PATH_TABLE, v) for v in range(4)}
        fastest = min(timings, key=lambda t: t[2])
        assert (path, variant if path == gf.PATH_TABLE else 0) == (fastest[0], fastest[1])
        assert all(ms > 0 for _, _, ms in timings)
        assert path == expect, timings
        # AUTO now takes the recorded choice for this bucket
        assert gf.gf_autotune_query(field, N, K, L) == (path, variant if path == gf.PATH_TABLE else 0)
        # more generations than two per SM, so that AUTO consults the tuned choice (smaller batches
        # take the tensor-core path, which spreads a generation's columns over CTAs)
        g = synth.choice(64, field, N, K, L)
        n = 400
        src = synth.random_bytes(g, (n, N, L))
        coef = synth.coefficients(g, field, (n, K, N), nonzero=False)
        s, c = to_dev(src), to_dev(coef)
        out = torch.zeros((n, K, L), dtype=torch.uint8, device=dev())
        gf.gf_encode_batched([(field, N, K, L, s[i], c[i], out[i]) for i in range(n)], path=gf.PATH_AUTO)
        got = to_host(out)
        bad = oracle_pool.mismatches(lambda i: np.array_equal(got[i], oracle.encode(field, src[i], coef[i])), range(n))
        assert not bad, bad[:8]
    finally:
        gf.gf_autotune_clear()
