"""The continuous-batching server: every encode result equals the oracle's
Eq. 2, every decode recovers its sources (and equals the oracle's decode of
the packets it used), and each result is the same served alone and in the
mix."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import serve, synth

from gpu_util import dev, torch

pytestmark = pytest.mark.gpu


def _requests(n=40, rate=2000.0, index=0):
    batch = synth.uneven_batch(n_gens=n, n_min=4, n_max=40, len_min=64, len_max=1500, index=100 + index)
    times = synth.arrivals(rate, n, index=index)
    g = synth.choice(80, index)
    reqs = []
    for i, (ge, t) in enumerate(zip(batch.gens, times)):
        if i % 2 == 0:
            K = int(g.integers(1, ge.n_src + 8))
            reqs.append(serve.EncodeRequest(i, float(t), ge.field, ge.src, np.ascontiguousarray(ge.coef_stream[:K])))
        else:
            keep = ~ge.erased
            coef = np.ascontiguousarray(ge.coef_stream[keep])
            payload = oracle.encode(ge.field, ge.src, coef)
            ptimes = float(t) + 20e-6 * np.arange(1, coef.shape[0] + 1)
            reqs.append(serve.DecodeRequest(i, float(t), ge.field, ge.n_src, ge.length, coef, payload, ptimes))
    return batch, reqs


def _fresh(r):
    if isinstance(r, serve.EncodeRequest):
        return serve.EncodeRequest(r.rid, 0.0, r.field, r.src, r.coef)
    return serve.DecodeRequest(r.rid, 0.0, r.field, r.n_src, r.length, r.coef, r.payload,
                               r.packet_times - r.arrival)


def test_mix_matches_oracle():
    dev()
    batch, reqs = _requests()
    server = serve.Server(mem_budget=1 << 28, max_active=16, n_streams=3)
    server.run(reqs)
    assert server.batches >= 2
    for r, ge in zip(reqs, batch.gens):
        assert r.done_at is not None and r.done_at >= r.arrival
        if isinstance(r, serve.EncodeRequest):
            assert np.array_equal(r.result, oracle.encode(r.field, r.src, r.coef)), r.rid
        else:
            assert r.rank == r.n_src
            assert np.array_equal(r.result, ge.src), r.rid
            ref, _, rank, used = oracle.decode(r.field, r.coef, r.payload)
            assert np.array_equal(r.result, ref)
    stats = serve.latency_stats(reqs)
    assert stats["n"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_alone_equals_in_mix():
    dev()
    _, reqs = _requests(index=1)
    serve.Server(mem_budget=1 << 28, max_active=8).run(reqs)
    for pick in (0, 1, 6, 7):
        alone = _fresh(reqs[pick])
        serve.Server(mem_budget=1 << 28).run([alone])
        assert np.array_equal(alone.result, reqs[pick].result), pick


def test_admission_by_memory_budget():
    """A budget that holds only a few requests still serves everything."""
    dev()
    _, reqs = _requests(n=16, rate=1e6, index=2)
    biggest = max(r.device_bytes() for r in reqs)
    server = serve.Server(mem_budget=2 * biggest, max_active=64)
    server.run(reqs)
    assert all(r.done_at is not None for r in reqs)
    assert server.mem_used == 0
