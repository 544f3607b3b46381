"""Uneven batched encode + decode over a lossy channel (generations of
different field, size and packet length in one launch each), its CUDA-graph
replay and the plain one-call-per-generation form, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, pipeline, synth

from gpu_util import dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def work():
    dev()
    batch = synth.uneven_batch(n_gens=48, n_min=8, n_max=80, len_min=64, len_max=3000, index=3)
    return pipeline.build(batch)


def _check_all(w, sample=(0, 1, 2, 47)):
    for i, g in enumerate(w.batch.gens):
        assert np.array_equal(pipeline.decoded(w, i), g.src), i
    assert (w.dev["rank"].cpu().numpy() == np.array([g.n_src for g in w.batch.gens])).all()
    for i in sample:
        g = w.batch.gens[i]
        rr = w.recv_rows[i]
        coded = oracle.encode(g.field, g.src, g.coef_stream[rr])
        out, solved, rank, used = oracle.decode(g.field, g.coef_stream[rr], coded)
        assert rank == g.n_src and used == rr.size and solved.all()
        assert np.array_equal(out, pipeline.decoded(w, i))


def test_sender_stops_at_rank_n(work):
    for i, g in enumerate(work.batch.gens):
        rr = work.recv_rows[i]
        assert oracle.rank(g.field, g.coef_stream[rr]) == g.n_src
        # one packet fewer would not have been enough
        assert oracle.rank(g.field, g.coef_stream[rr[:-1]]) == g.n_src - 1
        assert work.k_sent[i] == rr.size + work.lost_rows[i].size


def test_one_step_round_trip(work):
    step = pipeline.UnevenStep(work)
    step.launch()
    torch.cuda.synchronize()
    _check_all(work)
    step.close()


def test_received_packets_match_oracle(work):
    step = pipeline.UnevenStep(work)
    step.launch()
    torch.cuda.synchronize()
    for i in (0, 5, 47):
        g = work.batch.gens[i]
        rr = work.recv_rows[i]
        assert np.array_equal(pipeline.received(work, i), oracle.encode(g.field, g.src, g.coef_stream[rr]))
        lr = work.lost_rows[i]
        assert np.array_equal(pipeline.lost(work, i), oracle.encode(g.field, g.src, g.coef_stream[lr]))
    step.close()


def test_graph_replay_and_plain_form(work):
    step = pipeline.UnevenStep(work)
    stream = torch.cuda.Stream()
    step.capture(stream)
    work.dev["out"].zero_()
    work.dev["sent"].zero_()
    step.replay()
    step.replay()
    torch.cuda.synchronize()
    _check_all(work, sample=(3,))
    work.dev["out"].zero_()
    pipeline.plain_step(work)
    torch.cuda.synchronize()
    _check_all(work, sample=(4,))
    step.close()
