"""The uneven encode + decode step at the benchmark's shapes: generations with
N ~ U{8..255}, packet length log-uniform in 64..9000 B, field ~ U{GF(2),
GF(4), GF(16), GF(256)} and 10 % i.i.d. erasures (the sender sends coded
packets until the receiver reaches rank N).  256 generations in one step
(one CUDA-graph replay); every generation's received coded packets, decoded
sources, rank and rows consumed are compared with the oracle's encode and
progressive Gauss-Jordan decode, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import pipeline, synth

import oracle_pool
from gpu_util import dev, torch

pytestmark = pytest.mark.gpu

N_GENS = 256


@pytest.fixture(scope="module")
def stepped():
    dev()
    batch = synth.uneven_batch(n_gens=N_GENS, index=11)
    assert {g.field for g in batch.gens} == {1, 2, 4, 8}
    assert max(g.n_src for g in batch.gens) > 240 and max(g.length for g in batch.gens) > 7000
    work = pipeline.build(batch)
    step = pipeline.UnevenStep(work)
    stream = torch.cuda.Stream()
    step.capture(stream)
    work.dev["out"].zero_()
    work.dev["sent"].zero_()
    step.replay()
    torch.cuda.synchronize()
    recv = [pipeline.received(work, i) for i in range(N_GENS)]
    rank = work.dev["rank"].cpu().numpy()
    used = work.dev["used"].cpu().numpy()
    outs = [pipeline.decoded(work, i) for i in range(N_GENS)]
    step.close()
    return batch, work, recv, rank, used, outs


def _check(args):
    batch, work, recv, rank, used, outs, i = args
    g = batch.gens[i]
    rr = work.recv_rows[i]
    coded = oracle.encode(g.field, g.src, g.coef_stream[rr])
    got = recv[i]
    if not np.array_equal(got, coded):
        return f"{i}: received packets"
    out, solved, r, u = oracle.decode(g.field, g.coef_stream[rr], coded)
    if r != g.n_src or not solved.all() or not np.array_equal(out, g.src):
        return f"{i}: oracle decode did not recover the sources"
    if int(rank[i]) != r or int(used[i]) != u:
        return f"{i}: rank/used {int(rank[i])}/{int(used[i])} vs {r}/{u}"
    if not np.array_equal(outs[i], out):
        return f"{i}: decoded sources"
    return None


def test_every_generation_against_oracle(stepped):
    problems = [p for p in oracle_pool.pmap(_check, [(*stepped, i) for i in range(N_GENS)]) if p]
    assert not problems, problems[:8]
