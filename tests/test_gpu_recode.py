"""Recoding at intermediate nodes (gf_recode_batched) against the oracle,
bit-exact: every field, a batch of uneven generations in one call, and
recoded packets that the GPU decode turns back into the sources."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _recode(items):
    """items: (field, coef_in R x N, payload_in R x L, mix K2 x R) -> [(coef_out, payload_out)]."""
    keep, args, outs = [], [], []
    for field, ci, pi, mix in items:
        R, N = ci.shape
        K2 = mix.shape[0]
        L = pi.shape[1]
        d_ci, d_pi, d_mix = to_dev(ci.reshape(-1)), to_dev(pi.reshape(-1)), to_dev(mix.reshape(-1))
        d_co = torch.full((max(K2 * N, 1),), 0xA5, dtype=torch.uint8, device=dev())
        d_po = torch.full((max(K2 * L, 1),), 0xA5, dtype=torch.uint8, device=dev())
        keep += [d_ci, d_pi, d_mix, d_co, d_po]
        args.append((field, N, R, K2, L, d_ci, d_pi, d_mix, d_co, d_po))
        outs.append((d_co, d_po, K2, N, L))
    gf.gf_recode_batched(args)
    torch.cuda.synchronize()
    return [(to_host(co)[:K2 * N].reshape(K2, N), to_host(po)[:K2 * L].reshape(K2, L)) for co, po, K2, N, L in outs]


@pytest.mark.parametrize("field", [1, 2, 4, 8])
@pytest.mark.parametrize("shape", [(16, 20, 16, 1500), (64, 70, 64, 1500), (5, 9, 3, 77), (100, 110, 40, 600)])
def test_recode_vs_oracle(field, shape):
    N, R, K2, L = shape
    g = synth.choice(90, field, *shape)
    ci = synth.coefficients(g, field, (R, N), nonzero=False)
    pi = synth.random_bytes(g, (R, L))
    mix = synth.coefficients(g, field, (K2, R), nonzero=False)
    ((co, po),) = _recode([(field, ci, pi, mix)])
    wc, wp = oracle.recode(field, ci, pi, mix)
    assert np.array_equal(co, wc) and np.array_equal(po, wp)


def test_uneven_batch_one_call():
    g = synth.choice(91)
    items = []
    for i in range(20):
        field = (1, 2, 4, 8)[i % 4]
        N, R, K2, L = int(g.integers(1, 80)), int(g.integers(1, 90)), int(g.integers(1, 70)), int(g.integers(1, 2500))
        items.append((field, synth.coefficients(g, field, (R, N), nonzero=False), synth.random_bytes(g, (R, L)),
                      synth.coefficients(g, field, (K2, R), nonzero=False)))
    for (field, ci, pi, mix), (co, po) in zip(items, _recode(items)):
        wc, wp = oracle.recode(field, ci, pi, mix)
        assert np.array_equal(co, wc) and np.array_equal(po, wp), (field, ci.shape, mix.shape)


@pytest.mark.parametrize("field", [2, 8])
def test_recoded_packets_decode_on_the_gpu(field):
    """sender encode -> relay recode -> receiver decode, all on the GPU."""
    g = synth.choice(92, field)
    N, L = 24, 900
    src = synth.random_bytes(g, (N, L))
    C = synth.coefficients(g, field, (N + 8, N), nonzero=False)
    M = synth.coefficients(g, field, (N + 12, N + 8), nonzero=False)
    d_src, d_C, d_M = to_dev(src.reshape(-1)), to_dev(C.reshape(-1)), to_dev(M.reshape(-1))
    coded = torch.empty((N + 8) * L, dtype=torch.uint8, device=dev())
    gf.gf_encode_batched([(field, N, N + 8, L, d_src, d_C, coded)])
    c2 = torch.empty((N + 12) * N, dtype=torch.uint8, device=dev())
    p2 = torch.empty((N + 12) * L, dtype=torch.uint8, device=dev())
    gf.gf_recode_batched([(field, N, N + 8, N + 12, L, d_C, coded, d_M, c2, p2)])
    out = torch.empty(N * L, dtype=torch.uint8, device=dev())
    rank = torch.zeros(1, dtype=torch.int32, device=dev())
    gf.gf_decode_batched([(field, N, N + 12, L, c2, p2, out, rank, None, None)])
    torch.cuda.synchronize()
    c2h = to_host(c2).reshape(N + 12, N)
    assert int(rank.item()) == oracle.rank(field, c2h) == N
    assert np.array_equal(to_host(out).reshape(N, L), src)


def test_recode_plan_equals_call():
    g = synth.choice(93)
    N, R, K2, L = 32, 40, 36, 1000
    ci = synth.coefficients(g, 8, (R, N), nonzero=False)
    pi = synth.random_bytes(g, (R, L))
    mix = synth.coefficients(g, 8, (K2, R), nonzero=False)
    d_ci, d_pi, d_mix = to_dev(ci.reshape(-1)), to_dev(pi.reshape(-1)), to_dev(mix.reshape(-1))
    co = torch.zeros(K2 * N, dtype=torch.uint8, device=dev())
    po = torch.zeros(K2 * L, dtype=torch.uint8, device=dev())
    plan = gf.Plan.recode([(8, N, R, K2, L, d_ci, d_pi, d_mix, co, po)])
    plan.launch()
    torch.cuda.synchronize()
    wc, wp = oracle.recode(8, ci, pi, mix)
    assert np.array_equal(to_host(co).reshape(K2, N), wc) and np.array_equal(to_host(po).reshape(K2, L), wp)
    plan.close()
