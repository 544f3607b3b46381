"""GPU parity of the batched encode (Eq. 2) against the oracle (bit-exact),
through the C ABI: single generation, ragged/uneven batches, every table
tile shape, the bit-sliced tensor-core path, plans and CUDA graph replay,
the full 4096 x 64 x 1500 B batch (every generation) and packets of up to
64 KiB."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

import oracle_pool
from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FIELDS = (1, 2, 4, 8)


def _run(items, path=gf.PATH_AUTO):
    """items: list of (field, src np N x L, coef np K x N) -> list of outputs."""
    keep, gens, outs = [], [], []
    for field, src, coef in items:
        K, N = coef.shape
        L = src.shape[1] if src.ndim == 2 else 0
        s = to_dev(src.reshape(-1)) if src.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        c = to_dev(coef.reshape(-1)) if coef.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        o = torch.full((max(K * L, 1),), 0xA5, dtype=torch.uint8, device=dev())
        keep += [s, c, o]
        gens.append((field, N, K, L, s, c, o))
        outs.append((o, K, L))
    gf.gf_encode_batched(gens, path=path)
    return [to_host(o)[:K * L].reshape(K, L) for o, K, L in outs]


@pytest.mark.parametrize("field", FIELDS)
def test_single_generation(field):
    gen = synth.generation(field)
    coef = gen.coef_stream[:gen.n_coded]
    (out,) = _run([(field, gen.src, coef)])
    assert np.array_equal(out, oracle.encode(field, gen.src, coef))


def _ragged_items(seed, fields=FIELDS):
    g = synth.choice(50, seed)
    items = []
    for N in (0, 1, 3, 17, 64):
        for K in (0, 1, 15, 16, 17, 33):
            L = int(g.choice([0, 1, 5, 127, 128, 129, 513, 1500, 4097]))
            field = int(g.choice(fields))
            src = synth.random_bytes(g, (N, L))
            coef = synth.coefficients(g, field, (K, N), nonzero=False)
            items.append((field, src, coef))
    return items


@pytest.mark.parametrize("seed", [0, 1])
def test_ragged_uneven_batch_one_launch(seed):
    items = _ragged_items(seed)
    outs = _run(items)
    for (field, src, coef), out in zip(items, outs):
        assert np.array_equal(out, oracle.encode(field, src, coef)), (field, src.shape, coef.shape)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_table_tile_shape(variant):
    items = [it for it in _ragged_items(7) if it[2].size and it[1].size]
    try:
        for field, src, coef in items:
            gf.gf_autotune_set(field, src.shape[0], coef.shape[0], src.shape[1], gf.PATH_TABLE, variant)
        outs = _run(items, path=gf.PATH_TABLE)
    finally:
        gf.gf_autotune_clear()
    for (field, src, coef), out in zip(items, outs):
        assert np.array_equal(out, oracle.encode(field, src, coef))


def _bitsliced_ok():
    try:
        (o,) = _run([(8, np.zeros((32, 512), np.uint8), np.ones((32, 32), np.uint8))], path=gf.PATH_BITSLICED)
        return True
    except gf.GFError as e:
        if e.status == gf.GF_ENOTSUP:
            return False
        raise


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("shape", [(64, 64, 1500), (17, 40, 777), (1, 1, 1), (64, 33, 129), (40, 64, 4096),
                                   (65, 70, 300), (130, 64, 1000), (255, 33, 257)])
def test_bitsliced_every_field(field, shape):
    """GF(2), GF(4), GF(16) bytes hold 8/n words multiplied by the same
    coefficient: the bit-sliced path uses block-diagonal 8x8 matrices.  N > 64
    runs in 64-source chunks whose parities are XORed together."""
    if not _bitsliced_ok():
        pytest.skip("bit-sliced path unavailable")
    N, K, L = shape
    g = synth.choice(61, field, N, K, L)
    src = synth.random_bytes(g, (N, L))
    coef = synth.coefficients(g, field, (K, N), nonzero=False)
    (out,) = _run([(field, src, coef)], path=gf.PATH_BITSLICED)
    assert np.array_equal(out, oracle.encode(field, src, coef))


def test_bitsliced_mixed_fields_one_launch():
    if not _bitsliced_ok():
        pytest.skip("bit-sliced path unavailable")
    g = synth.choice(62)
    items = []
    for i in range(24):
        field = FIELDS[i % 4]
        N, K, L = int(g.integers(1, 256)), int(g.integers(1, 100)), int(g.integers(1, 3000))
        items.append((field, synth.random_bytes(g, (N, L)), synth.coefficients(g, field, (K, N), nonzero=False)))
    outs = _run(items, path=gf.PATH_BITSLICED)
    for (field, src, coef), out in zip(items, outs):
        assert np.array_equal(out, oracle.encode(field, src, coef)), (field, src.shape, coef.shape)


@pytest.mark.parametrize("shape", [(64, 64, 1500), (16, 16, 1500), (1, 1, 1), (33, 70, 255), (128, 96, 4097),
                                   (255, 300, 700), (64, 64, 256), (7, 200, 3000)])
def test_bitsliced_vs_oracle(shape):
    if not _bitsliced_ok():
        pytest.skip("bit-sliced path unavailable")
    N, K, L = shape
    g = synth.choice(60, N, K, L)
    src = synth.random_bytes(g, (N, L))
    coef = synth.coefficients(g, 8, (K, N), nonzero=False)
    (out,) = _run([(8, src, coef)], path=gf.PATH_BITSLICED)
    assert np.array_equal(out, oracle.encode(8, src, coef))


def test_bitsliced_equals_table_on_batch():
    if not _bitsliced_ok():
        pytest.skip("bit-sliced path unavailable")
    b = synth.uniform_batch(n_gens=24, index=3)
    items = [(8, b.src[i], b.coef[i]) for i in range(24)]
    a = _run(items, path=gf.PATH_BITSLICED)
    t = _run(items, path=gf.PATH_TABLE)
    for x, y in zip(a, t):
        assert np.array_equal(x, y)
    for i in (0, 23):
        assert np.array_equal(a[i], oracle.encode(8, b.src[i], b.coef[i]))


def test_plan_and_graph_replay():
    items = _ragged_items(3)
    keep, gens, outs = [], [], []
    for field, src, coef in items:
        K, N = coef.shape
        L = src.shape[1]
        s = to_dev(src.reshape(-1)) if src.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        c = to_dev(coef.reshape(-1)) if coef.size else torch.zeros(1, dtype=torch.uint8, device=dev())
        o = torch.zeros(max(K * L, 1), dtype=torch.uint8, device=dev())
        keep += [s, c, o]
        gens.append((field, N, K, L, s, c, o))
        outs.append((o, K, L))
    plan = gf.Plan.encode(gens)
    assert plan.kernel_count >= 1
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan.launch(stream)  # warm-up outside capture
        stream.synchronize()
        for o, _, _ in outs:
            o.zero_()
        with torch.cuda.graph(graph, stream=stream):
            plan.launch(stream)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    for (field, src, coef), (o, K, L) in zip(items, outs):
        assert np.array_equal(to_host(o)[:K * L].reshape(K, L), oracle.encode(field, src, coef))
    plan.close()


def test_full_uniform_batch_every_generation():
    """The 4096 x (N=64 x 1500 B) GF(256) batch, K = 64, in the launch the
    benchmark times (path chosen by the autotuner): every generation compared
    with the oracle (run on every host core); the table path's launch is
    compared with it byte for byte."""
    b = synth.uniform_batch()
    G, N, L = b.src.shape
    K = b.coef.shape[1]
    src = to_dev(b.src)
    coef = to_dev(b.coef)
    out = torch.empty((G, K, L), dtype=torch.uint8, device=dev())
    gens = [(8, N, K, L, src[i], coef[i], out[i]) for i in range(G)]
    out.fill_(0)
    gf.gf_encode_batched(gens, path=gf.PATH_AUTO)
    got = to_host(out)
    bad = oracle_pool.mismatches(lambda i: np.array_equal(got[i], oracle.encode(8, b.src[i], b.coef[i])), range(G))
    assert not bad, f"{len(bad)} generations differ from the oracle, first {bad[:8]}"
    out.fill_(0)
    gf.gf_encode_batched(gens, path=gf.PATH_TABLE)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.from_numpy(got).to(dev())), "table path differs from the benchmarked launch"


@pytest.mark.parametrize("path", [gf.PATH_TABLE, gf.PATH_BITSLICED])
@pytest.mark.parametrize("field", FIELDS)
def test_fig1_packet_sizes(field, path):
    """The packet sizes of the paper's Fig. 1 sweep beyond 4 KiB: generations
    of N = 16 sources and K = 16 coded packets of 8, 16, 32 and 64 KiB (and
    a ragged 64 KiB - 3), several generations per launch, on both paths."""
    if path == gf.PATH_BITSLICED and not _bitsliced_ok():
        pytest.skip("bit-sliced path unavailable")
    g = synth.choice(63, field, path)
    items = []
    for L in (8 << 10, 16 << 10, 32 << 10, 64 << 10, (64 << 10) - 3):
        for _ in range(2):
            items.append((field, synth.random_bytes(g, (16, L)), synth.coefficients(g, field, (16, 16), nonzero=True)))
    outs = _run(items, path=path)
    bad = oracle_pool.mismatches(lambda j: np.array_equal(outs[j], oracle.encode(field, items[j][1], items[j][2])),
                                 range(len(items)))
    assert not bad, [items[j][1].shape for j in bad]


def test_host_encoder_pipelined_steps():
    """pipeline.HostEncoder: host-resident batch in chunks on three streams;
    two steps in a row (the second reusing the device buffers while the
    first's downloads may still run) give the oracle's coded packets."""
    from paper_1909_02871_gb300 import pipeline
    dev()
    G, N, K, L = 40, 16, 24, 700
    g = synth.choice(97)
    src = synth.random_bytes(g, (G, N, L))
    coef = synth.coefficients(g, 8, (G, K, N), nonzero=False)
    src_h = torch.from_numpy(src).pin_memory()
    coef_h = torch.from_numpy(coef).pin_memory()
    out_h = torch.zeros((G, K, L), dtype=torch.uint8).pin_memory()
    src_d = torch.empty((G, N, L), dtype=torch.uint8, device=dev())
    coef_d = torch.empty((G, K, N), dtype=torch.uint8, device=dev())
    out_d = torch.empty((G, K, L), dtype=torch.uint8, device=dev())
    enc = pipeline.HostEncoder(8, src_h, coef_h, out_h, src_d, coef_d, out_d, chunks=5)
    enc.step()
    enc.step()
    enc.synchronize()
    got = out_h.numpy()
    for i in range(G):
        assert np.array_equal(got[i], oracle.encode(8, src[i], coef[i])), i
    enc.close()
