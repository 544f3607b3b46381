"""Systematic coding: the sender sends its N sources uncoded first (unit
coding vectors), then coded packets.  The decode flag GF_DEC_SYSTEMATIC (the
payload phase on the table path, which skips zero multipliers) gives the
oracle's decode, bit-exact, with and without losses; resident decoders fed
from host memory recognise the unit rows; the server's systematic encode and
decode requests equal the oracle and are the same alone and in the mix."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, serve, synth

import oracle_pool
from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FIELDS = (1, 2, 4, 8)


def _systematic_rows(ge, loss, *key):
    stream = synth.systematic_stream(ge.coef_stream)
    lost = synth.erasures(stream.shape[0], loss, *key)
    return np.ascontiguousarray(stream[~lost])


@pytest.mark.parametrize("loss", [0.0, 0.1])
def test_systematic_decode_matches_oracle(loss):
    batch = synth.uneven_batch(n_gens=24, n_min=8, n_max=255, len_min=64, len_max=3000, index=21)
    items, keep, meta = [], [], []
    for i, ge in enumerate(batch.gens):
        coef = _systematic_rows(ge, loss, 21, i)
        payload = oracle.encode(ge.field, ge.src, coef)
        N, R, L = ge.n_src, coef.shape[0], ge.length
        bufs = [to_dev(coef.reshape(-1)), to_dev(payload.reshape(-1))]
        outs = [torch.zeros(N * L, dtype=torch.uint8, device=dev()), torch.zeros(1, dtype=torch.int32, device=dev()),
                torch.zeros(1, dtype=torch.int32, device=dev()), torch.zeros(N, dtype=torch.uint8, device=dev())]
        keep += bufs + outs
        meta.append((ge, coef, payload, outs))
        items.append((ge.field, N, R, L, *bufs, *outs))
    results = {}
    for flags in (gf.DEC_SYSTEMATIC, 0):
        gf.gf_decode_batched([it + (flags,) for it in items])
        torch.cuda.synchronize()
        results[flags] = [(to_host(o[0]).copy(), int(o[1].item()), int(o[2].item()), to_host(o[3]).copy())
                          for _, _, _, o in meta]

    def check(j):
        ge, coef, payload, _ = meta[j]
        out, solved, rank, used = oracle.decode(ge.field, coef, payload)
        got = results[gf.DEC_SYSTEMATIC][j]
        return (np.array_equal(got[0], out.reshape(-1)) and got[1] == rank and got[2] == used
                and np.array_equal(got[3], solved.astype(np.uint8)) and rank == ge.n_src)

    assert not oracle_pool.mismatches(check, range(len(meta)))
    for a, b in zip(results[gf.DEC_SYSTEMATIC], results[0]):
        assert np.array_equal(a[0], b[0]) and a[1:3] == b[1:3] and np.array_equal(a[3], b[3])


def test_resident_decoder_with_uncoded_sources():
    dev()
    for field in FIELDS:
        ge = synth.uneven_batch(n_gens=1, n_min=40, n_max=40, len_min=700, len_max=700, index=22,
                                fields=(field,)).gens[0]
        coef = _systematic_rows(ge, 0.1, 22, field)
        payload = oracle.encode(field, ge.src, coef)
        d = gf.Decoder(field, ge.n_src, coef.shape[0], ge.length)
        ch = torch.from_numpy(coef).pin_memory()
        ph = torch.from_numpy(payload).pin_memory()
        d.push(ch, ph, coef.shape[0])
        gf.Decoder.poll([d])
        rank = d.status(wait=True)[0]
        out = torch.zeros(ge.n_src * ge.length, dtype=torch.uint8).pin_memory()
        d.read(out)
        torch.cuda.synchronize()
        assert rank == ge.n_src
        assert np.array_equal(out.numpy().reshape(ge.n_src, ge.length), ge.src)
        d.close()


def _requests(n=30, index=0, loss=0.1):
    batch = synth.uneven_batch(n_gens=n, n_min=4, n_max=60, len_min=64, len_max=1500, index=200 + index)
    times = synth.arrivals(3000.0, n, index=50 + index)
    reqs = []
    for i, (ge, t) in enumerate(zip(batch.gens, times)):
        if i % 2 == 0:
            extra = int(np.ceil(0.2 * ge.n_src)) + 1
            reqs.append(serve.EncodeRequest(i, float(t), ge.field, ge.src,
                                            np.ascontiguousarray(ge.coef_stream[:extra]), systematic=True))
        else:
            coef = _systematic_rows(ge, loss, 23, index, i)
            payload = oracle.encode(ge.field, ge.src, coef)
            ptimes = float(t) + 20e-6 * np.arange(1, coef.shape[0] + 1)
            reqs.append(serve.DecodeRequest(i, float(t), ge.field, ge.n_src, ge.length, coef, payload, ptimes))
    return batch, reqs


@pytest.mark.parametrize("loss", [0.0, 0.1])
def test_server_systematic_mix_and_alone(loss):
    dev()
    batch, reqs = _requests(index=int(loss * 10), loss=loss)
    serve.Server(mem_budget=1 << 28, max_active=8, n_streams=3).run(reqs)
    for r, ge in zip(reqs, batch.gens):
        if isinstance(r, serve.EncodeRequest):
            want = np.concatenate([ge.src, oracle.encode(r.field, r.src, r.coef)])
            assert np.array_equal(r.result, want), r.rid
        else:
            assert r.rank == r.n_src and np.array_equal(r.result, ge.src), r.rid
    for pick in (0, 1, 4, 5):
        r = reqs[pick]
        if isinstance(r, serve.EncodeRequest):
            alone = serve.EncodeRequest(r.rid, 0.0, r.field, r.src, r.coef, systematic=True)
        else:
            alone = serve.DecodeRequest(r.rid, 0.0, r.field, r.n_src, r.length, r.coef, r.payload,
                                        r.packet_times - r.arrival)
        serve.Server(mem_budget=1 << 28).run([alone])
        assert np.array_equal(alone.result, r.result), pick
