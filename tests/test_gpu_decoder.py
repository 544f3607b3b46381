"""Resident decoders (gf_dec_open / push / poll / status / close): packets
pushed one at a time from host or device memory, many decoders in one poll,
rank growing as packets arrive, the decoded packets equal to the sources and
to the oracle's decode of the same packets."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, to_host, torch

pytestmark = pytest.mark.gpu


def _stream_packets(field, n, length, extra, index, dup_first=0):
    """Sources, a stream of coding vectors (optionally starting with repeats
    of the first vector) and the coded packets the oracle makes of them."""
    g = synth.choice(70, field, n, length, index)
    src = synth.random_bytes(g, (n, length))
    coef = synth.coefficients(g, field, (n + extra, n), nonzero=False)
    if dup_first:
        coef = np.concatenate([np.repeat(coef[:1], dup_first, axis=0), coef])
    return src, coef, oracle.encode(field, src, coef)


def _download(d, stream):
    out = torch.empty(max(d.n_src * d.length, 1), dtype=torch.uint8, device=dev())
    d.read(out, stream=stream)
    stream.synchronize()
    return to_host(out)[:d.n_src * d.length]


@pytest.mark.parametrize("field", [1, 2, 4, 8])
def test_packets_one_at_a_time(field):
    dev()
    n, L = 12, 777
    src, coef, coded = _stream_packets(field, n, L, extra=20, index=0)
    d = gf.Decoder(field, n, coef.shape[0], L)
    stream = torch.cuda.Stream()
    coef_h = torch.from_numpy(coef).pin_memory()
    coded_h = torch.from_numpy(coded).pin_memory()
    done_at = None
    try:
        for i in range(coef.shape[0]):
            d.push(coef_h[i], coded_h[i], 1, stream=stream)
            k = gf.Decoder.poll([d], stream=stream)
            assert k == (1 if i + 1 >= n else 0)
            rank, received, addr = d.status(wait=True)
            assert received == i + 1
            want_rank = oracle.rank(field, coef[:i + 1]) if i + 1 >= n else -1
            assert rank == want_rank
            if rank == n:
                done_at = i + 1
                out = _download(d, stream).reshape(n, L)
                assert np.array_equal(out, src)
                ref, _, r2, used = oracle.decode(field, coef[:i + 1], coded[:i + 1])
                assert r2 == n and np.array_equal(out, ref)
                break
        assert done_at is not None
        # nothing new: a poll attempts nothing
        assert gf.Decoder.poll([d], stream=stream) == 0
    finally:
        d.close()


def test_many_decoders_one_poll_mixed_fields_and_sources():
    dev()
    stream = torch.cuda.Stream()
    decs, want = [], []
    for i, (field, n, L) in enumerate([(8, 16, 1500), (4, 40, 300), (2, 7, 4097), (1, 33, 64), (8, 64, 2000),
                                       (8, 200, 512)]):
        src, coef, coded = _stream_packets(field, n, L, extra=12, index=10 + i)
        d = gf.Decoder(field, n, coef.shape[0], L)
        if i % 2:   # device tensors
            c = torch.from_numpy(coef).to(dev())
            p = torch.from_numpy(coded).to(dev())
        else:       # pinned host tensors
            c = torch.from_numpy(coef).pin_memory()
            p = torch.from_numpy(coded).pin_memory()
        d.push(c, p, coef.shape[0], stream=stream)
        decs.append((d, c, p))
        want.append((field, src, coef, coded))
    try:
        assert gf.Decoder.poll([d for d, _, _ in decs], stream=stream) == len(decs)
        for (d, _, _), (field, src, coef, coded) in zip(decs, want):
            rank, received, addr = d.status(wait=True)
            assert received == coef.shape[0]
            assert rank == src.shape[0] == oracle.rank(field, coef)
            out = _download(d, stream).reshape(src.shape)
            assert np.array_equal(out, src)
    finally:
        for d, _, _ in decs:
            d.close()


def test_rank_deficient_until_more_packets():
    """Repeats of one coding vector carry no information: the first attempt
    stops short of rank N, later packets complete it."""
    dev()
    field, n, L = 8, 10, 256
    src, coef, coded = _stream_packets(field, n, L, extra=8, index=30, dup_first=n)
    d = gf.Decoder(field, n, coef.shape[0], L)
    stream = torch.cuda.Stream()
    try:
        d.push(torch.from_numpy(coef[:n]).to(dev()), torch.from_numpy(coded[:n]).to(dev()), n, stream=stream)
        assert gf.Decoder.poll([d], stream=stream) == 1
        rank, _, _ = d.status(wait=True)
        assert rank == 1 == oracle.rank(field, coef[:n])
        rest = coef.shape[0] - n
        d.push(torch.from_numpy(coef[n:]).to(dev()), torch.from_numpy(coded[n:]).to(dev()), rest, stream=stream)
        assert gf.Decoder.poll([d], stream=stream) == 1
        st = None
        while st is None:  # the non-waiting form eventually reports the attempt
            st = d.status(wait=False)
        rank, received, addr = st
        assert received == coef.shape[0] and rank == n
        assert np.array_equal(_download(d, stream).reshape(n, L), src)
    finally:
        d.close()


def test_push_beyond_capacity_is_rejected():
    dev()
    d = gf.Decoder(8, 4, 4, 16)
    try:
        c = torch.zeros(20, dtype=torch.uint8, device=dev())
        p = torch.zeros(80, dtype=torch.uint8, device=dev())
        d.push(c, p, 4)
        with pytest.raises(gf.GFError) as e:
            d.push(c, p, 1)
        assert e.value.status == gf.GF_EINVAL
    finally:
        d.close()
