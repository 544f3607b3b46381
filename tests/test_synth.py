"""The seeded synthetic inputs follow the recipes stated for the workloads:
the same key gives the same bytes, and the drawn shapes, fields, coefficients,
erasures and arrival times have the stated ranges and distributions (means
within about five standard errors)."""
import math

import numpy as np

from paper_1909_02871_gb300 import synth


def test_same_key_same_draws_other_key_other_draws():
    a = synth.uniform_batch(n_gens=3, n_src=4, length=50, n_coded=5, index=0)
    b = synth.uniform_batch(n_gens=3, n_src=4, length=50, n_coded=5, index=0)
    c = synth.uniform_batch(n_gens=3, n_src=4, length=50, n_coded=5, index=1)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.coef, b.coef)
    assert not np.array_equal(a.src, c.src)


def test_uniform_batch_coefficients_are_nonzero_field_elements():
    for field in synth.FIELDS:
        b = synth.uniform_batch(n_gens=8, n_src=16, length=32, n_coded=16, field=field)
        lo = 0 if field == 1 else 1   # GF(2) minus zero would leave only 1: zero is kept there
        assert b.coef.min() >= lo and b.coef.max() < (1 << field)
        if field == 8:
            assert b.coef.min() == 1 and b.coef.max() == 255
    b = synth.uniform_batch(n_gens=64, n_src=64, length=64, n_coded=64)
    mean = b.src.mean()
    assert abs(mean - 127.5) < 5 * 73.9 / math.sqrt(b.src.size)   # uniform bytes: sd 73.9


def test_single_generation_codes_the_same_bytes_in_every_field():
    gens = [synth.generation(f) for f in synth.FIELDS]
    for g in gens[1:]:
        assert np.array_equal(g.src, gens[0].src)
    for f, g in zip(synth.FIELDS, gens):
        assert g.src.shape == (16, 1500) and g.coef_stream.shape[1] == 16
        assert g.coef_stream.max() < (1 << f)


def test_uneven_batch_follows_its_recipe():
    G = 300
    b = synth.uneven_batch(n_gens=G, index=11)
    n = np.array([g.n_src for g in b.gens])
    ln = np.array([g.length for g in b.gens])
    f = np.array([g.field for g in b.gens])
    assert n.min() >= 8 and n.max() <= 255
    # N ~ U{8..255}: mean 131.5, sd 71.6
    assert abs(n.mean() - 131.5) < 5 * 71.6 / math.sqrt(G)
    # len log-uniform on [64, 9000]: log mean (ln 64 + ln 9000) / 2, sd (ln 9000 - ln 64) / sqrt(12)
    assert ln.min() >= 64 and ln.max() <= 9000
    lmu, lsd = (math.log(64) + math.log(9000)) / 2, (math.log(9000) - math.log(64)) / math.sqrt(12)
    assert abs(np.log(ln).mean() - lmu) < 5 * lsd / math.sqrt(G)
    # field ~ U{1, 2, 4, 8}
    for fld in synth.FIELDS:
        share = (f == fld).mean()
        assert abs(share - 0.25) < 5 * math.sqrt(0.25 * 0.75 / G)
    # coding vectors over GF(q) with zero, streams long enough, i.i.d. 10 % erasures
    erased = total = 0
    for g in b.gens:
        assert g.coef_stream.shape == (synth.uneven_stream_len(g.n_src, 0.10), g.n_src)
        assert g.coef_stream.max() < (1 << g.field)
        assert g.erased.shape == (g.coef_stream.shape[0],)
        assert (~g.erased).sum() >= g.n_src + 40     # enough rows get through for rank N
        erased += int(g.erased.sum())
        total += g.erased.size
    p = erased / total
    assert abs(p - 0.10) < 5 * math.sqrt(0.10 * 0.90 / total)
    zero_share = np.mean([(g.coef_stream == 0).mean() for g in b.gens if g.field == 8])
    assert abs(zero_share - 1 / 256) < 0.002


def test_arrivals_are_poisson():
    rate, n = 2000.0, 20000
    t = synth.arrivals(rate, n, index=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 5 / math.sqrt(n)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def test_systematic_stream_and_erasures():
    """A systematic sender's stream: the N unit vectors in source order, then
    the coded vectors unchanged; erasures are seeded and near their rate."""
    g = synth.uneven_batch(n_gens=1, n_min=12, n_max=12, index=5).gens[0]
    s = synth.systematic_stream(g.coef_stream)
    assert s.shape == (12 + g.coef_stream.shape[0], 12) and s.dtype == np.uint8
    assert np.array_equal(s[:12], np.eye(12, dtype=np.uint8))
    assert np.array_equal(s[12:], g.coef_stream)
    a = synth.erasures(20000, 0.1, 3)
    assert np.array_equal(a, synth.erasures(20000, 0.1, 3))
    assert not np.array_equal(a, synth.erasures(20000, 0.1, 4))
    assert abs(a.mean() - 0.1) < 0.01
    assert not synth.erasures(100, 0.0, 1).any()
