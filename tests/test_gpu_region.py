"""GPU parity of gf_region_madd / gf_region_mul against the oracle
(bit-exact), through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, device_bytes, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FIELDS = (1, 2, 4, 8)
LENGTHS = [0, 1, 3, 4, 15, 16, 17, 31, 64, 100, 1000, 1500, 4099, 65536 + 7, (1 << 20) + 13]


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("length", LENGTHS)
def test_madd_mul_vs_oracle(field, length):
    src, dst, c = synth.region(length, field)
    buf_d = to_dev(dst)
    gf.gf_region_madd(field, buf_d, to_dev(src), c)
    assert np.array_equal(to_host(buf_d), oracle.region_madd(field, dst, src, c))
    buf_m = to_dev(dst)
    gf.gf_region_mul(field, buf_m, to_dev(src), c)
    assert np.array_equal(to_host(buf_m), oracle.region_mul(field, src, c))


@pytest.mark.parametrize("field", FIELDS)
def test_every_coefficient(field):
    src, dst, _ = synth.region(4096 + 5, field, index=7)
    s_d = to_dev(src)
    for c in range(1 << field):
        d = to_dev(dst)
        gf.gf_region_madd(field, d, s_d, c)
        assert np.array_equal(to_host(d), oracle.region_madd(field, dst, src, c)), c
        m = to_dev(dst)
        gf.gf_region_mul(field, m, s_d, c)
        assert np.array_equal(to_host(m), oracle.region_mul(field, src, c)), c


@pytest.mark.parametrize("field", FIELDS)
@pytest.mark.parametrize("doff,soff", [(0, 0), (1, 1), (3, 3), (0, 1), (1, 0), (5, 2), (2, 7), (8, 3), (4, 0)])
def test_misaligned(field, doff, soff):
    length = 10000 + 3
    src, dst, c = synth.region(length, field, index=doff * 16 + soff)
    big_s = torch.zeros(length + 32, dtype=torch.uint8, device=dev())
    big_d = torch.zeros(length + 32, dtype=torch.uint8, device=dev())
    big_s[soff:soff + length] = to_dev(src)
    big_d[doff:doff + length] = to_dev(dst)
    gf.gf_region_madd(field, big_d.data_ptr() + doff, big_s.data_ptr() + soff, c, length)
    out = to_host(big_d)
    assert np.array_equal(out[doff:doff + length], oracle.region_madd(field, dst, src, c))
    assert not out[:doff].any() and not out[doff + length:].any(), "wrote outside the region"
    gf.gf_region_mul(field, big_d.data_ptr() + doff, big_s.data_ptr() + soff, c, length)
    out = to_host(big_d)
    assert np.array_equal(out[doff:doff + length], oracle.region_mul(field, src, c))
    assert not out[:doff].any() and not out[doff + length:].any()


@pytest.mark.parametrize("field", FIELDS)
def test_in_place(field):
    src, _, c = synth.region(5000, field, index=3)
    d = to_dev(src)
    gf.gf_region_mul(field, d, d, c)
    assert np.array_equal(to_host(d), oracle.region_mul(field, src, c))
    d = to_dev(src)
    gf.gf_region_madd(field, d, d, c)
    assert np.array_equal(to_host(d), oracle.region_madd(field, src, src, c))


def test_errors_on_device_pointers():
    d = torch.zeros(64, dtype=torch.uint8, device=dev())
    p = d.data_ptr()
    assert gf.region_status("gf_region_madd", 8, p, p + 8, 3, 16) == gf.GF_EOVERLAP
    assert gf.region_status("gf_region_madd", 4, p, p + 32, 16, 16) == gf.GF_EINVAL
    assert gf.region_status("gf_region_mul", 7, p, p + 32, 1, 16) == gf.GF_EINVAL


@pytest.mark.parametrize("field", FIELDS)
def test_full_size_1gib_sampled(field):
    """1 GiB region (the largest size of the bandwidth sweep) in the launch
    configuration the benchmark times; sampled bytes against the oracle."""
    n = 1 << 30
    src = device_bytes(n, 11 + field)
    dst = device_bytes(n, 29 + field)
    g = synth.choice(40, field)
    idx = np.unique(np.concatenate([g.integers(0, n, 200000), np.arange(64), np.arange(n - 64, n)]))
    idx_t = torch.from_numpy(idx).to(dev())
    s_in = to_host(src[idx_t])
    d_in = to_host(dst[idx_t])
    c = int(g.integers(1, 1 << field)) if field > 1 else 1
    gf.gf_region_madd(field, dst, src, c)
    assert np.array_equal(to_host(dst[idx_t]), oracle.region_madd(field, d_in, s_in, c))
    gf.gf_region_mul(field, dst, src, c)
    assert np.array_equal(to_host(dst[idx_t]), oracle.region_mul(field, s_in, c))
    del src, dst
    torch.cuda.empty_cache()
