"""The device-side bounded waits give up instead of hanging: a kernel waits
on an mbarrier nothing arrives at (gf_selftest_wait); the wait runs out, the
status word reports GF_ETIMEOUT, and the context keeps working (an encode
after it is still bit-exact)."""
import time

import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import gf, synth

from gpu_util import dev, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _encode_ok():
    g = synth.choice(98)
    src = synth.random_bytes(g, (32, 600))
    coef = synth.coefficients(g, 8, (40, 32), nonzero=False)
    out = torch.zeros(40 * 600, dtype=torch.uint8, device=dev())
    gf.gf_encode_batched([(8, 32, 40, 600, to_dev(src.reshape(-1)), to_dev(coef.reshape(-1)), out)])
    torch.cuda.synchronize()
    return np.array_equal(to_host(out).reshape(40, 600), oracle.encode(8, src, coef))


def test_wait_that_nothing_ends_times_out():
    dev()
    lib = gf.load()
    assert lib.gf_device_status() == gf.GF_OK
    t0 = time.perf_counter()
    assert lib.gf_selftest_wait(0, None) == gf.GF_OK
    assert lib.gf_device_status() == gf.GF_ETIMEOUT  # waits for the kernel, then reads and clears the word
    took = time.perf_counter() - t0
    assert 0.5 < took < 30.0                          # the wait's limit is one second
    assert lib.gf_device_status() == gf.GF_OK
    assert _encode_ok()


def test_abort_flag_ends_a_wait_at_once():
    dev()
    lib = gf.load()
    t0 = time.perf_counter()
    assert lib.gf_selftest_wait(1, None) == gf.GF_OK
    assert lib.gf_device_status() == gf.GF_ETIMEOUT
    assert time.perf_counter() - t0 < 0.5
    assert _encode_ok()
