"""Seeded synthetic inputs for the network-coding workloads.

This module only draws random numbers: it holds none of the field arithmetic,
so both the CUDA library's tests/benchmarks and the CPU oracle can take their
inputs from it.  Every stream is a numpy PCG64 generator keyed by
``(190902871, workload id, item index)``.

Workloads (shapes of the random linear network coding setting of section II
of the paper: N source packets of M words, coding vectors drawn i.i.d. from
the field):

* ``region``        one contiguous region, uniform bytes, one random nonzero
                    coefficient;
* ``generation``    N = 16 source packets of 1500 B and a stream of coding
                    vectors (the first K are "the K coded packets", the rest
                    are extra packets sent while the receiver lacks rank N);
* ``uniform_batch`` G generations of N x len uniform bytes and K x N coding
                    matrices drawn from GF(q) minus zero;
* ``uneven_batch``  generations with N ~ U{8..255}, len log-uniform in
                    [64, 9000] B, field ~ U{GF(2), GF(4), GF(16), GF(256)},
                    coding vectors uniform over GF(q) and i.i.d. erasures;
* ``arrivals``      Poisson request arrival times for the serving loop.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field

import numpy as np

BASE_SEED = 190902871
FIELDS = (1, 2, 4, 8)

# workload ids used in the seeds
W_REGION, W_GENERATION, W_UNIFORM, W_UNEVEN, W_SERVE, W_MISC = 1, 2, 3, 4, 5, 9


def rng(*key: int) -> np.random.Generator:
    """Independent PCG64 stream for a key tuple."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED, *map(int, key)])))


def random_bytes(g: np.random.Generator, shape) -> np.ndarray:
    return g.integers(0, 256, size=shape, dtype=np.uint8)


def coefficients(g: np.random.Generator, field: int, shape, nonzero: bool) -> np.ndarray:
    """Field elements, one per byte, uniform over GF(2^field) (minus 0 if
    ``nonzero`` and the field has a nonzero element other than 1)."""
    q = 1 << field
    lo = 1 if (nonzero and q > 2) else 0
    return g.integers(lo, q, size=shape, dtype=np.uint8)


def region(length: int, field: int, index: int = 0):
    """(src, dst, coef) for one region op: uniform bytes, random nonzero c."""
    g = rng(W_REGION, field, length, index)
    src = random_bytes(g, length)
    dst = random_bytes(g, length)
    coef = int(g.integers(1, 1 << field)) if field > 1 else 1
    return src, dst, coef


@dataclass
class Generation:
    field: int
    src: np.ndarray          # N x len
    coef_stream: np.ndarray  # R x N (first K rows = the K coded packets)
    n_coded: int

    @property
    def n_src(self) -> int:
        return self.src.shape[0]

    @property
    def length(self) -> int:
        return self.src.shape[1]


def generation(field: int, n_src: int = 16, length: int = 1500, n_coded: int = 16,
               extra: int = 48, index: int = 0) -> Generation:
    """Single generation: the source bytes depend only on (n_src, length,
    index), so every field codes the same bytes; coding vectors are uniform
    over GF(q) minus 0 (GF(2): over GF(2), since its only nonzero element
    would make every coded packet identical)."""
    gs = rng(W_GENERATION, n_src, length, index)
    src = random_bytes(gs, (n_src, length))
    gc = rng(W_GENERATION, 1000 + field, n_src, index)
    coef = coefficients(gc, field, (n_coded + extra, n_src), nonzero=True)
    return Generation(field, src, coef, n_coded)


@dataclass
class UniformBatch:
    field: int
    src: np.ndarray   # G x N x len
    coef: np.ndarray  # G x K x N


def uniform_batch(n_gens: int = 4096, n_src: int = 64, length: int = 1500, n_coded: int = 64,
                  field: int = 8, index: int = 0) -> UniformBatch:
    """Batched uniform encode: uniform source bytes and coding matrices
    uniform over GF(q) minus 0."""
    g = rng(W_UNIFORM, n_gens, n_src, length, n_coded, field, index)
    src = random_bytes(g, (n_gens, n_src, length))
    coef = coefficients(g, field, (n_gens, n_coded, n_src), nonzero=True)
    return UniformBatch(field, src, coef)


@dataclass
class UnevenGen:
    field: int
    src: np.ndarray          # N x len
    coef_stream: np.ndarray  # S x N: coding vectors of the packets the sender may send
    erased: np.ndarray       # S bools: packet lost on the way

    @property
    def n_src(self) -> int:
        return self.src.shape[0]

    @property
    def length(self) -> int:
        return self.src.shape[1]


@dataclass
class UnevenBatch:
    gens: list = dc_field(default_factory=list)


def uneven_stream_len(n_src: int, loss: float) -> int:
    """Length of the coding-vector stream drawn per generation: enough
    packets that, after losses, the receiver sees N + 40 rows with a wide
    margin (a stream this long fails to reach rank N with negligible
    probability)."""
    return int(np.ceil((n_src + 40) / (1.0 - loss) * 1.15)) + 8


def uneven_batch(n_gens: int = 2048, n_min: int = 8, n_max: int = 255, len_min: int = 64,
                 len_max: int = 9000, loss: float = 0.10, index: int = 0,
                 fields=FIELDS) -> UnevenBatch:
    """Uneven batch: per generation N ~ U{n_min..n_max}, len log-uniform in
    [len_min, len_max] bytes, field ~ U(fields), coding vectors uniform over
    GF(q) (zero included), i.i.d. erasures with probability ``loss``."""
    g = rng(W_UNEVEN, n_gens, n_min, n_max, len_min, len_max, int(loss * 1000), index)
    out = UnevenBatch()
    for _ in range(n_gens):
        fld = int(fields[int(g.integers(0, len(fields)))])
        n = int(g.integers(n_min, n_max + 1))
        length = int(np.round(np.exp(g.uniform(np.log(len_min), np.log(len_max)))))
        s = uneven_stream_len(n, loss)
        src = random_bytes(g, (n, length))
        coef = coefficients(g, fld, (s, n), nonzero=False)
        erased = g.random(s) < loss
        out.gens.append(UnevenGen(fld, src, coef, erased))
    return out


def erasures(n: int, loss: float, *key: int) -> np.ndarray:
    """n i.i.d. packet losses with probability ``loss`` (True = lost)."""
    g = rng(W_MISC, 77, n, int(loss * 1000), *key)
    return g.random(n) < loss


def systematic_stream(coef_stream: np.ndarray) -> np.ndarray:
    """A systematic sender's coding vectors: the N unit vectors (the sources
    sent uncoded, in order) followed by the coded packets' vectors."""
    n = coef_stream.shape[1]
    return np.concatenate([np.eye(n, dtype=np.uint8), coef_stream])


def arrivals(rate_per_s: float, n: int, index: int = 0) -> np.ndarray:
    """Poisson arrival times (seconds from 0) of n requests."""
    g = rng(W_SERVE, int(rate_per_s * 1000), n, index)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def choice(index: int, *key: int) -> np.random.Generator:
    """Generic stream for tests that need their own random draws."""
    return rng(W_MISC, index, *key)
