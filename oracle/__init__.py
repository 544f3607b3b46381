"""CPU oracle for GF(2^n) random linear network coding.

TEST INFRASTRUCTURE ONLY.  This package is the correctness authority for the
CUDA library: a plain, slow C implementation (``gf_oracle.c``) of the field
arithmetic of section II of Guenther, Appel and Carle, arXiv:1909.02871 (field
GF(2^n), addition = XOR, multiplication = polynomial product modulo a field
polynomial), the madd region operation (section II; Algorithms 1 and 2 of
section IV restated), the generation encode of Eq. 2 and a Gauss-Jordan decode.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference leg of ``bench.py`` may import it.  It shares no code with the CUDA
library and imports nothing from it; both sides only share the seeded input
generators, which hold none of the field arithmetic.

The C source is compiled on first use (``gcc -O2``) into ``oracle/_build/``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgf_oracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = (1, 2, 4, 8)


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def compile_source(source: str, path: str) -> str:
    """Compile C source text with the oracle's flags into a shared library at
    ``path`` (the planted-mistake tests compile altered copies of
    ``gf_oracle.c`` this way)."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", path, src])
    return path


def source() -> str:
    """Text of ``gf_oracle.c``."""
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def library(path: str):
    """Run every function of this module on another compiled copy of the
    oracle (a library built by ``compile_source``) inside the ``with`` block."""
    global _lib
    other = _configure(ctypes.CDLL(path))
    with _lock:
        saved, _lib = _lib, other
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _configure(lib):
    """Declare the argument and result types of the oracle's C functions."""
    u8p = ctypes.POINTER(ctypes.c_uint8)
    sz = ctypes.c_size_t
    lib.gfo_field_ok.argtypes = [ctypes.c_int]
    lib.gfo_poly.argtypes = [ctypes.c_int]
    lib.gfo_poly.restype = ctypes.c_uint
    lib.gfo_mul.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_uint]
    lib.gfo_mul.restype = ctypes.c_uint
    lib.gfo_inv.argtypes = [ctypes.c_int, ctypes.c_uint]
    lib.gfo_inv.restype = ctypes.c_uint
    lib.gfo_mul_table.argtypes = [ctypes.c_int, u8p]
    for name in ("gfo_region_madd", "gfo_region_mul", "gfo_madd_shuffle", "gfo_madd_imul"):
        getattr(lib, name).argtypes = [ctypes.c_int, u8p, u8p, ctypes.c_uint, sz]
    lib.gfo_encode.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, sz, u8p, u8p, u8p]
    lib.gfo_decode.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, sz, u8p, u8p, u8p,
                               u8p, ctypes.POINTER(ctypes.c_int)]
    lib.gfo_decode.restype = ctypes.c_int
    lib.gfo_recode.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, sz, u8p, u8p, u8p, u8p,
                               u8p]
    lib.gfo_recode.restype = None
    lib.gfo_rank.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p]
    lib.gfo_rank.restype = ctypes.c_int
    return lib


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"], "oracle takes contiguous uint8"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _check_field(n: int, c: int | None = None):
    if n not in FIELDS:
        raise ValueError(f"field must be one of {FIELDS}, got {n}")
    if c is not None and not (0 <= c < (1 << n)):
        raise ValueError(f"coefficient {c} is not an element of GF(2^{n})")


def poly(n: int) -> int:
    """Reduction polynomial of GF(2^n) (bit i = coefficient of x^i)."""
    _check_field(n)
    return int(_load().gfo_poly(n))


def mul(n: int, a: int, b: int) -> int:
    """Field product a*b in GF(2^n)."""
    _check_field(n)
    return int(_load().gfo_mul(n, a, b))


def inv(n: int, a: int) -> int:
    """Multiplicative inverse in GF(2^n) (0 maps to 0)."""
    _check_field(n)
    return int(_load().gfo_inv(n, a))


def mul_table(n: int) -> np.ndarray:
    """q x q multiplication table of GF(2^n)."""
    _check_field(n)
    q = 1 << n
    out = np.zeros((q, q), dtype=np.uint8)
    _load().gfo_mul_table(n, _u8(out))
    return out


def _region(fn: str, n: int, dst: np.ndarray, src: np.ndarray, c: int) -> np.ndarray:
    _check_field(n, c)
    dst = np.ascontiguousarray(dst, dtype=np.uint8).copy()
    src = np.ascontiguousarray(src, dtype=np.uint8)
    assert dst.size == src.size
    getattr(_load(), fn)(n, _u8(dst), _u8(src), c, dst.size)
    return dst


def region_madd(n: int, dst: np.ndarray, src: np.ndarray, c: int) -> np.ndarray:
    """Returns dst + c*src over GF(2^n) (section II madd); inputs untouched."""
    return _region("gfo_region_madd", n, dst, src, c)


def region_mul(n: int, src: np.ndarray, c: int) -> np.ndarray:
    """Returns c*src over GF(2^n)."""
    src = np.ascontiguousarray(src, dtype=np.uint8)
    return _region("gfo_region_mul", n, np.zeros_like(src), src, c)


def madd_shuffle(n: int, dst: np.ndarray, src: np.ndarray, c: int) -> np.ndarray:
    """madd by the shuffle algorithm (Algorithm 1, restated)."""
    return _region("gfo_madd_shuffle", n, dst, src, c)


def madd_imul(n: int, dst: np.ndarray, src: np.ndarray, c: int) -> np.ndarray:
    """madd by the imul algorithm (Algorithm 2, restated)."""
    return _region("gfo_madd_imul", n, dst, src, c)


def encode(n: int, src: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Eq. 2 for K coded packets: src is N x len, coef is K x N -> K x len."""
    src = np.ascontiguousarray(src, dtype=np.uint8)
    coef = np.ascontiguousarray(coef, dtype=np.uint8)
    N, L = src.shape
    K, N2 = coef.shape
    assert N == N2
    _check_field(n)
    if coef.size and int(coef.max()) >= (1 << n):
        raise ValueError("coefficient outside the field")
    out = np.zeros((K, L), dtype=np.uint8)
    _load().gfo_encode(n, N, K, L, _u8(src), _u8(coef), _u8(out))
    return out


def decode(n: int, coef: np.ndarray, payload: np.ndarray, n_src: int | None = None):
    """Gauss-Jordan decode of one generation.

    coef is R x N (received coding vectors in arrival order), payload R x len.
    Returns (out N x len, solved N bools, rank, used) where ``used`` counts
    the received rows consumed before the rank reached N.
    """
    coef = np.ascontiguousarray(coef, dtype=np.uint8)
    R, N = coef.shape
    if n_src is not None:
        assert n_src == N
    payload = np.ascontiguousarray(payload, dtype=np.uint8)
    if payload.ndim != 2:
        payload = payload.reshape(R, -1)
    assert payload.shape[0] == R
    L = payload.shape[1]
    _check_field(n)
    out = np.zeros((N, L), dtype=np.uint8)
    solved = np.zeros(N, dtype=np.uint8)
    used = ctypes.c_int(0)
    pay = payload if payload.size else np.zeros(1, dtype=np.uint8)
    rank = _load().gfo_decode(n, N, R, L, _u8(coef), _u8(pay), _u8(out) if out.size else _u8(np.zeros(1, np.uint8)),
                              _u8(solved) if solved.size else _u8(np.zeros(1, np.uint8)), ctypes.byref(used))
    if rank < 0:
        raise MemoryError("oracle decode: allocation failed")
    return out, solved.astype(bool), int(rank), int(used.value)


def rank(n: int, coef: np.ndarray) -> int:
    """Rank over GF(2^n) of an R x N coefficient matrix."""
    coef = np.ascontiguousarray(coef, dtype=np.uint8)
    R, N = coef.shape
    _check_field(n)
    return int(_load().gfo_rank(n, R, N, _u8(coef) if coef.size else _u8(np.zeros(1, np.uint8))))


def recode(n: int, coef_in: np.ndarray, payload_in: np.ndarray, mix: np.ndarray):
    """Recoding at an intermediate node: K2 new packets, each a combination
    (coefficients mix, K2 x R) of the R coded packets held (coef_in R x N,
    payload_in R x len).  Returns (coef_out K2 x N, payload_out K2 x len)."""
    coef_in = np.ascontiguousarray(coef_in, dtype=np.uint8)
    payload_in = np.ascontiguousarray(payload_in, dtype=np.uint8)
    mix = np.ascontiguousarray(mix, dtype=np.uint8)
    R, N = coef_in.shape
    K2, R2 = mix.shape
    assert R == R2 and payload_in.shape[0] == R
    L = payload_in.shape[1]
    _check_field(n)
    for a in (coef_in, mix):
        if a.size and int(a.max()) >= (1 << n):
            raise ValueError("coefficient outside the field")
    coef_out = np.zeros((K2, N), dtype=np.uint8)
    payload_out = np.zeros((K2, L), dtype=np.uint8)
    z = np.zeros(1, np.uint8)
    _load().gfo_recode(n, N, R, K2, L, _u8(coef_in) if coef_in.size else _u8(z),
                       _u8(payload_in) if payload_in.size else _u8(z), _u8(mix) if mix.size else _u8(z),
                       _u8(coef_out) if coef_out.size else _u8(z), _u8(payload_out) if payload_out.size else _u8(z))
    return coef_out, payload_out
