"""Thin ctypes binding of ``libgf_gb300.so`` (declared in ``include/gf.h``).

Argument marshalling only: every function takes torch CUDA tensors (or raw
device addresses), passes their addresses, sizes and the current CUDA stream
to the C entry point of the same name, and raises :class:`GFError` on a
nonzero status.  All arithmetic runs in the library's CUDA kernels; there is
no fallback.  The library is loaded (and built if missing) on first use and
loading fails loudly when it cannot be built or opened.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

GF_OK, GF_EINVAL, GF_EOVERLAP, GF_ENOMEM, GF_ERANK, GF_ETIMEOUT, GF_ECUDA, GF_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
GF_EBUSY = -8
DEC_SYSTEMATIC = 1
PATH_AUTO, PATH_TABLE, PATH_BITSLICED = 0, 1, 2

_lock = threading.Lock()
_lib = None


class GFError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status} ({strerror(status) if _lib else status})")


class GfGen(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int32), ("n_src", ctypes.c_int32), ("n_coded", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("len", ctypes.c_uint64), ("src", ctypes.c_void_p),
                ("coef", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class GfRecode(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int32), ("n_src", ctypes.c_int32), ("n_in", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("len", ctypes.c_uint64), ("coef_in", ctypes.c_void_p),
                ("payload_in", ctypes.c_void_p), ("mix", ctypes.c_void_p), ("coef_out", ctypes.c_void_p),
                ("payload_out", ctypes.c_void_p)]


class GfDec(ctypes.Structure):
    _fields_ = [("field", ctypes.c_int32), ("n_src", ctypes.c_int32), ("n_recv", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("len", ctypes.c_uint64), ("coef", ctypes.c_void_p),
                ("payload", ctypes.c_void_p), ("out", ctypes.c_void_p), ("rank", ctypes.c_void_p),
                ("used", ctypes.c_void_p), ("solved", ctypes.c_void_p)]


# name -> (restype, argtypes)
_SIGS = {
    "gf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gf_version": (ctypes.c_int, []),
    "gf_region_madd": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint8,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    "gf_region_mul": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint8,
                                     ctypes.c_size_t, ctypes.c_void_p]),
    "gf_encode_batched": (ctypes.c_int, [ctypes.POINTER(GfGen), ctypes.c_int, ctypes.c_void_p]),
    "gf_encode_batched_ex": (ctypes.c_int, [ctypes.POINTER(GfGen), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "gf_encode_validate": (ctypes.c_int, [ctypes.POINTER(GfGen), ctypes.c_int, ctypes.c_void_p]),
    "gf_decode_batched": (ctypes.c_int, [ctypes.POINTER(GfDec), ctypes.c_int, ctypes.c_void_p]),
    "gf_decode_check": (ctypes.c_int, [ctypes.POINTER(GfDec), ctypes.c_int, ctypes.c_void_p]),
    "gf_decode_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "gf_encode_plan_create": (ctypes.c_int, [ctypes.POINTER(GfGen), ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "gf_decode_plan_create": (ctypes.c_int, [ctypes.POINTER(GfDec), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "gf_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gf_plan_kernel_count": (ctypes.c_int, [ctypes.c_void_p]),
    "gf_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gf_autotune_encode": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "gf_autotune_last": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]),
    "gf_autotune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_int]),
    "gf_autotune_query": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gf_autotune_clear": (ctypes.c_int, []),
    "gf_autotune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "gf_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "gf_device_status": (ctypes.c_int, []),
    "gf_selftest_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "gf_dec_open": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "gf_dec_push": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "gf_dec_poll": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_int)]),
    "gf_dec_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p)]),
    "gf_dec_close": (ctypes.c_int, [ctypes.c_void_p]),
    "gf_recode_batched": (ctypes.c_int, [ctypes.POINTER(GfRecode), ctypes.c_int, ctypes.c_void_p]),
    "gf_recode_plan_create": (ctypes.c_int, [ctypes.POINTER(GfRecode), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "gf_dec_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(status: int) -> str:
    return load().gf_strerror(status).decode()


def _check(status: int, where: str) -> int:
    if status != GF_OK:
        raise GFError(status, where)
    return status


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _nbytes(t) -> int:
    return int(t.numel() * t.element_size())


# ----------------------------------------------------------------------------
# region operations
# ----------------------------------------------------------------------------
def gf_region_madd(field: int, dst, src, coef: int, length: int | None = None, stream=None) -> None:
    """dst += coef * src over GF(2^field) (device tensors or addresses)."""
    n = _nbytes(dst) if length is None else int(length)
    _check(load().gf_region_madd(field, _ptr(dst), _ptr(src), coef, n, _stream(stream)), "gf_region_madd")


def gf_region_mul(field: int, dst, src, coef: int, length: int | None = None, stream=None) -> None:
    """dst = coef * src over GF(2^field)."""
    n = _nbytes(dst) if length is None else int(length)
    _check(load().gf_region_mul(field, _ptr(dst), _ptr(src), coef, n, _stream(stream)), "gf_region_mul")


def region_status(fn: str, field: int, dst, src, coef: int, length: int, stream=None) -> int:
    """Raw status of a region call (for error-path tests)."""
    return getattr(load(), fn)(field, _ptr(dst), _ptr(src), coef, length, _stream(stream))


# ----------------------------------------------------------------------------
# batched encode / decode
# ----------------------------------------------------------------------------
def make_gens(items) -> ctypes.Array:
    """items: iterable of (field, n_src, n_coded, len, src, coef, out)."""
    items = list(items)
    arr = (GfGen * max(1, len(items)))()
    for i, (field, n_src, n_coded, length, src, coef, out) in enumerate(items):
        arr[i] = GfGen(field, n_src, n_coded, 0, length, _ptr(src), _ptr(coef), _ptr(out))
    return arr, len(items)


def make_decs(items) -> ctypes.Array:
    """items: iterable of (field, n_src, n_recv, len, coef, payload, out, rank, used, solved[, flags])."""
    items = list(items)
    arr = (GfDec * max(1, len(items)))()
    for i, it in enumerate(items):
        field, n_src, n_recv, length, coef, payload, out, rank, used, solved = it[:10]
        flags = it[10] if len(it) > 10 else 0
        arr[i] = GfDec(field, n_src, n_recv, flags, length, _ptr(coef), _ptr(payload), _ptr(out), _ptr(rank),
                       _ptr(used), _ptr(solved))
    return arr, len(items)


def gf_encode_batched(gens, path: int = PATH_AUTO, stream=None) -> None:
    arr, n = gens if isinstance(gens, tuple) else make_gens(gens)
    _check(load().gf_encode_batched_ex(arr, n, path, _stream(stream)), "gf_encode_batched")


def gf_encode_validate(gens, stream=None) -> int:
    arr, n = gens if isinstance(gens, tuple) else make_gens(gens)
    return load().gf_encode_validate(arr, n, _stream(stream))


def encode_status(gens, path: int = PATH_AUTO, stream=None) -> int:
    arr, n = gens if isinstance(gens, tuple) else make_gens(gens)
    return load().gf_encode_batched_ex(arr, n, path, _stream(stream))


def make_recodes(items):
    """items: iterable of (field, n_src, n_in, n_out, len, coef_in, payload_in, mix, coef_out, payload_out)."""
    items = list(items)
    arr = (GfRecode * max(1, len(items)))()
    for i, (field, n_src, n_in, n_out, length, ci, pi, mix, co, po) in enumerate(items):
        arr[i] = GfRecode(field, n_src, n_in, n_out, length, _ptr(ci), _ptr(pi), _ptr(mix), _ptr(co), _ptr(po))
    return arr, len(items)


def gf_recode_batched(items, stream=None) -> None:
    arr, n = items if isinstance(items, tuple) else make_recodes(items)
    _check(load().gf_recode_batched(arr, n, _stream(stream)), "gf_recode_batched")


def gf_decode_batched(decs, stream=None) -> None:
    arr, n = decs if isinstance(decs, tuple) else make_decs(decs)
    _check(load().gf_decode_batched(arr, n, _stream(stream)), "gf_decode_batched")


def decode_status(decs, stream=None) -> int:
    arr, n = decs if isinstance(decs, tuple) else make_decs(decs)
    return load().gf_decode_batched(arr, n, _stream(stream))


def gf_decode_check(decs, stream=None) -> int:
    arr, n = decs if isinstance(decs, tuple) else make_decs(decs)
    return load().gf_decode_check(arr, n, _stream(stream))


def gf_decode_noalloc(field: int, n_src: int, n_recv: int, length: int, coef, payload, out, rank, used=None,
                      solved=None, stream=None) -> int:
    """Single-generation decode that allocates nothing (scratch in a fixed
    device array of the library); returns the raw status."""
    return int(load().gf_decode_noalloc(field, n_src, n_recv, length, _ptr(coef), _ptr(payload), _ptr(out),
                                        _ptr(rank), _ptr(used), _ptr(solved), _stream(stream)))


class Decoder:
    """Owner of a gf_decoder_t: one generation's received packets resident in
    library-owned device memory (gf_dec_open ... gf_dec_close)."""

    def __init__(self, field: int, n_src: int, max_recv: int, length: int):
        h = ctypes.c_void_p()
        _check(load().gf_dec_open(field, n_src, max_recv, length, ctypes.byref(h)), "gf_dec_open")
        self.handle = h.value
        self.field, self.n_src, self.max_recv, self.length = field, n_src, max_recv, length

    def push(self, coef, payload, n: int, stream=None) -> None:
        """Append n packets (coef n x n_src, payload n x len; tensors on the
        host (pinned) or the device, or raw addresses)."""
        _check(load().gf_dec_push(self.handle, _ptr(coef), _ptr(payload), n, _stream(stream)), "gf_dec_push")

    @staticmethod
    def poll(decoders, stream=None) -> int:
        """One batched decode over every decoder with new packets and at least
        n_src of them; returns how many were attempted."""
        arr = (ctypes.c_void_p * max(len(decoders), 1))(*[d.handle for d in decoders])
        k = ctypes.c_int()
        _check(load().gf_dec_poll(arr, len(decoders), _stream(stream), ctypes.byref(k)), "gf_dec_poll")
        return k.value

    def status(self, wait: bool = True):
        """(rank, received, device address of the decoded packets), or None
        while the latest attempt is still running (wait=False)."""
        r, n, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
        st = load().gf_dec_status(self.handle, 1 if wait else 0, ctypes.byref(r), ctypes.byref(n), ctypes.byref(o))
        if st == GF_EBUSY:
            return None
        _check(st, "gf_dec_status")
        return r.value, n.value, o.value

    def read(self, dst, stream=None) -> None:
        """Enqueue a copy of the n_src x len decoded packets into dst (tensor
        on the host, pinned, or the device)."""
        _check(load().gf_dec_read(self.handle, _ptr(dst), _stream(stream)), "gf_dec_read")

    def close(self) -> None:
        if self.handle:
            h, self.handle = self.handle, None
            _check(load().gf_dec_close(h), "gf_dec_close")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owner of a gf_plan_t (pre-uploaded batch, launchable inside stream capture)."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = handle
        self._keep = keepalive

    @classmethod
    def encode(cls, gens, path: int = PATH_AUTO) -> "Plan":
        arr, n = gens if isinstance(gens, tuple) else make_gens(gens)
        h = ctypes.c_void_p()
        _check(load().gf_encode_plan_create(arr, n, path, ctypes.byref(h)), "gf_encode_plan_create")
        return cls(h.value, arr)

    @classmethod
    def recode(cls, items) -> "Plan":
        arr, n = items if isinstance(items, tuple) else make_recodes(items)
        h = ctypes.c_void_p()
        _check(load().gf_recode_plan_create(arr, n, ctypes.byref(h)), "gf_recode_plan_create")
        return cls(h.value, arr)

    @classmethod
    def decode(cls, decs) -> "Plan":
        arr, n = decs if isinstance(decs, tuple) else make_decs(decs)
        h = ctypes.c_void_p()
        _check(load().gf_decode_plan_create(arr, n, ctypes.byref(h)), "gf_decode_plan_create")
        return cls(h.value, arr)

    def launch(self, stream=None) -> None:
        _check(load().gf_plan_launch(self.handle, _stream(stream)), "gf_plan_launch")

    @property
    def kernel_count(self) -> int:
        return int(load().gf_plan_kernel_count(self.handle))

    def close(self) -> None:
        if self.handle:
            load().gf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# autotuner / status
# ----------------------------------------------------------------------------
def gf_autotune_encode(field: int, n_src: int, n_coded: int, length: int, n_gens: int, stream=None):
    p, v = ctypes.c_int(), ctypes.c_int()
    _check(load().gf_autotune_encode(field, n_src, n_coded, length, n_gens, _stream(stream), ctypes.byref(p),
                                     ctypes.byref(v)), "gf_autotune_encode")
    return p.value, v.value


def gf_autotune_last():
    """[(path, variant, mean ms)] of the candidates this thread's last
    gf_autotune_encode call timed."""
    n = ctypes.c_int()
    _check(load().gf_autotune_last(0, None, None, None, ctypes.byref(n)), "gf_autotune_last")
    k = n.value
    paths, variants, ms = (ctypes.c_int * max(k, 1))(), (ctypes.c_int * max(k, 1))(), (ctypes.c_float * max(k, 1))()
    _check(load().gf_autotune_last(k, paths, variants, ms, ctypes.byref(n)), "gf_autotune_last")
    return [(paths[i], variants[i], float(ms[i])) for i in range(k)]


def gf_autotune_set(field: int, n_src: int, n_coded: int, length: int, path: int, variant: int) -> None:
    _check(load().gf_autotune_set(field, n_src, n_coded, length, path, variant), "gf_autotune_set")


def gf_autotune_query(field: int, n_src: int, n_coded: int, length: int):
    p, v = ctypes.c_int(), ctypes.c_int()
    _check(load().gf_autotune_query(field, n_src, n_coded, length, ctypes.byref(p), ctypes.byref(v)),
           "gf_autotune_query")
    return p.value, v.value


def gf_autotune_clear() -> None:
    load().gf_autotune_clear()


def gf_autotune_save(path: str) -> None:
    _check(load().gf_autotune_save(os.fsencode(path)), "gf_autotune_save")


def gf_autotune_load(path: str) -> None:
    _check(load().gf_autotune_load(os.fsencode(path)), "gf_autotune_load")


def gf_device_status() -> int:
    return int(load().gf_device_status())
