"""The C ABI library builds, loads without a GPU and exports every entry
point that include/gf.h declares; the binding declares them all too."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_boundary():
    names = _declared()
    for required in ("gf_region_madd", "gf_region_mul", "gf_encode_batched", "gf_decode_batched"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1909_02871_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1909_02871_gb300 import gf
    missing = [n for n in sorted(_declared()) if n not in gf._SIGS]
    assert not missing, missing


def test_host_side_errors_without_gpu():
    """Argument checks happen on the host before any CUDA call."""
    from paper_1909_02871_gb300 import gf
    lib = gf.load()
    assert lib.gf_region_madd(3, 16, 32, 1, 16, None) == gf.GF_EINVAL      # bad field
    assert lib.gf_region_madd(4, 16, 32, 16, 16, None) == gf.GF_EINVAL     # coef >= 2^n
    assert lib.gf_region_madd(8, 0, 32, 5, 16, None) == gf.GF_EINVAL       # NULL dst
    assert lib.gf_region_madd(8, 100, 108, 5, 16, None) == gf.GF_EOVERLAP  # partial overlap
    assert lib.gf_region_madd(8, 0, 0, 5, 0, None) == gf.GF_OK             # empty region
    assert lib.gf_region_mul(2, 100, 100, 4, 16, None) == gf.GF_EINVAL     # coef >= 4
    assert gf.strerror(gf.GF_EOVERLAP).startswith("GF_EOVERLAP")
    bad = gf.GfGen(5, 1, 1, 0, 16, 1, 1, 1)
    arr = (gf.GfGen * 1)(bad)
    assert lib.gf_encode_batched_ex(arr, 1, 0, None) == gf.GF_EINVAL
    dec = gf.GfDec(8, 2000, 1, 0, 16, 1, 1, 1, 1, 0, 0)  # n_src above the limit
    darr = (gf.GfDec * 1)(dec)
    assert lib.gf_decode_batched(darr, 1, None) == gf.GF_EINVAL


@pytest.mark.parametrize("n_gens", [0])
def test_empty_batches_are_noops(n_gens):
    from paper_1909_02871_gb300 import gf
    lib = gf.load()
    arr = (gf.GfGen * 1)()
    assert lib.gf_encode_batched_ex(arr, n_gens, 0, None) == gf.GF_OK
    darr = (gf.GfDec * 1)()
    assert lib.gf_decode_batched(darr, n_gens, None) == gf.GF_OK


def test_decoder_host_side_errors_without_gpu():
    """The resident-decoder entry points check their arguments first."""
    import ctypes
    from paper_1909_02871_gb300 import gf
    lib = gf.load()
    h = ctypes.c_void_p()
    assert lib.gf_dec_open(3, 16, 32, 100, ctypes.byref(h)) == gf.GF_EINVAL   # bad field
    assert lib.gf_dec_open(8, 0, 32, 100, ctypes.byref(h)) == gf.GF_EINVAL    # n_src < 1
    assert lib.gf_dec_open(8, 16, 5000, 100, ctypes.byref(h)) == gf.GF_EINVAL  # max_recv too large
    assert lib.gf_dec_open(8, 16, 32, 100, None) == gf.GF_EINVAL
    k = ctypes.c_int(7)
    assert lib.gf_dec_poll(None, -1, None, ctypes.byref(k)) == gf.GF_EINVAL and k.value == 0
    assert lib.gf_dec_poll(None, 0, None, ctypes.byref(k)) == gf.GF_OK and k.value == 0
    assert lib.gf_dec_status(None, 1, None, None, None) == gf.GF_EINVAL
    assert lib.gf_dec_push(None, None, None, 1, None) == gf.GF_EINVAL
    assert lib.gf_dec_close(None) == gf.GF_OK
    assert gf.strerror(gf.GF_EBUSY) != "unknown status"
