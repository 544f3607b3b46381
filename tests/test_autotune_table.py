"""The autotuner's table of path choices, through the C ABI, on the host.

Tuned choices are kept per shape bucket (field, and the powers of two at or
above n_src, n_coded and len); gf_autotune_query returns the tuned choice of
the bucket, else the built-in rule.  Setting, clearing, saving and loading the
table are host operations, so they are checked here without a GPU (where no
tensor-core device is present the built-in rule picks the table path)."""
import pytest

from paper_1909_02871_gb300 import gf


@pytest.fixture(autouse=True)
def _empty_table():
    gf.gf_autotune_clear()
    yield
    gf.gf_autotune_clear()


def _rule(field, n_src, n_coded, length):
    gf.gf_autotune_clear()
    return gf.gf_autotune_query(field, n_src, n_coded, length)


def test_set_choice_covers_its_bucket():
    default = _rule(8, 64, 64, 1500)
    gf.gf_autotune_set(8, 64, 64, 1500, gf.PATH_TABLE, 2)
    assert gf.gf_autotune_query(8, 64, 64, 1500) == (gf.PATH_TABLE, 2)
    # same buckets: n_src 33..64, n_coded 33..64, len 1025..2048
    assert gf.gf_autotune_query(8, 40, 60, 1100) == (gf.PATH_TABLE, 2)
    assert gf.gf_autotune_query(8, 33, 33, 2048) == (gf.PATH_TABLE, 2)
    # neighbouring buckets and other fields fall back to the rule
    for shape in [(8, 65, 64, 1500), (8, 64, 32, 1500), (8, 64, 64, 1024), (4, 64, 64, 1500)]:
        gf.gf_autotune_set(8, 64, 64, 1500, gf.PATH_TABLE, 2)
        got = gf.gf_autotune_query(*shape)
        assert got == _rule(*shape), shape
    assert default == _rule(8, 64, 64, 1500)


def test_later_setting_replaces_earlier():
    gf.gf_autotune_set(2, 100, 100, 9000, gf.PATH_TABLE, 1)
    gf.gf_autotune_set(2, 128, 128, 16384, gf.PATH_BITSLICED, 0)  # the same bucket
    assert gf.gf_autotune_query(2, 100, 100, 9000) == (gf.PATH_BITSLICED, 0)


def test_save_clear_load_round_trip(tmp_path):
    choices = {(8, 64, 64, 1500): (gf.PATH_TABLE, 3), (1, 16, 16, 128): (gf.PATH_BITSLICED, 0),
               (4, 255, 300, 9000): (gf.PATH_TABLE, 1)}
    for (f, n, k, l), (p, v) in choices.items():
        gf.gf_autotune_set(f, n, k, l, p, v)
    path = str(tmp_path / "tune.txt")
    gf.gf_autotune_save(path)
    gf.gf_autotune_clear()
    for shape in choices:
        assert gf.gf_autotune_query(*shape) == _rule(*shape)
    gf.gf_autotune_load(path)
    for shape, choice in choices.items():
        assert gf.gf_autotune_query(*shape) == choice


def test_load_skips_invalid_lines(tmp_path):
    path = tmp_path / "tune.txt"
    # bucket exponents: field n_src n_coded len; then path and variant
    path.write_text("8 6 6 11 1 2\n"        # valid: table, variant 2
                    "3 6 6 11 1 0\n"        # no such field
                    "8 5 5 10 7 0\n"        # no such path
                    "8 4 4 9 1 99\n"        # no such variant
                    "garbage\n")
    gf.gf_autotune_load(str(path))
    assert gf.gf_autotune_query(8, 64, 64, 1500) == (gf.PATH_TABLE, 2)
    assert gf.gf_autotune_query(8, 32, 32, 1000) == _rule(8, 32, 32, 1000)


def test_invalid_settings_are_rejected():
    lib = gf.load()
    assert lib.gf_autotune_set(3, 64, 64, 1500, gf.PATH_TABLE, 0) == gf.GF_EINVAL      # field
    assert lib.gf_autotune_set(8, 64, 64, 1500, gf.PATH_AUTO, 0) == gf.GF_EINVAL       # AUTO is not a choice
    assert lib.gf_autotune_set(8, 64, 64, 1500, gf.PATH_TABLE, 99) == gf.GF_EINVAL     # variant
    assert lib.gf_autotune_load(b"/nonexistent/tune.txt") == gf.GF_EINVAL
    assert lib.gf_autotune_save(None) == gf.GF_EINVAL
