"""Planted mistakes in the oracle.

Each case compiles a copy of the oracle's C source with one plausible mistake
(a reducible or non-primitive field polynomial, a dropped or misplaced
reduction step, partial products ORed instead of XORed, a misplaced word, a
transposed coding matrix, a missing step of the elimination, ...) and runs
the committed pins of test_oracle_field, test_oracle_region and
test_oracle_codec against it: at least one pin must fail.  A control copy
without a mistake passes every one of them, so a failure is the mistake's
doing.  The two pins that restate the reading polynomials are left out, so
that the polynomial mistakes have to be caught by the mathematics (field
axioms, primitivity of x, the textbook powers of x in tests/golden/)."""
import functools
import itertools

import pytest

import oracle
import test_oracle_codec
import test_oracle_field
import test_oracle_region

RESTATEMENTS = {"test_reading_polynomials", "test_mul_by_x_is_shift_and_reduce"}
# the pins that take seconds run last (most mistakes are caught before them)
SLOW = {"test_field_axioms_exhaustive", "test_madd_agrees_with_shuffle_and_imul_every_byte_every_coef",
        "test_full_rank_probability"}


def _pin_calls():
    calls = []
    for mod in (test_oracle_field, test_oracle_region, test_oracle_codec):
        for name, fn in vars(mod).items():
            if not name.startswith("test_") or not callable(fn) or name in RESTATEMENTS:
                continue
            grids = []
            for mark in getattr(fn, "pytestmark", []):
                if mark.name != "parametrize":
                    continue
                names, values = mark.args[0], mark.args[1]
                names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
                grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in values])
            for combo in itertools.product(*grids):
                kw = {}
                for d in combo:
                    kw.update(d)
                slow = name in SLOW and kw.get("n", 0) == 8 or name == "test_full_rank_probability"
                calls.append((slow, f"{name}{kw}", functools.partial(fn, **kw)))
    calls.sort(key=lambda c: c[0])
    return [(label, call) for _, label, call in calls]


PINS = _pin_calls()

# (name, text in gf_oracle.c, replacement); each text occurs exactly once
MISTAKES = [
    ("gf4 polynomial reducible (x^2+1)", "case 2: return 0x7;", "case 2: return 0x5;"),
    ("gf16 polynomial another primitive one (x^4+x^3+1)", "case 4: return 0x13;", "case 4: return 0x19;"),
    ("gf256 polynomial irreducible but not primitive (0x11B)", "case 8: return 0x11D;", "case 8: return 0x11B;"),
    ("reduction stops one degree early", "for (d = 2 * n - 2; d >= n; d--)", "for (d = 2 * n - 2; d > n; d--)"),
    ("reduction starts one degree low", "for (d = 2 * n - 2; d >= n; d--)", "for (d = 2 * n - 3; d >= n; d--)"),
    ("partial products ORed", "prod ^= a << i;", "prod |= a << i;"),
    ("reduction subtracts", "prod ^= p << (d - n);", "prod -= p << (d - n);"),
    ("inverse returns the element", "if (gfo_mul(n, a, b) == 1)\n            return b;",
     "if (gfo_mul(n, a, b) == 1)\n            return a;"),
    ("madd word misplaced", "acc ^= gfo_mul(n, c, w) << (j * n);", "acc ^= gfo_mul(n, c, w) << j;"),
    ("mul keeps the old destination bits", "unsigned byte = src[k], res = 0;",
     "unsigned byte = src[k], res = dst[k];"),
    ("shuffle nibble tables swapped", "(uint8_t)(tl[src[k] & 15u] ^ th[src[k] >> 4])",
     "(uint8_t)(tl[src[k] >> 4] ^ th[src[k] & 15u])"),
    ("imul multipliers are powers of c, not c*x^i", "p[i] = gfo_mul(n, c, 1u << i);",
     "p[i] = i ? gfo_mul(n, p[i - 1], c) : c;"),
    ("encode reads the coding matrix transposed", "coef[(size_t)k * N + i]", "coef[(size_t)i * K + k]"),
    ("decode leaves the payload out of the elimination",
     "gfo_region_madd(n, cur + N, rows + (size_t)s * width + N, f, len);", ";"),
    ("decode skips back-substitution", "f = row[pivot];", "f = 0;"),
    ("decode normalises by the pivot, not its inverse", "f = gfo_inv(n, cur[pivot]);", "f = cur[pivot];"),
    ("decode pivot is the first zero", "if (cur[col] != 0) { pivot = col; break; }",
     "if (cur[col] == 0) { pivot = col; break; }"),
    ("decode does not stop at rank N", "for (r = 0; r < R && rank < N; r++)", "for (r = 0; r < R; r++)"),
    ("decode reports every pivot row as solved", "{ unit = 0; break; }", "{ break; }"),
    ("recode composes the vectors transposed", "coef_in[(size_t)r * N + i]", "coef_in[(size_t)i * R + r]"),
    # off by one at a loop boundary
    ("madd skips the last byte", "    for (k = 0; k < len; k++) {\n        unsigned byte = src[k], acc = dst[k];",
     "    for (k = 0; k + 1 < len; k++) {\n        unsigned byte = src[k], acc = dst[k];"),
    ("madd skips the last word of a byte",
     "for (j = 0; j < words; j++) {\n            unsigned w = (byte >> (j * n)) & mask;\n            acc ^=",
     "for (j = 0; j + 1 < words; j++) {\n            unsigned w = (byte >> (j * n)) & mask;\n            acc ^="),
    ("imul restatement drops the last tail byte", "    for (; k < len; k++) {", "    for (; k + 1 < len; k++) {"),
    ("encode skips the last source", "        for (i = 0; i < N; i++)\n            gfo_region_madd(n, acc, src",
     "        for (i = 0; i + 1 < N; i++)\n            gfo_region_madd(n, acc, src"),
    ("recode skips the last held packet", "            for (r = 0; r < R; r++)\n                acc ^= gfo_mul(n, mix",
     "            for (r = 0; r + 1 < R; r++)\n                acc ^= gfo_mul(n, mix"),
]


def _first_failing_pin(lib):
    with oracle.library(lib):
        for label, call in PINS:
            try:
                call()
            except Exception:  # an assertion, or the oracle's own range check tripping
                return label
    return None


def test_pins_were_collected():
    names = {label.split("{")[0] for label, _ in PINS}
    assert {"test_field_axioms_exhaustive", "test_gf256_powers_golden", "test_round_trip_single_generation",
            "test_madd_agrees_with_shuffle_and_imul_every_byte_every_coef"} <= names


def test_control_copy_passes_every_pin(tmp_path):
    lib = oracle.compile_source(oracle.source(), str(tmp_path / "control.so"))
    assert _first_failing_pin(lib) is None


@pytest.mark.parametrize("name,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    src = oracle.source()
    assert src.count(old) == 1, f"the text to alter must occur exactly once: {old!r}"
    lib = oracle.compile_source(src.replace(old, new), str(tmp_path / "mutant.so"))
    assert _first_failing_pin(lib) is not None, f"no pin fails with the mistake: {name}"
