"""Plant plausible mistakes in copies of the oracle source and check that the
pins of ``test_oracle.py`` reject every one of them.  This is what makes the
pins trustworthy: a dropped term, a wrong index, a transposed bit order or a
flipped parity sense in the oracle cannot slip through."""
import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_oracle as pins
from tests import test_oracle_secded as secded_pins
from tests import test_oracle_short as short_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hd_oracle.c")

MUTANTS = {
    "zero_indexed_positions": ("s ^= p;", "s ^= p - 1u;"),
    "flip_off_by_one": ("bit[s] ^= 1u;", "bit[s < n ? s + 1 : s] ^= 1u;"),
    "no_correction": ("bit[s] ^= 1u;", ";"),
    "data_order_reversed": ("put_bit(out_bits, i * k + d, bit[p]);",
                            "put_bit(out_bits, i * k + (k - 1 - d), bit[p]);"),
    "wrong_checksum_positions": ("return p != 0 && (p & (p - 1u)) == 0;",
                                 "return p != 0 && (p & (p + 1u)) == 0;"),
    "odd_parity_encoder": ("bit[1u << j] = (unsigned char)((s >> j) & 1u);",
                           "bit[1u << j] = (unsigned char)(((s >> j) & 1u) ^ 1u);"),
    "msb_first_reads": ("return (int)((w[b >> 5] >> (b & 31u)) & 1u);",
                        "return (int)((w[b >> 5] >> (31u - (b & 31u))) & 1u);"),
    "count_every_codeword": ("if (s != 0) {", "if (s != 0 || 1) {"),
    "u8_syndrome_truncated": ("((uint8_t *)syndromes)[i] = (uint8_t)s;",
                              "((uint8_t *)syndromes)[i] = (uint8_t)(s & 0x7Fu);"),
    "adjacent_data_bits_swapped": ("put_bit(out_bits, i * k + d, bit[p]);",
                                   "put_bit(out_bits, i * k + ((d ^ 1u) < k ? (d ^ 1u) : d), bit[p]);"),
}

# Mistakes in the shortened-code functions, caught by the pins of
# ``test_oracle_short.py``.
SHORT_MUTANTS = {
    "short_r_too_small": ("while ((1u << r) < n + 1u) ++r;", "while ((1u << r) < n) ++r;"),
    "short_flip_past_length": ("if (s <= n)\n                bit[s] ^= 1u; /* names a position",
                               "if (1)\n                bit[s] ^= 1u; /* names a position"),
    "short_detect_not_counted": ("++de; /* names no position", "; /* names no position"),
    "short_odd_parity_encoder": ("bit[1u << j] = (unsigned char)(1u & (s >> j));",
                                 "bit[1u << j] = (unsigned char)(1u & ~(s >> j));"),
    "short_last_position_skipped": ("for (uint32_t p = 1; p <= n; ++p)\n            if (bit[p]) s ^= p;\n        if (s != 0) {",
                                    "for (uint32_t p = 1; p < n; ++p)\n            if (bit[p]) s ^= p;\n        if (s != 0) {"),
}


def _pin_suite(o):
    """Run the pins against oracle ``o``; return the names of those that fail."""
    checks = [
        ("index_sets", lambda: pins.test_index_sets_match_paper(o)),
        ("worked_7_4", lambda: pins.test_worked_example_7_4(o)),
        ("brute_7", lambda: pins.test_bruteforce_single_and_double_errors(o, 7)),
        ("parity_check_63", lambda: pins.test_syndrome_equals_parity_check(o, 63)),
        ("perfect_15", lambda: pins.test_perfect_code_property(o, 15)),
        ("err_events_255", lambda: pins.test_err_count_equals_injected_events(o, 255)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:  # an assertion or a decode error both reject the mutant
            failed.append(name)
    return failed


# Mistakes in the SECDED functions, caught by the pins of ``test_oracle_secded.py``.
SECDED_MUTANTS = {
    "secded_parity_skips_position_0": ("        for (uint32_t p = 0; p <= n; ++p) {\n            if (bit[p]) {\n                s ^= p;\n                par ^= 1u;",
                                       "        for (uint32_t p = 1; p <= n; ++p) {\n            if (bit[p]) {\n                s ^= p;\n                par ^= 1u;"),
    "secded_corrects_double_errors": ("        if (par)\n            bit[s] ^= 1u; /* one error",
                                      "        if (par || s)\n            bit[s] ^= 1u; /* one error"),
    "secded_detects_on_odd_parity": ("        else if (s != 0)\n            ++de; /* two errors",
                                     "        if (s != 0)\n            ++de; /* two errors"),
    "secded_encoder_parity_of_data_only": ("        for (uint32_t p = 1; p <= n; ++p) par ^= bit[p];",
                                           "        for (uint32_t p = 3; p <= n; ++p) par ^= (p & (p - 1u)) ? bit[p] : 0u;"),
    "secded_syndrome_without_parity_bit": ("        uint32_t v = s | (par << m);", "        uint32_t v = s;"),
}


def _secded_pin_suite(o):
    checks = [
        ("brute_7", lambda: secded_pins.test_secded_bruteforce(o, 7)),
        ("relation_31", lambda: secded_pins.test_secded_relation_to_single_error_decoder(o, 31)),
        ("matrix_63", lambda: secded_pins.test_secded_matrix_form(o, 63)),
        ("events", lambda: secded_pins.test_secded_injected_events(o)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(name)
    return failed


@pytest.mark.parametrize("name", sorted(SECDED_MUTANTS))
def test_secded_mutant_is_caught(tmp_path, name):
    old, new = SECDED_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique: {old}"
    src = tmp_path / "hd_oracle.c"
    src.write_text(text.replace(old, new, 1))
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "lib.so"))
    assert _secded_pin_suite(oracle.Oracle(lib)), f"mutant {name} passed every pin"


def _short_pin_suite(o):
    checks = [
        ("params", lambda: short_pins.test_short_params_are_minimal(o)),
        ("index_sets_11", lambda: short_pins.test_short_index_sets_match_paper(o)),
        ("brute_11", lambda: short_pins.test_short_bruteforce(o, 11)),
        ("padded_100", lambda: short_pins.test_short_equals_zero_padded_full_length(o, 100)),
        ("matrix_545", lambda: short_pins.test_short_matrix_form_long(o, 545)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except Exception:
            failed.append(name)
    return failed


def test_unmutated_copy_passes(tmp_path):
    src = tmp_path / "hd_oracle.c"
    shutil.copy(SRC, src)
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "lib.so"))
    assert _pin_suite(oracle.Oracle(lib)) == []
    assert _short_pin_suite(oracle.Oracle(lib)) == []
    assert _secded_pin_suite(oracle.Oracle(lib)) == []


@pytest.mark.parametrize("name", sorted(SHORT_MUTANTS))
def test_short_mutant_is_caught(tmp_path, name):
    old, new = SHORT_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique: {old}"
    src = tmp_path / "hd_oracle.c"
    src.write_text(text.replace(old, new, 1))
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "lib.so"))
    assert _short_pin_suite(oracle.Oracle(lib)), f"mutant {name} passed every pin"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, f"mutation anchor missing: {old}"
    src = tmp_path / "hd_oracle.c"
    src.write_text(text.replace(old, new, 1))
    lib = oracle.build(force=True, src=str(src), out=str(tmp_path / "lib.so"))
    assert _pin_suite(oracle.Oracle(lib)), f"mutant {name} passed every pin"
