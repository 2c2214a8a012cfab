"""Planted mistakes in the oracle, each of which a pin must catch (no GPU).

Each mutant is a copy of one oracle source with one plausible slip in it: a
dropped term or factor, a wrong sign or index, an off-by-one, truncation
replaced by rounding, the wrong tie rule. The copy is built (C) or executed
(Python) apart from the real oracle, which is never modified, and the pins of
test_oracle_pins.py, test_oracle_config.py and test_oracle_forms.py run
against it. At least one of them must fail, or the pins would not have told
that oracle from the right one.
"""
import os
import types

import pytest

import oracle
from oracle import forms
from tests import test_oracle_config as cfg_pins
from tests import test_oracle_forms as form_pins
from tests import test_oracle_pins as pins

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, original text, planted text[, count]); the original occurs in the
# source, and its first occurrence is the one changed (every occurrence when
# count is 0).
C_MUTANTS = [
    ("shift one too large", "*s = beta - e;", "*s = beta - e + 1;"),
    ("shift one too small", "*s = beta - e;", "*s = beta - e - 1;"),
    ("round instead of truncate", "double v = trunc(ldexp(x, s));", "double v = nearbyint(ldexp(x, s));"),
    ("floor instead of truncate", "double v = trunc(ldexp(x, s));", "double v = floor(ldexp(x, s));"),
    ("tie of an even modulus kept positive", "if (r >= (m + 1) / 2) r -= m;", "if (r > m / 2) r -= m;"),
    ("last term of the residue GEMM dropped",
     "for (int64_t h = 0; h < K; ++h) acc += (int64_t)u[h] * (int64_t)v[h];",
     "for (int64_t h = 0; h + 1 < K; ++h) acc += (int64_t)u[h] * (int64_t)v[h];"),
    ("planes of the wrong modulus",
     "const int16_t* u = U + ((int64_t)k * M + i) * K;",
     "const int16_t* u = U + ((int64_t)((k + 1) % Q) * M + i) * K;"),
    ("W mod m left negative", "W[((int64_t)k * M + i) * N + j] = (int32_t)r;",
     "W[((int64_t)k * M + i) * N + j] = (int32_t)(acc % mod[k]);"),
    ("Garner difference with the wrong sign", "int64_t d = ((int64_t)w[k] - acc) % mk;",
     "int64_t d = (acc - (int64_t)w[k]) % mk;"),
    ("CRT result not centred", "if (u256_cmp(&twoX, &P) >= 0) {", "if (0) {"),
    ("ties rounded away from zero", "if (half && (sticky || (q & 1))) q += 1;", "if (half) q += 1;"),
    ("sticky bit ignored", "if (half && (sticky || (q & 1))) q += 1;", "if (half && (q & 1)) q += 1;"),
    ("no gradual underflow", "int64_t lsb = (E >= -1022) ? E - 52 : -1074;", "int64_t lsb = E - 52;"),
    ("unscale with the column shift's sign flipped",
     "C[i * ldc + j] = round_scaled(&mag, neg, -((int64_t)s[i] + t[j]));",
     "C[i * ldc + j] = round_scaled(&mag, neg, -((int64_t)s[i] - t[j]));"),
    ("zero vector shifted by beta", "if (mx == 0.0) { *s = 0; return 0; }", "if (mx == 0.0) { *s = beta; return 0; }"),
    ("non-finite entries not refused", "if (!isfinite(", "if (0 && !isfinite(", 0),
]

PY_MUTANTS = [
    ("beta_max without the factor 2", "while 2 * K * (2**(b + 1) - 1) ** 2 < P:",
     "while K * (2**(b + 1) - 1) ** 2 < P:"),
    ("kappa_rec without the factor 2", "k_rec = (P - 1) // (2 * B * B)", "k_rec = (P - 1) // (B * B)"),
    ("radius rounded up", "return m // 2", "return (m + 1) // 2"),
    ("kappa_acc with the modulus for the radius", "k_acc = lam // (r * r)", "k_acc = lam // (2 * r * r)"),
    ("coprimality not checked", "                if nm & mask:\n                    continue\n", ""),
    ("least_q window without the factor 2", "need = K * 2**107", "need = K * 2**106"),
    ("counting bound without the factor 2", "n = 2 * K * B * B + 1", "n = K * B * B + 1"),
]

FORMS_MUTANTS = [
    ("subnormals one binade too small", "v = Fraction(mt, 2**mb) * Fraction(2) ** (1 - bias)",
     "v = Fraction(mt, 2**mb) * Fraction(2) ** (-bias)"),
    ("NaN code of E4M3 counted as a value", "            if style == \"fn\" and e == 2**eb - 1 and mt == 2**mb - 1:\n"
     "                continue\n", ""),
    ("plane radius from Lambda / 2K", "return math.isqrt(lam // K)", "return math.isqrt(lam // (2 * K))"),
    ("Toom weight of the a0 b0 product with the wrong sign", "return [(0, 0, 1 - b), (1, 1, b), (2, 2, b * b - b)]",
     "return [(0, 0, b - 1), (1, 1, b), (2, 2, b * b - b)]"),
    ("three-GEMM schoolbook without the m | b^2 test", "if (b * b) % m == 0 and np.unique", "if np.unique"),
    ("encoding tie picks the larger plane value", "key = (size, abs(a1), a1, a0)", "key = (-size, abs(a1), a1, a0)"),
]

C_PINS = [
    (pins.test_oracle_equals_exact_definition, (0, 0.5, 53, pins.MODS16)),
    (pins.test_oracle_equals_exact_definition, (2, 1.0, 50, pins.MODS14)),
    (pins.test_planes_are_balanced_residues_of_truncation, ()),
    (pins.test_lossless_conversion_returns_fl_of_exact_product, ()),
    (pins.test_lossless_53bit_operands_exercise_rounding, ()),
    (pins.test_k1_is_the_plain_product, ()),
    (pins.test_invariants_scaling_sign_transpose, ()),
    (pins.test_crt_invariants_and_window, ()),
    (pins.test_x_is_bounded_and_exact, ()),
    (pins.test_rounding_against_exact_rationals, ()),
    (pins.test_subnormal_and_huge_operands_match_definition, ()),
    (pins.test_zero_rows_and_columns, ()),
    (pins.test_nonfinite_input_is_refused, ()),
    (pins.test_truncation_error_bound, (53,)),
]

CONFIG_PINS = [
    (cfg_pins.test_dp_matches_exhaustive_search, (4, 30)),
    (cfg_pins.test_int8_set_reproduces_printed_kmax, ()),
    (cfg_pins.test_kmax_is_largest_at_239_and_256_gives_ozii_int8, ()),
    (cfg_pins.test_rmax_and_counting_bound, ()),
    (cfg_pins.test_least_q_row_of_table, ()),
    (cfg_pins.test_kappa_rec_reproduces_the_least_q_row_of_table, ()),
    (cfg_pins.test_beta_max_definition, ()),
]

FORMS_PINS = [
    (form_pins.test_e2m1_alphabet_and_products, ()),
    (form_pins.test_plane_radius_under_fp32_accumulation, ()),
    (form_pins.test_fp8_values_and_codes_match_a_library_decoder, ("E4M3", "float8_e4m3fn")),
    (form_pins.test_fp8_values_and_codes_match_a_library_decoder, ("E5M2", "float8_e5m2")),
    (form_pins.test_fp8_fp6_alphabets_agree, ()),
    (form_pins.test_example_base13_limbs, ()),
    (form_pins.test_fig3_schoolbook_pool_and_its_optimum, ()),
    (form_pins.test_table_moduli_e2m1, (2**14, 59)),
    (form_pins.test_form_tables_decode_and_recombine, ("E2M1", 2**14, None)),
    (form_pins.test_form_tables_decode_and_recombine, ("E3M2", 2**13, 400)),
]


def _plant(src: str, old: str, new: str, count: int = 1) -> str:
    assert old in src, f"mutation site not found: {old!r}"
    return src.replace(old, new, count if count > 0 else -1)


def _caught(battery) -> str:
    """Name of the first pin that fails, or '' if every pin passes."""
    for fn, args in battery:
        try:
            fn(*args)
        except (Exception, pytest.fail.Exception):
            return fn.__name__
    return ""


def _python_mutant(path: str, name: str, old: str, new: str):
    src = _plant(open(path).read(), old, new)
    mod = types.ModuleType(name)
    mod.__file__ = path                    # the same directory, so the C library paths resolve
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


def test_every_mutation_site_exists_once_or_first():
    c_src = open(os.path.join(ORACLE_DIR, "oz_oracle.c")).read()
    py_src = open(os.path.join(ORACLE_DIR, "__init__.py")).read()
    f_src = open(os.path.join(ORACLE_DIR, "forms.py")).read()
    for src, muts in ((c_src, C_MUTANTS), (py_src, PY_MUTANTS), (f_src, FORMS_MUTANTS)):
        for name, old, new, *_ in muts:
            assert old in src and old != new, name


@pytest.mark.parametrize("mut", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_oracle_mutant_is_caught(mut, tmp_path, monkeypatch):
    name = mut[0]
    src = _plant(open(os.path.join(ORACLE_DIR, "oz_oracle.c")).read(), *mut[1:])
    path = tmp_path / "oz_oracle_mutant.c"
    path.write_text(src)
    monkeypatch.setattr(oracle, "_SRC", str(path))
    monkeypatch.setattr(oracle, "_LIB_PATH", str(tmp_path / "liboz_oracle_mutant.so"))
    monkeypatch.setattr(oracle, "_lib", None)
    oracle.build(force=True)
    assert _caught(C_PINS), f"no pin fails for the planted mistake: {name}"


@pytest.mark.parametrize("name,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_oracle_mutant_is_caught(name, old, new, monkeypatch):
    mutant = _python_mutant(os.path.join(ORACLE_DIR, "__init__.py"), "oracle_mutant", old, new)
    monkeypatch.setattr(cfg_pins, "oracle", mutant)
    assert _caught(CONFIG_PINS), f"no pin fails for the planted mistake: {name}"


@pytest.mark.parametrize("name,old,new", FORMS_MUTANTS, ids=[m[0] for m in FORMS_MUTANTS])
def test_forms_oracle_mutant_is_caught(name, old, new, monkeypatch):
    mutant = _python_mutant(os.path.join(ORACLE_DIR, "forms.py"), "forms_mutant", old, new)
    monkeypatch.setattr(form_pins, "forms", mutant)
    assert _caught(FORMS_PINS), f"no pin fails for the planted mistake: {name}"
