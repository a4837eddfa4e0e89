"""Planted mistakes in the oracle must fail at least one pin.

Each mutant is the oracle source with one plausible slip (a transposed
operand, a wrong sign, a dropped term or factor, a wrong index, a wrong
rounding rule), compiled on the CPU into a temporary directory.  The pins
in ``oracle_pins`` are run against it and at least one must fail; the
committed oracle itself is never modified.
"""
import os
import subprocess
import sys

import pytest

from oracle.build import SRC, build_variant

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs every pin against one mutant build in a child process: a mutant that
# reads out of bounds may crash, which also counts as caught.
_RUNNER = """
import sys
sys.path.insert(0, %r)
import oracle
from tests import oracle_pins
orc = oracle.load_variant(sys.argv[1])
failed = []
for check in oracle_pins.ALL_CHECKS:
    try:
        check(orc)
    except Exception:
        failed.append(check.__name__)
print("FAILED:" + ",".join(failed))
"""

MUTANTS = {
    "transposed_operand": ("return trans ? (double)X[c * ld + r] : (double)X[r * ld + c];",
                           "return trans ? (double)X[r * ld + c] : (double)X[c * ld + r];"),
    "beta_sign": ("c += beta * c0;", "c -= beta * c0;"),
    "alpha_dropped": ("double c = alpha * acc[j];", "double c = acc[j];"),
    "last_k_dropped": ("for (int64_t k = 0; k < K; ++k) {\n                    double a = op_at",
                       "for (int64_t k = 0; k < K - 1; ++k) {\n                    double a = op_at"),
    "no_accumulate": ("acc[j] += a * b;", "acc[j] = a * b;"),
    "ties_away": ("if (dropped > 0x8000u || (dropped == 0x8000u && (upper & 1u)))",
                  "if (dropped >= 0x8000u)"),
    "truncating_split": ("if (dropped > 0x8000u || (dropped == 0x8000u && (upper & 1u)))",
                         "if (0)"),
    "lo_sign": ("l = oracle_bf16_rne((float)((double)x[t] - hv));",
                "l = oracle_bf16_rne((float)((double)x[t] + hv));"),
    "denominator_beta_dropped": ("d += fabs(beta) * fabs(c0);", "d += 0.0 * fabs(c0);"),
    "denominator_signed": ("mag[j] += fabs(a) * fabs(b);", "mag[j] += a * b;"),
    "term_index": ("if (terms & 2) s += ah * bl[k * N + j];", "if (terms & 2) s += al * bl[k * N + j];"),
    "rows_ignored": ("int64_t i = rows ? rows[r] : r;\n            for (int64_t j = 0; j < N; ++j) {\n                acc[j] = 0.0;\n                mag[j] = 0.0;",
                     "int64_t i = r;\n            for (int64_t j = 0; j < N; ++j) {\n                acc[j] = 0.0;\n                mag[j] = 0.0;"),
    "beta_read_when_zero": ("if (beta != 0.0) {\n                    double c0", "if (1) {\n                    double c0"),
    # SYR2K (Section 5.1)
    "syr2k_second_product_dropped": ("acc += aip * bjp + bip * ajp;", "acc += aip * bjp;"),
    "syr2k_wrong_operand": ("acc += aip * bjp + bip * ajp;", "acc += aip * bjp + aip * ajp;"),
    "syr2k_diagonal_excluded": ("int inside = uplo == 0 ? (j <= i) : (j >= i);",
                                "int inside = uplo == 0 ? (j < i) : (j >= i);"),
    "syr2k_triangle_swapped": ("int inside = uplo == 0 ? (j <= i) : (j >= i);",
                               "int inside = uplo == 0 ? (j >= i) : (j <= i);"),
    "syr2k_outside_scaled": ("C64[r * N + j] = C0 ? (double)C0[i * ldc0 + j] : 0.0;",
                             "C64[r * N + j] = C0 ? beta * (double)C0[i * ldc0 + j] : 0.0;"),
    "syr2k_split_roles": ("split_product((float)bip, (float)ajp, terms);",
                          "split_product((float)ajp, (float)bip, terms);"),
    "syr2k_denominator_signed": ("mag += fabs(aip) * fabs(bjp) + fabs(bip) * fabs(ajp);",
                                 "mag += aip * bjp + bip * ajp;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %s" % name
    path = build_variant(src.replace(old, new, 1), os.path.join(str(tmp_path), "mut_%s.so" % name))
    res = subprocess.run([sys.executable, "-c", _RUNNER % ROOT, path],
                         capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        return  # the mutant crashed on a pin input: caught
    line = [l for l in res.stdout.splitlines() if l.startswith("FAILED:")][-1]
    assert line != "FAILED:", "mutant %s passed every pin" % name


# Planted mistakes in the error measure (Python, so they are applied to a
# copy of the function's source rather than to gemm_ref.c).
ERROR_MUTANTS = {
    "returns_zero": ("    if num == 0.0:\n        return 0.0", "    if True:\n        return 0.0"),
    "mean_for_max": ("num = float(np.max(np.abs(C - C64)))", "num = float(np.mean(np.abs(C - C64)))"),
    "elementwise_ratio": ("num = float(np.max(np.abs(C - C64))) if C.size else 0.0\n    den = float(np.max(D))",
                          "num = float(np.max(np.abs(C - C64) / np.where(D > 0, D, 1.0))) if C.size else 0.0\n    den = 1.0 or float(np.max(D))"),
    "denominator_dropped": ("    return num / den", "    return num"),
    "denominator_ignores_d": ("den = float(np.max(D))", "den = float(np.max(np.abs(C64)))"),
    "signed_difference": ("num = float(np.max(np.abs(C - C64)))", "num = float(np.max(C - C64))"),
    "nan_ignored": ("num = float(np.max(np.abs(C - C64)))", "num = float(np.nanmax(np.abs(C - C64)))"),
    "difference_in_f32": ("C = np.asarray(C, dtype=np.float64)",
                          "C = np.asarray(C, dtype=np.float32); C64 = np.asarray(C64, dtype=np.float32)"),
    "mean_denominator": ("den = float(np.max(D))", "den = float(np.mean(D))"),
}


@pytest.mark.parametrize("name", sorted(ERROR_MUTANTS))
def test_error_measure_mutant_is_caught(name):
    import inspect
    import types

    import numpy as np

    import oracle
    from tests import oracle_pins

    old, new = ERROR_MUTANTS[name]
    src = inspect.getsource(oracle.normwise_error)
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    orc = types.SimpleNamespace(**{n: getattr(oracle, n) for n in dir(oracle) if not n.startswith("__")})
    orc.normwise_error = ns["normwise_error"]
    failed = []
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(orc)
        except Exception:
            failed.append(check.__name__)
    assert failed, "error-measure mutant %s passed every pin" % name
