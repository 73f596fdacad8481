"""Planted mistakes in the oracle must be caught by its pins.

Each case edits one plausible slip into a copy of the oracle's C source (a
dropped error term, a wrong sign, a transposed or wrong index, an off-by-one,
a wrong rounding rule), builds it on the CPU, swaps it in for the real oracle
and runs every pin: at least one must fail.  Mistakes are planted only in the
oracle, never in the CUDA path, and every mutant stays in bounds.
"""
import os
import subprocess

import pytest

import oracle
from oracle_pins import PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "lak_oracle.c")

MUTANTS = [
    ("two_sum_no_remainder", "*e = (a - av) + (b - bv);", "*e = 0.0;"),
    ("two_prod_no_remainder", "*e = fma(a, b, -prod);", "*e = 0.0;"),
    ("axpy_sign", "x[i] = y[i] + az;", "x[i] = y[i] - az;"),
    ("axpy_wrong_operand", "double az = alpha * z[i];\n        x[i] = y[i] + az;",
     "double az = alpha * y[i];\n        x[i] = y[i] + az;"),
    ("axpby_drop_scale", "double ay = alpha_y * y[i];", "double ay = y[i];"),
    ("dot_drop_first_term", "for (int64_t i = 0; i < n; ++i) acc_add_prod(&acc, x[i], y[i]);",
     "for (int64_t i = 1; i < n; ++i) acc_add_prod(&acc, x[i], y[i]);"),
    ("sparse_dot_gather_by_position", "acc_add_prod(&acc, v[k], y[c[k]]);",
     "acc_add_prod(&acc, v[k], y[k < nnz ? c[0] : 0]);"),
    ("sparse_dot_drop_last", "for (int64_t k = 0; k < nnz; ++k) acc_add_prod(&acc, v[k], y[c[k]]);",
     "for (int64_t k = 0; k + 1 < nnz; ++k) acc_add_prod(&acc, v[k], y[c[k]]);"),
    ("row_bins_edge_inclusive", "while (b < nbins - 1 && len > (per_lane << b)) ++b;",
     "while (b < nbins - 1 && len >= (per_lane << b)) ++b;"),
    ("row_bins_unstable", "perm[next[b]++] = (int32_t)i;", "perm[bin_ptr[b + 1] - 1 - (next[b]++ - bin_ptr[b])] = (int32_t)i;"),
    ("gemv_row_transposed",
     "double a = (layout == 0) ? A[i * lda + j] : A[i + j * lda];\n            acc_add_prod(&acc, a, x[j]);\n        }\n        y[i]",
     "double a = (layout == 0) ? A[j * lda + i] : A[i + j * lda];\n            acc_add_prod(&acc, a, x[j]);\n        }\n        y[i]"),
    ("gemv_col_transposed",
     "double a = (layout == 0) ? A[i * lda + j] : A[i + j * lda];\n            acc_add_prod(&acc, a, x[j]);\n        }\n        y[i]",
     "double a = (layout == 0) ? A[i * lda + j] : A[j + i * lda];\n            acc_add_prod(&acc, a, x[j]);\n        }\n        y[i]"),
    ("spmv_gather_by_position",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)\n            acc_add_prod(&acc, vals[k], x[col_idx[k]]);\n        y[i]",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)\n            acc_add_prod(&acc, vals[k], x[col_idx[row_ptr[i]]]);\n        y[i]"),
    ("spmv_skip_first_entry",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)\n            acc_add_prod(&acc, vals[k], x[col_idx[k]]);\n        y[i]",
     "for (int64_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k)\n            acc_add_prod(&acc, vals[k], x[col_idx[k]]);\n        y[i]"),
    ("csc_no_cursor_advance", "int64_t q = cursor[col_idx[k]]++;", "int64_t q = cursor[col_idx[k]];"),
    ("dense_outer_operator", "dA[i * ldd + j] = dy[i] * x[j];", "dA[i * ldd + j] = dy[i] + x[j];"),
    ("sampled_outer_row_first_col", "dvals[k] = dy[i] * x[col_idx[k]];",
     "dvals[k] = dy[i] * x[col_idx[row_ptr[i]]];"),
    ("scale_operator", "out[i] = s * v[i];", "out[i] = s + v[i];"),
    ("bf16_round_half_up", "if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;",
     "if (rest >= 0x8000u) keep += 1u;"),
    ("bf16_f64_through_f32", "double r = nearbyint(a / quantum);   /* exact scaling; nearest-even */",
     "double r = nearbyint((double)(float)a / quantum);"),
    ("bf16_f64_fraction_bits", "double quantum = (exp_unb < -126) ? ldexp(1.0, -133) : ldexp(1.0, exp_unb - 7);",
     "double quantum = (exp_unb < -126) ? ldexp(1.0, -133) : ldexp(1.0, exp_unb - 8);"),
    ("f16_subnormal_quantum", "double quantum = (exp_unb < -14) ? ldexp(1.0, -24)",
     "double quantum = (exp_unb < -14) ? ldexp(1.0, -23)"),
    ("f16_widen_bias", "else v = ldexp((double)(1024 + f), e - 25);",
     "else v = ldexp((double)(1024 + f), e - 24);"),
    ("sell_tie_order", "if (lo > lr || (lo == lr && (o >= 0 ? o : m + q) < (r >= 0 ? r : m + p))) break;",
     "if (lo > lr || (lo == lr && (o >= 0 ? o : m + q) > (r >= 0 ? r : m + p))) break;"),
    ("sell_row_major_slot", "int64_t slot = slice_ptr[s] + j * C + r;\n                if (j < l) {",
     "int64_t slot = slice_ptr[s] + r * slice_len[s] + j;\n                if (j < l) {"),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, source, tmp_path, monkeypatch):
    assert source.count(old) >= 1, f"mutation site for {name} not found in the oracle"
    mutated = source.replace(old, new, 1)
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(so), str(csrc), "-lm"], check=True, capture_output=True)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(str(so)))
    failed = []
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake {name}"
