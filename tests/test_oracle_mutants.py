"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/ca_oracle.c`` (a dropped
term, a flipped sign, a wrong index, a transposed operand, a wrong tie rule
or tree grouping), builds it on the CPU, and runs the pin suite
``tests/test_oracle.py`` against it; the suite must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ca_oracle.c")

MUTANTS = {
    "argmax_last_max": ("if (a > amax) {", "if (a >= amax) {"),
    "perm_not_swapped": ("perm[j] = perm[p];\n        perm[p] = ti;", "(void)ti;"),
    "update_sign": ("AT(W, ldw, i, q) - AT(W, ldw, i, j) * u;", "AT(W, ldw, i, q) + AT(W, ldw, i, j) * u;"),
    "no_scale_by_pivot": ("AT(W, ldw, i, j) = AT(W, ldw, i, j) / piv;", "AT(W, ldw, i, j) = AT(W, ldw, i, j);"),
    "binary_pairs_skip": ("start[nout] = off + 2 * o;", "start[nout] = off + o;"),
    "flat_as_one_group": ("int f = (l == t->nlevels - 1) ? cur : t->fan_in[l];", "int f = cur;"),
    "calu_trsm_dropped_term": ("for (int l = 0; l < j; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, kb + j);",
                               "for (int l = 0; l + 1 < j; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, kb + j);"),
    "calu_u12_transposed": ("s = s - AT(A, lda, kb + i, kb + l) * AT(A, lda, kb + l, q);",
                            "s = s - AT(A, lda, kb + l, kb + i) * AT(A, lda, kb + l, q);"),
    "schur_wrong_index": ("for (int l = 0; l < bk; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, q);",
                          "for (int l = 1; l < bk; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, q);"),
    "householder_beta_sign": ("real beta = (alpha >= 0.0) ? -nrm : nrm;", "real beta = (alpha >= 0.0) ? nrm : -nrm;"),
    "larft_missing_tau": ("AT(T, ldt, i, j) = -tau[j] * s;", "AT(T, ldt, i, j) = -s;"),
    "apply_t_not_transposed": ("for (int l = 0; l <= j; ++l) s = s + AT(T, ldt, l, j) * AT(Wk, k, l, q);",
                               "for (int l = 0; l <= j; ++l) s = s + AT(T, ldt, j, l) * AT(Wk, k, l, q);"),
    "merge_r_lower_kept": ("AT(S, rows, at + i, q) = (q >= i) ? AT(P, ldp, top[ch] + i, q) : 0.0;",
                           "AT(S, rows, at + i, q) = AT(P, ldp, top[ch] + i, q);"),
    "getrs_no_swap": ("int p = ipiv[i] - 1;", "int p = i;"),
    "getrs_forward_reads_own_row": ("for (int l = 0; l < i; ++l) s = s - AT(LU, lda, i, l) * x[l];",
                                    "for (int l = 0; l <= i; ++l) s = s - AT(LU, lda, i, l) * x[l];"),
    "geqrs_r_transposed": ("for (int l = i + 1; l < n; ++l) s = s - AT(QR, lda, i, l) * AT(B, ldb, l, c);",
                           "for (int l = i + 1; l < n; ++l) s = s - AT(QR, lda, l, i) * AT(B, ldb, l, c);"),
    "op_inner_tree_flat": ("in.style[0] = ORA_BINARY;", "in.style[0] = ORA_FLAT;"),
    "op_inner_width_wrong_level": ("in.op_b[0] = t->op_b[1];", "in.op_b[0] = t->op_b[0];"),
    "op_pivots_not_applied": ("perm[i] = perm[sw];\n    perm[sw] = ti;", "(void)ti;\n    (void)sw;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC", "-o", str(so),
                    str(mut), "-lm"], check=True)
    env = dict(os.environ, CA_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught by the pins"
