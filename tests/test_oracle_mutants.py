"""The oracle's pins catch plausible mistakes (mutation tests, CPU only).

Each case below plants one mistake in a copy of the oracle's C sources -- a
wrong rounding rule, a dropped sticky bit, a wrong sign, index or operand
order in the printed Strassen / Winograd formulas (Sec. 2), a missing odd-size
fix-up, a reordered sum, a pivot or elimination step of Sec. 4 done another
way, a dropped term of the exact dot product -- builds that copy, and runs the
pin tests against it (ORACLE_LIB points the oracle at the copy).  At least one
pin must fail.  A control run of the same pins against an unmodified copy,
built the same way, must pass.  The Python part (the Section 4 benchmark's
exact product and error routine) gets the same treatment in a swapped-in
copy of one function.  The mistakes live only in the temporary copies; the
oracle's sources are never changed.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORC = os.path.join(ROOT, "oracle")
SOURCES = ["orc_num.c", "orc_mat.c", "orc_gemm.c", "orc_sampled.c", "orc_lu.c", "orc_api.c"]

SCALAR = ["tests/test_oracle_scalar.py"]
GEMM = ["tests/test_oracle_gemm.py"]
LU = ["tests/test_oracle_lu.py", "-k", "not 8650"]          # the 8650-bit factorisations add time, not reach
DOT = ["tests/test_oracle_lu.py", "-k", "exact_dot"]

# (name, file, text in the oracle, planted replacement, pin files)
MUTANTS = [
    # scalar arithmetic (Sec. 1, Sec. 3: every operation rounded to nearest, ties to even)
    ("ties_away_from_zero", "orc_num.c", "if (rb && (st || (q[0] & 1u))) {", "if (rb) {", SCALAR),
    ("sticky_below_round_bit_dropped", "orc_num.c", "int st = sticky || big_any_below(N, n, s - 1);",
     "int st = sticky;", SCALAR),
    ("add_far_operand_cut_too_early", "orc_num.c", "if (d >= p + 2) { orc_copy(r, x); return; }",
     "if (d >= p) { orc_copy(r, x); return; }", SCALAR),
    ("exact_zero_sum_keeps_sign", "orc_num.c", "if (big_is_zero(S, n)) { orc_set_zero(r, 0); return; }",
     "if (big_is_zero(S, n)) { orc_set_zero(r, x->sign); return; }", SCALAR),
    ("product_exponent_off_by_one", "orc_num.c", "a->exp + b->exp - 64 * (int64_t)nw, 0, sign);",
     "a->exp + b->exp - 64 * (int64_t)nw + 1, 0, sign);", SCALAR),
    ("product_row_carry_dropped", "orc_num.c", "r[i + bn] = (uint32_t)c;", "r[i + bn] = 0u;", SCALAR),
    ("quotient_remainder_ignored", "orc_num.c", "!big_is_zero(rem, nw), sign);", "0, sign);", SCALAR),
    # Strassen (Sec. 2, P1..P7 and the C blocks)
    ("strassen_c11_sign", "orc_gemm.c", "mat_addsub(&X, &T, &P[4], -1);", "mat_addsub(&X, &T, &P[4], +1);", GEMM),
    ("strassen_p6_operands_swapped", "orc_gemm.c", "mat_addsub(&X, A21, A11, -1);",
     "mat_addsub(&X, A11, A21, -1);", GEMM),
    ("strassen_c22_last_term_subtracted", "orc_gemm.c", "mat_addsub(&Cq[3], &X, &P[5], +1);",
     "mat_addsub(&Cq[3], &X, &P[5], 0);", GEMM),
    # Winograd's variant (Sec. 2, S1..S8, M1..M7, T1, T2)
    ("winograd_s4_wrong_index", "orc_gemm.c", "mat_addsub(&S[4], A12, &S[2], -1);",
     "mat_addsub(&S[4], A12, &S[1], -1);", GEMM),
    ("winograd_m3_transposed_operands", "orc_gemm.c", "rc |= mul(ctx, A12, B21, &M[3]);",
     "rc |= mul(ctx, A21, B12, &M[3]);", GEMM),
    ("winograd_c12_summed_right_to_left", "orc_gemm.c",
     "mat_addsub(&U, &T1, &M[5], +1);       /* C12 = T1 + M5 + M6 */\n    mat_addsub(&Cq[1], &U, &M[6], +1);",
     "mat_addsub(&U, &M[5], &M[6], +1);\n    mat_addsub(&Cq[1], &T1, &U, +1);", GEMM),
    ("winograd_t2_from_m3", "orc_gemm.c", "mat_addsub(&T2, &T1, &M[4], +1);",
     "mat_addsub(&T2, &T1, &M[3], +1);", GEMM),
    # recursion control and odd sizes
    ("odd_l_rank1_fixup_missing", "orc_gemm.c",
     "if (Lr < l) {                                  /* l peeled: rank-1 fix-up */", "if (0) {", GEMM),
    ("mixed_policy_pads_the_wrong_class", "orc_gemm.c",
     "if (policy == ORC_MIXED && x % 4 == 3) return x + 1;   /* pad */",
     "if (policy == ORC_MIXED && x % 4 == 1) return x + 1;   /* pad */", GEMM),
    ("recursion_stops_one_size_late", "orc_gemm.c",
     "if (!(m > cfg->cutoff && l > cfg->cutoff && n > cfg->cutoff)) {",
     "if (!(m >= cfg->cutoff && l >= cfg->cutoff && n >= cfg->cutoff)) {", GEMM),
    # Simple (Eq. 1): the sum runs k = 1..l in order
    ("simple_sum_descending", "orc_gemm.c", "for (int64_t k = 0; k < A->cols; ++k) {",
     "for (int64_t k = A->cols - 1; k >= 0; --k) {", GEMM),
    # sampled recursion: the closure must hold both halves' partner rows
    ("sampled_closure_partner_missing", "orc_sampled.c",
     "if (!rc && C.v[i] + half < x && iset_add(S, C.v[i] + half)) rc = -1;", "(void)half;", GEMM),
    ("sampled_rank1_fixup_missing", "orc_sampled.c",
     "if (Lr < l) {                                   /* peeled l: rank-1 */", "if (0) {", GEMM),
    ("sampled_b_quadrant_rows_from_the_column_half", "orc_sampled.c", "int64_t rr = r + (q / 2) * k;",
     "int64_t rr = r + (q % 2) * k;", GEMM),
    # LU (Sec. 4) with partial pivoting
    ("pivot_last_of_equal_magnitudes", "orc_lu.c", "if (orc_cmpabs(&x, &best, p) > 0) {",
     "if (orc_cmpabs(&x, &best, p) >= 0) {", LU),
    ("multiplier_by_reciprocal", "orc_lu.c", "orc_div(&l, &x, &d, p);",
     "{ orc_num one, rcp; orc_from_rational(&one, 1, 1, p); orc_div(&rcp, &one, &d, p); "
     "orc_mul(&l, &x, &rcp, p); }", LU),
    ("u12_terms_descending", "orc_lu.c", "for (int64_t s = j0; s < r; ++s) {",
     "for (int64_t s = r - 1; s >= j0; --s) {", LU),
    ("trailing_update_adds", "orc_lu.c", "orc_get(&T, i, c, &t);\n                orc_sub(&y, &y, &t, p);",
     "orc_get(&T, i, c, &t);\n                orc_add(&y, &y, &t, p);", LU),
    ("solve_skips_row_exchanges", "orc_lu.c",
     "if (piv[k] != k) { orc_num s = v[k]; v[k] = v[piv[k]]; v[piv[k]] = s; }", "(void)piv;", LU),
    # interchange format, conversion, Block, operation counts, the unpivoted
    # LU and the forward substitution
    ("limb_halves_swapped_on_import", "orc_mat.c",
     "x.m[2 * (L - 1 - k)] = (uint32_t)v;\n                x.m[2 * (L - 1 - k) + 1] = (uint32_t)(v >> 32);",
     "x.m[2 * (L - 1 - k) + 1] = (uint32_t)v;\n                x.m[2 * (L - 1 - k)] = (uint32_t)(v >> 32);",
     SCALAR),
    ("conversion_drops_sign", "orc_num.c",
     "orc_round_int(r, p_to, x->m, nwf, x->exp - 32 * (int64_t)nwf, 0, x->sign);",
     "orc_round_int(r, p_to, x->m, nwf, x->exp - 32 * (int64_t)nwf, 0, 0);", SCALAR),
    ("block_k_blocks_descending", "orc_gemm.c", "for (int64_t K = 0; K < l; K += nb) {",
     "for (int64_t K = ((l - 1) / nb) * nb; K >= 0; K -= nb) {", GEMM),
    ("winograd_count_eight_combination_sums", "orc_gemm.c", "cc_ = algo == ORC_STRASSEN ? 8 : 7;",
     "cc_ = algo == ORC_STRASSEN ? 8 : 8;", GEMM),
    ("pivoting_flag_ignored", "orc_lu.c", "for (int64_t i = k + 1; pivoting && i < n; ++i) {",
     "for (int64_t i = k + 1; i < n; ++i) {", LU),
    ("forward_substitution_adds", "orc_lu.c",
     "orc_sub(&v[i], &v[i], &t, p);\n        }\n    for (int64_t j = n - 1; j >= 0; --j) {",
     "orc_add(&v[i], &v[i], &t, p);\n        }\n    for (int64_t j = n - 1; j >= 0; --j) {", LU),
    # correctly rounded exact dot product
    ("exact_dot_sign_of_a_only", "orc_num.c", "big_add_at((a[k].sign ^ b[k].sign) ? neg : pos",
     "big_add_at(a[k].sign ? neg : pos", DOT),
    ("exact_dot_alignment_off_by_one", "orc_num.c", "int64_t sh = E - Emin;", "int64_t sh = E - Emin + 1;",
     DOT),
]


_CFLAGS = ["gcc", "-O1", "-std=c11", "-fPIC", "-fopenmp", "-w"]


@pytest.fixture(scope="module")
def base_objects(tmp_path_factory):
    """The unmodified sources compiled once; a mutant recompiles one file."""
    d = str(tmp_path_factory.mktemp("oracle_base"))
    for f in SOURCES + ["orc.h"]:
        shutil.copy(os.path.join(ORC, f), os.path.join(d, f))
    for f in SOURCES:
        subprocess.check_call(_CFLAGS + ["-c", os.path.join(d, f), "-o", os.path.join(d, f[:-2] + ".o")])
    return d


def _build(base, dest, name=None, old=None, new=None):
    """Link a copy of the oracle with one source file carrying a planted
    replacement (none for the control copy)."""
    os.makedirs(dest, exist_ok=True)
    objs = [os.path.join(base, f[:-2] + ".o") for f in SOURCES]
    if name is not None:
        src = os.path.join(dest, name)
        shutil.copy(os.path.join(base, "orc.h"), os.path.join(dest, "orc.h"))
        text = open(os.path.join(base, name)).read()
        assert text.count(old) == 1, "the planted text must occur once: %r" % old
        open(src, "w").write(text.replace(old, new))
        obj = os.path.join(dest, name[:-2] + ".o")
        subprocess.check_call(_CFLAGS + ["-c", src, "-o", obj])
        objs[SOURCES.index(name)] = obj
    lib = os.path.join(dest, "liboracle.so")
    subprocess.check_call(["gcc", "-shared", "-fopenmp", "-o", lib] + objs)
    return lib


def _run_pins(lib, pins, stop_first=True):
    env = dict(os.environ, ORACLE_LIB=lib, OMP_NUM_THREADS="4")
    cmd = [sys.executable, "-m", "pytest", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
    if stop_first:
        cmd.append("-x")
    r = subprocess.run(cmd + pins, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


def test_control_copy_passes_the_pins(tmp_path, base_objects):
    lib = _build(base_objects, str(tmp_path / "control"))
    rc, out = _run_pins(lib, SCALAR + GEMM + ["tests/test_oracle_lu.py"], stop_first=True)
    assert rc == 0, out


@pytest.mark.parametrize("name,file,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, base_objects, name, file, old, new, pins):
    lib = _build(base_objects, str(tmp_path / name), file, old, new)
    rc, out = _run_pins(lib, pins)
    # 1: a pin failed; a negative code: the broken copy crashed a pin run
    assert rc == 1 or rc < 0, "mutant %s survived the pins (pytest exit %d):\n%s" % (name, rc, out)


# The Section 4 benchmark part of the oracle is Python: its mistakes are
# planted in a copy of one function, swapped in for the duration of the test.
def _pins_sqrt():
    from tests import test_oracle_sqrt as ts
    return [lambda: ts.test_product_S_closed_form(5, 7, 6), lambda: ts.test_product_S_closed_form(30, 65, 1024),
            lambda: ts.test_product_rows_rounded_once(128), lambda: ts.test_product_rows_rounded_once(512),
            ts.test_rel_errors_pinned]


PY_MUTANTS = [
    ("S_sum_stops_one_term_early", "sqrt_product_S", "for k in range(1, l + 1)", "for k in range(1, l)"),
    ("S_second_factor_off_by_one", "sqrt_product_S", "* (n - k + 1)", "* (n - k)"),
    ("sqrt15_truncated", "_rn_sqrt15", "keep += 1", "keep += 0"),
    ("sqrt15_exponent_off_by_one", "_rn_sqrt15", "return (1 if S < 0 else 0, keep, s - d)",
     "return (1 if S < 0 else 0, keep, s - d + 1)"),
    ("rel_error_absolute", "sqrt_rel_errors", "/ ((float(x) + r15) * r15)", "/ (float(x) + r15)"),
    ("rel_error_wrong_sign_branch", "sqrt_rel_errors", "out[i, j] = 1.0 + float(-x) / r15",
     "out[i, j] = float(-x) / r15"),
]


@pytest.mark.parametrize("name,func,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_mistake_in_python_part_is_caught(monkeypatch, name, func, old, new):
    import inspect
    import textwrap

    from oracle import oracle as orc

    fn = getattr(orc, func)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, "the planted text must occur once: %r" % old
    ns = dict(fn.__globals__)
    exec(compile(src.replace(old, new), "<planted %s>" % name, "exec"), ns)
    monkeypatch.setattr(orc, func, ns[func])
    caught = 0
    for pin in _pins_sqrt():
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, "mutant %s survived the pins" % name


def test_python_pins_pass_unmutated():
    for pin in _pins_sqrt():
        pin()
