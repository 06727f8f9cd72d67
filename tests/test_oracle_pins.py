"""Pins for the oracle (CPU only): each test checks the oracle against something other
than itself -- exact rational brute force over a case-by-case statement of the
paper's table, an independent library (numpy/BLAS zgemm) on explicitly cast and
projected operands, the paper's 1m worked example, closed-form invariants, the scalar
rules, and error-free summation on an ill-conditioned sum.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import oracle_mxgemm, OracleError
from paper_1901_06015_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CPLX = synth.COMPLEX_DTS


# ---------------------------------------------------------------- exact brute force
def _rnd(x, prec):
    """Round a binary64 value to the precision with numpy's own cast (IEEE RN-even)."""
    return float(np.float32(x)) if prec == "s" else float(x)


def _fr_op(X, trans):
    """op(X) as a list of rows of (re, im) Fractions (independent of the oracle)."""
    X = np.asarray(X)
    rows = [[complex(v) for v in row] for row in X.tolist()]
    if trans in ("t", "h"):
        rows = [list(r) for r in zip(*rows)]
    out = []
    for r in rows:
        o = []
        for v in r:
            re, im = Fraction(v.real), Fraction(v.imag)
            if trans in ("c", "h"):
                im = -im
            o.append((re, im))
        out.append(o)
    return out


def frac_reference(combo, transa, transb, alpha, A, B, beta, C):
    """Case-by-case statement of Fig. 'mixeddom' + Secs. 5.1 and 7, in exact rationals."""
    dc, da, db, x = combo
    prec_c = "d" if dc in ("d", "z") else "s"
    comp = prec_c if x == "c" else x
    opA, opB = _fr_op(A, transa), _fr_op(B, transb)
    m, k = len(opA), len(opA[0]) if opA else 0
    n = len(opB[0]) if opB else 0
    cast = lambda z: (Fraction(_rnd(float(z[0]), comp)), Fraction(_rnd(float(z[1]), comp)))
    Ah = [[cast(v) for v in r] for r in opA]
    Bh = [[cast(v) for v in r] for r in opB]
    al = complex(alpha); be = complex(beta)
    ar, ai = Fraction(_rnd(al.real, comp)), Fraction(_rnd(al.imag, comp))
    br, bi = Fraction(_rnd(be.real, prec_c)), Fraction(_rnd(be.imag, prec_c))
    Cin = [[complex(v) for v in r] for r in np.asarray(C).tolist()]
    res = []
    for i in range(m):
        row = []
        for j in range(n):
            c_re, c_im = Fraction(Cin[i][j].real), Fraction(Cin[i][j].imag)
            if br == 0 and bi == 0:
                c_re = c_im = Fraction(0)
            # products term by term, per the case table
            s_rr = sum((Ah[i][p][0] * Bh[p][j][0] for p in range(k)), Fraction(0))
            s_ii = sum((Ah[i][p][1] * Bh[p][j][1] for p in range(k)), Fraction(0))
            s_ri = sum((Ah[i][p][0] * Bh[p][j][1] for p in range(k)), Fraction(0))
            s_ir = sum((Ah[i][p][1] * Bh[p][j][0] for p in range(k)), Fraction(0))
            if dc not in CPLX:
                if da not in CPLX and db not in CPLX:      # case 0: C := AB + C
                    P = s_rr
                elif da not in CPLX:                       # 1b: C := A Re(B) + C
                    P = s_rr
                elif db not in CPLX:                       # 1a: C := Re(A) B + C
                    P = s_rr
                else:                                      # 2ab: C := Re(AB) + C
                    P = s_rr - s_ii
                row.append((br * c_re + ar * P, Fraction(0)))
            else:
                bc_re = br * c_re - bi * c_im
                bc_im = br * c_im + bi * c_re
                if da not in CPLX and db not in CPLX:      # 1c: Re(C) += AB
                    row.append((bc_re + ar * s_rr, bc_im))
                    continue
                if da not in CPLX:                         # 2bc: A real, B complex
                    P_re, P_im = s_rr, s_ri
                elif db not in CPLX:                       # 2ac: A complex, B real
                    P_re, P_im = s_rr, s_ir
                else:                                      # 3: complex gemm
                    P_re, P_im = s_rr - s_ii, s_ri + s_ir
                row.append((bc_re + ar * P_re - ai * P_im, bc_im + ar * P_im + ai * P_re))
        res.append(row)
    return res


def _layout(rng, arr, kind):
    """Return arr stored column-major, row-major, or as a general-stride view."""
    if kind == "col":
        return np.asfortranarray(arr)
    if kind == "row":
        return np.ascontiguousarray(arr)
    big = np.zeros((arr.shape[0] * 2 + 1, arr.shape[1] * 3 + 2), dtype=arr.dtype)
    view = big[1::2, 2::3][: arr.shape[0], : arr.shape[1]]
    view[...] = arr
    return view


def _dyadic(rng, shape, dt):
    re = rng.integers(-8, 9, size=shape) / 4.0
    if dt in CPLX:
        im = rng.integers(-8, 9, size=shape) / 4.0
        return (re + 1j * im).astype(synth.NP_OF_DT[dt])
    return re.astype(synth.NP_OF_DT[dt])


@pytest.mark.parametrize("combo", synth.all_combos())
def test_bruteforce_exact_all_combos(combo):
    """Tiny dyadic inputs: every partial sum is exact in binary64, so the oracle must
    equal the exact rational result bit for bit, for every trans pair and layout."""
    rng = np.random.default_rng(abs(hash(combo)) % (2 ** 32))
    dc, da, db = combo[:3]
    case = oracle.oracle_case_of(dc, da, db)
    for ta, tb in itertools.product("ntch", repeat=2):
        m, n, k = (int(v) for v in rng.integers(1, 4, size=3))
        A = _dyadic(rng, (k, m) if ta in "th" else (m, k), da)
        B = _dyadic(rng, (n, k) if tb in "th" else (k, n), db)
        C0 = _dyadic(rng, (m, n), dc)
        alpha = (0.75 + 0.5j) if case in (0, 7) else -1.5
        beta = [0.0, -0.5, 1.0, 0.25 - 0.75j][int(rng.integers(0, 4))]
        lay = [("col", "row", "gen")[int(v)] for v in rng.integers(0, 3, size=3)]
        A_, B_, C_ = _layout(rng, A, lay[0]), _layout(rng, B, lay[1]), _layout(rng, C0, lay[2])
        Cw = C_.copy() if lay[2] != "gen" else C_
        out = oracle_mxgemm(ta, tb, alpha, A_, B_, beta, Cw, comp=combo[3])
        exp = frac_reference(combo, ta, tb, alpha, A, B, beta, C0)
        for i in range(m):
            for j in range(n):
                er, ei = exp[i][j]
                assert out[i, j].real == float(er) and out[i, j].imag == float(ei), \
                    (combo, ta, tb, i, j, out[i, j], er, ei)
                want = complex(float(er), float(ei))
                if dc not in CPLX:
                    want = want.real
                assert Cw[i, j] == synth.NP_OF_DT[dc](want)


@pytest.mark.parametrize("combo", ["sdds", "dsss", "zddd", "cdzs", "zzcs", "szzs", "cdds"])
def test_bruteforce_cast_to_comp_precision(combo):
    """Inputs that single precision cannot hold: the oracle must first round A, B and
    alpha to the computation precision (Sec. 5.1.2, Sec. 7.1) and beta to C's."""
    rng = np.random.default_rng(7)
    dc, da, db, x = combo
    m, n, k = 2, 3, 3
    def odd(shape, dt):
        v = 1.0 + rng.integers(1, 1000, size=shape) * 2.0 ** -40
        if dt in CPLX:
            v = v - 1j * (1.0 + rng.integers(1, 1000, size=shape) * 2.0 ** -38)
        return np.asfortranarray(v.astype(synth.NP_OF_DT[dt]))
    A, B, C0 = odd((m, k), da), odd((k, n), db), odd((m, n), dc)
    alpha, beta = 1.0 + 2.0 ** -35, -(1.0 + 2.0 ** -33)
    Cw = C0.copy(order="F")
    out = oracle_mxgemm("n", "n", alpha, A, B, beta, Cw, comp=x)
    exp = frac_reference(combo, "n", "n", alpha, A, B, beta, C0)
    for i in range(m):
        for j in range(n):
            er, ei = exp[i][j]
            assert abs(out[i, j].real - float(er)) <= 2.0 ** -52 * abs(float(er)) + 1e-300
            assert abs(out[i, j].imag - float(ei)) <= 2.0 ** -52 * abs(float(ei)) + 1e-300


# ---------------------------------------------------------------- identity vs numpy
def _cast(X, prec):
    X = np.asarray(X).astype(np.complex128)
    if prec == "s":
        return X.real.astype(np.float32).astype(np.float64) + 1j * X.imag.astype(np.float32).astype(np.float64)
    return X


@pytest.mark.parametrize("combo", synth.all_combos())
def test_identity_same_type_gemm(combo):
    """Every mixed case equals a complex128 gemm (numpy/BLAS) on explicitly cast and
    projected operands, with Re taken and the scalars projected when C is real."""
    dc, da, db, x = combo
    prec_c = "d" if dc in ("d", "z") else "s"
    comp = prec_c if x == "c" else x
    m, n, k = 23, 17, 41
    A, B, C0 = synth.problem(11, combo, m, n, k)
    case = oracle.oracle_case_of(dc, da, db)
    alpha = (1.25 - 0.5j) if case == 7 else 1.5
    beta = (-0.5 + 0.25j)
    Ah, Bh = _cast(A, comp), _cast(B, comp)
    ah = complex(_cast(np.array([alpha]), comp)[0]); bh = complex(_cast(np.array([beta]), prec_c)[0])
    C = C0.astype(np.complex128)
    if dc not in CPLX:
        if db not in CPLX:
            Ah = Ah.real
        if da not in CPLX:
            Bh = Bh.real
        want = bh.real * C.real + ah.real * (Ah @ Bh).real
    else:
        want = bh * C + ah * (Ah @ Bh)
    Cw = C0.copy(order="F")
    got = oracle_mxgemm("n", "n", alpha, A, B, beta, Cw, comp=x)
    scale = abs(alpha) * np.linalg.norm(Ah) * np.linalg.norm(Bh) + abs(beta) * np.linalg.norm(C)
    assert np.linalg.norm(got - want) / scale < 1e-14


# ---------------------------------------------------------------- 1m worked example
def _build_from_pattern(pattern, mats):
    R = np.zeros((len(pattern), len(pattern[0])))
    for r, row in enumerate(pattern):
        for c, ent in enumerate(row):
            sign = -1.0 if ent[0] == "-" else 1.0
            comp, name = ent[1:3], ent[4:]
            X = mats[name[0]]
            v = X[int(name[1]), int(name[2])]
            R[r, c] = sign * (v.real if comp == "re" else v.imag)
    return R


@pytest.mark.parametrize("variant", ["column", "row"])
def test_1m_worked_example(variant):
    """Eq. (1)/(2): the real product of the 1e/1r packed matrices equals the complex
    product, element for element, in the layout of C the equation shows. The oracle's
    case-3 result (beta = 0, alpha = 1) must equal that real product."""
    g = json.load(open(os.path.join(GOLDEN, "onem_example.json")))[variant]
    m, n, k = g["m"], g["n"], g["k"]
    A, B, _ = synth.problem(5, "zzzd", m, n, k)
    Cz = np.zeros((m, n), dtype=np.complex128, order="F")
    out = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, Cz, comp="d")
    Ar, Br = _build_from_pattern(g["A"], {"a": A}), _build_from_pattern(g["B"], {"b": B})
    Creal = Ar @ Br
    Cpat = _build_from_pattern(g["C"], {"c": out})
    assert np.allclose(Creal, Cpat, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- invariants
def test_real_C_ignores_discarded_imaginary_parts():
    """Cases 1a / 1b: with C real, Im(A) (B real) and Im(B) (A real) cannot matter."""
    for combo in ("dzdd", "sdcs", "ddzd", "scss"):
        A, B, C0 = synth.problem(3, combo, 9, 8, 7)
        A2, B2 = A.copy(), B.copy()
        if combo[1] in CPLX:
            A2 = (A2.real + 1j * (A2.imag + 3.0)).astype(A.dtype)
        if combo[2] in CPLX:
            B2 = (B2.real - 1j * (B2.imag * 5.0)).astype(B.dtype)
        C1, C2 = C0.copy(order="F"), C0.copy(order="F")
        r1 = oracle_mxgemm("n", "n", 1.5, A, B, -0.5, C1, comp=combo[3])
        r2 = oracle_mxgemm("n", "n", 1.5, A2, B2, -0.5, C2, comp=combo[3])
        assert np.array_equal(r1, r2) and np.array_equal(C1, C2)


def test_1c_imaginary_part_gets_only_beta():
    """Case 1c: Im(C_new) = Im(beta*C), whatever A and B are (real beta: beta*Im(C))."""
    for combo in ("zddd", "csss", "zsds"):
        A, B, C0 = synth.problem(4, combo, 6, 5, 9)
        C1 = C0.copy(order="F")
        r = oracle_mxgemm("n", "n", 2.0, A, B, -0.5, C1, comp=combo[3])
        assert np.array_equal(r.imag, -0.5 * C0.imag.astype(np.float64))


def test_conjugation_identities():
    """conj(A) conj(B) = conj(AB) via trans = conj-only, and A^H B^H = conj((BA)^T)."""
    A, B, _ = synth.problem(8, "zzzd", 7, 6, 5)
    Z = lambda: np.zeros((7, 6), dtype=np.complex128, order="F")
    ref = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, Z(), comp="d")
    cc = oracle_mxgemm("c", "c", 1.0, A, B, 0.0, Z(), comp="d")
    assert np.array_equal(cc, np.conj(ref))
    hh = oracle_mxgemm("h", "h", 1.0, np.conj(A).T.copy(), np.conj(B).T.copy(), 0.0, Z(), comp="d")
    assert np.array_equal(hh, ref)
    tt = oracle_mxgemm("t", "t", 1.0, A.T.copy(), B.T.copy(), 0.0, Z(), comp="d")
    assert np.array_equal(tt, ref)


def test_multiply_by_i():
    """Case 3: replacing A by i*A (a swap and negation of its planes) multiplies the
    product by i exactly."""
    A, B, _ = synth.problem(9, "zzzd", 5, 4, 6)
    Z = lambda: np.zeros((5, 4), dtype=np.complex128, order="F")
    ref = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, Z(), comp="d")
    iA = (1j * A).astype(A.dtype)
    got = oracle_mxgemm("n", "n", 1.0, iA, B, 0.0, Z(), comp="d")
    assert np.array_equal(got, 1j * ref)


def test_real_embedding_same_as_real_gemm():
    """A complex B with Im(B) = 0 under a real C gives the same as a real B (case 1b = 0)."""
    A, B, C0 = synth.problem(10, "sscs", 8, 7, 6)
    Breal = B.real.astype(np.float32)
    C1, C2 = C0.copy(order="F"), C0.copy(order="F")
    oracle_mxgemm("n", "n", 1.5, A, B, -0.5, C1, comp="s")
    oracle_mxgemm("n", "n", 1.5, A, np.asfortranarray(Breal), -0.5, C2, comp="s")
    assert np.array_equal(C1, C2)


# ---------------------------------------------------------------- scalar rules
@pytest.mark.parametrize("combo", ["sscs", "scss", "zdds", "dzzd", "zszd", "zzsd"])
def test_imaginary_alpha_rejected(combo):
    """Sec. 7.2: a non-zero Im(alpha) is an error in cases 1a, 1b, 1c, 2ab, 2ac, 2bc."""
    A, B, C0 = synth.problem(1, combo, 3, 3, 3)
    C1 = C0.copy(order="F")
    with pytest.raises(OracleError) as e:
        oracle_mxgemm("n", "n", 1.0 + 1e-3j, A, B, 1.0, C1, comp=combo[3])
    assert e.value.status == 2
    assert np.array_equal(C1, C0)


def test_case0_projects_complex_alpha_and_beta():
    """Sec. 7.2: with all operands real, Im(alpha) and Im(beta) are dropped."""
    A, B, C0 = synth.problem(2, "dddd", 4, 5, 6)
    C1, C2 = C0.copy(order="F"), C0.copy(order="F")
    r1 = oracle_mxgemm("n", "n", 1.5 + 7j, A, B, -0.5 - 3j, C1, comp="d")
    r2 = oracle_mxgemm("n", "n", 1.5, A, B, -0.5, C2, comp="d")
    assert np.array_equal(r1, r2)


def test_beta_zero_does_not_read_C_and_k_zero_scales():
    A, B, C0 = synth.problem(2, "dddd", 4, 5, 6)
    Cn = np.full_like(C0, np.nan)
    r = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, Cn, comp="d")
    assert np.all(np.isfinite(r)) and np.all(np.isfinite(Cn))
    A0 = np.zeros((4, 0)); B0 = np.zeros((0, 5))
    C1 = C0.copy(order="F")
    r = oracle_mxgemm("n", "n", 3.0, A0, B0, -0.5, C1, comp="d")
    assert np.array_equal(C1, -0.5 * C0)
    Ce = np.zeros((0, 5))
    oracle_mxgemm("n", "n", 1.0, np.zeros((0, 3)), np.zeros((3, 5)), 1.0, Ce, comp="d")


def test_compensated_sum_is_exact_on_cancellation():
    """Dot2 (Ogita-Rump-Oishi): 1e16 + 1 - 1e16 + 1 sums to 2 exactly; a plain
    binary64 loop gives 1."""
    A = np.array([[1e16, 1.0, -1e16, 1.0]])
    B = np.ones((4, 1))
    C = np.zeros((1, 1))
    r = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, C, comp="d")
    assert r[0, 0] == 2.0
    acc = 0.0
    for v in A[0]:
        acc += v
    assert acc != 2.0


def test_case_table_matches_figure():
    g = json.load(open(os.path.join(GOLDEN, "mixeddom.json")))
    order = ["0", "1b", "1a", "2ab", "1c", "2bc", "2ac", "3"]
    for row in g["cases"]:
        dc = "z" if row["C"] == "C" else "d"
        da = "z" if row["A"] == "C" else "d"
        db = "z" if row["B"] == "C" else "d"
        assert order[oracle.oracle_case_of(dc, da, db)] == row["case"]


def test_alpha_zero_does_not_read_A_and_B():
    """alpha == 0 (after its cast): C := beta*C and non-finite A or B cannot leak in."""
    A, B, C0 = synth.problem(12, "zzzs", 4, 5, 6)
    A[0, 0] = np.nan
    B[1, 1] = np.inf
    C1 = C0.copy(order="F")
    oracle_mxgemm("n", "n", 1e-50, A, B, -0.5, C1, comp="s")   # 1e-50 rounds to 0 in single
    assert np.array_equal(C1, (-0.5 * C0).astype(C0.dtype))


# ---------------------------------------------------------------- literal complex alpha
def frac_literal(combo, transa, transb, alpha, A, B, beta, C):
    """Sec. 7.2's literal interpretation in exact rationals: all domains at face value,
    C_new = beta*C + alpha*op(A)*op(B) in complex arithmetic, then projected onto C's
    domain (Re when C is real)."""
    dc, da, db, x = combo
    prec_c = "d" if dc in ("d", "z") else "s"
    comp = prec_c if x == "c" else x
    opA, opB = _fr_op(A, transa), _fr_op(B, transb)
    m, k = len(opA), len(opA[0]) if opA else 0
    n = len(opB[0]) if opB else 0
    cast = lambda z: (Fraction(_rnd(float(z[0]), comp)), Fraction(_rnd(float(z[1]), comp)))
    Ah = [[cast(v) for v in r] for r in opA]
    Bh = [[cast(v) for v in r] for r in opB]
    al, be = complex(alpha), complex(beta)
    ar, ai = Fraction(_rnd(al.real, comp)), Fraction(_rnd(al.imag, comp))
    br, bi = Fraction(_rnd(be.real, prec_c)), Fraction(_rnd(be.imag, prec_c))
    if dc not in CPLX:
        bi = Fraction(0)
    Cin = [[complex(v) for v in r] for r in np.asarray(C).tolist()]
    res = []
    for i in range(m):
        row = []
        for j in range(n):
            pr = sum((Ah[i][p][0] * Bh[p][j][0] - Ah[i][p][1] * Bh[p][j][1] for p in range(k)), Fraction(0))
            pi = sum((Ah[i][p][0] * Bh[p][j][1] + Ah[i][p][1] * Bh[p][j][0] for p in range(k)), Fraction(0))
            cr, ci = Fraction(Cin[i][j].real), Fraction(Cin[i][j].imag)
            re = br * cr - bi * ci + ar * pr - ai * pi
            im = br * ci + bi * cr + ar * pi + ai * pr
            row.append((re, Fraction(0) if dc not in CPLX else im))
        res.append(row)
    return res


@pytest.mark.parametrize("combo", [c for c in synth.all_combos()
                                   if oracle.oracle_case_of(c[0], c[1], c[2]) not in (0, 7)])
def test_literal_alpha_bruteforce(combo):
    """Literal complex alpha in the six mixed cases equals the exact face-value result."""
    rng = np.random.default_rng(abs(hash(combo + "lit")) % (2 ** 32))
    dc, da, db = combo[:3]
    for ta, tb in (("n", "n"), ("t", "c"), ("h", "t")):
        m, n, k = (int(v) for v in rng.integers(1, 4, size=3))
        A = _dyadic(rng, (k, m) if ta in "th" else (m, k), da)
        B = _dyadic(rng, (n, k) if tb in "th" else (k, n), db)
        C0 = _dyadic(rng, (m, n), dc)
        alpha, beta = 0.75 - 1.25j, (0.5 + 0.25j) if dc in CPLX else -0.5
        Cw = np.asfortranarray(C0.copy())
        out = oracle_mxgemm(ta, tb, alpha, A, B, beta, Cw, comp=combo[3], literal_alpha=True)
        exp = frac_literal(combo, ta, tb, alpha, A, B, beta, C0)
        for i in range(m):
            for j in range(n):
                assert out[i, j].real == float(exp[i][j][0]) and out[i, j].imag == float(exp[i][j][1]), \
                    (combo, ta, tb, i, j)
    # without the flag the same call is the paper's error
    with pytest.raises(OracleError):
        oracle_mxgemm("n", "n", 1j, synth.matrix(rng, 2, 2, da), synth.matrix(rng, 2, 2, db), 1.0,
                      synth.matrix(rng, 2, 2, dc), comp=combo[3])


def test_literal_alpha_agrees_with_paper_rule_for_real_alpha():
    """For real alpha the literal reading and the paper's rule coincide."""
    for combo in ("dzdd", "sszs", "dczd", "zsds", "zzsd", "cdzs"):
        A, B, C0 = synth.problem(31, combo, 7, 6, 5)
        C1, C2 = C0.copy(order="F"), C0.copy(order="F")
        r1 = oracle_mxgemm("n", "n", -1.5, A, B, 0.5, C1, comp=combo[3])
        r2 = oracle_mxgemm("n", "n", -1.5, A, B, 0.5, C2, comp=combo[3], literal_alpha=True)
        assert np.array_equal(r1, r2)


# ---------------------------------------------------------------- 16-bit formats (Sec. 5.3)
from oracle import oracle_round


def _bf16_ref(x):
    """bfloat16 round-to-nearest-even of a binary32-representable value, on its bits."""
    u = int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    if (u & 0x7F800000) == 0x7F800000:
        return float(np.float32(x))
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return float(np.array([u], dtype=np.uint32).view(np.float32)[0])


def test_binary16_rounding_matches_numpy():
    rng = np.random.default_rng(1)
    xs = list(rng.standard_normal(4000) * 10.0 ** rng.uniform(-9, 6, 4000))
    # exact ties between neighbouring binary16 values, subnormals, the overflow edge
    h = np.arange(0, 0x7C00, 7, dtype=np.uint16).view(np.float16).astype(np.float64)
    xs += list((h[:-1] + h[1:]) / 2) + [65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26]
    for x in xs:
        for v in (x, -x):
            assert oracle_round(v, "h") == float(np.float16(v)), v


def test_bfloat16_rounding_matches_bit_rule():
    rng = np.random.default_rng(2)
    xs = [float(np.float32(v)) for v in rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)]
    b = (np.arange(0, 0x7F80, 5, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)
    xs += list((b[:-1] + b[1:]) / 2)                       # ties (representable in binary32)
    tie = (2.0 - 2.0 ** -8) * 2.0 ** 127      # halfway between the largest finite value and 2^128
    xs += [float(np.float32(1e-40)), (2.0 - 2.0 ** -7) * 2.0 ** 127]
    for x in xs:
        for v in (x, -x):
            assert oracle_round(v, "b") == _bf16_ref(v), v
    # the overflow edge (ties to even: the largest finite value has an odd significand)
    assert oracle_round(tie, "b") == float("inf")
    assert oracle_round(np.nextafter(tie, 0.0), "b") == (2.0 - 2.0 ** -7) * 2.0 ** 127
    assert oracle_round(-tie, "b") == float("-inf")


_SAMPLE16 = [c for i, c in enumerate(synth.all_combos_16()) if i % 11 == 0]


def _rnd16(x, prec):
    if prec == "s":
        return float(np.float32(x))
    if prec == "h":
        return float(np.float16(x))
    if prec == "b":
        return _bf16_ref(x)
    return float(x)


@pytest.mark.parametrize("combo", _SAMPLE16)
def test_bruteforce_exact_16bit_combos(combo):
    """Tiny dyadic inputs in 16-bit storage and precisions: the oracle equals the exact
    rational statement of the case table bit for bit, and rounds C correctly."""
    rng = np.random.default_rng(abs(hash(combo + "16")) % (2 ** 32))
    dc, da, db, x = combo
    prec = {"s": "s", "c": "s", "d": "d", "z": "d", "h": "h", "k": "h", "b": "b", "w": "b"}
    for ta, tb in (("n", "n"), ("t", "h"), ("c", "t")):
        m, n, k = (int(v) for v in rng.integers(1, 4, size=3))
        def dy(shape, dt):
            re = rng.integers(-8, 9, size=shape) / 4.0
            im = rng.integers(-8, 9, size=shape) / 4.0 if synth.is_complex(dt) else 0.0
            return synth.from_values(re + 1j * im, dt)
        A = dy((k, m) if ta in "th" else (m, k), da)
        B = dy((n, k) if tb in "th" else (k, n), db)
        C0 = dy((m, n), dc)
        case = oracle.oracle_case_of(dc, da, db)
        alpha = (0.75 + 0.5j) if case in (0, 7) else -1.5
        beta = [0.0, -0.5, 1.0, 0.25 - 0.75j][int(rng.integers(0, 4))]
        Cw = C0.copy()
        out = oracle_mxgemm(ta, tb, alpha, A, B, beta, Cw, comp=x)
        # the rational statement, with the 16-bit cast done by numpy / the bit rule
        opA, opB = synth.to_c128(A), synth.to_c128(B)
        if ta in "th": opA = opA.T
        if tb in "th": opB = opB.T
        if ta in "ch": opA = np.conj(opA)
        if tb in "ch": opB = np.conj(opB)
        comp = prec[dc] if x == "c" else x
        exp = frac_reference(combo if x in "sd" else dc + da + db + "d", "n", "n",
                             complex(_rnd16(np.real(alpha), comp), _rnd16(np.imag(alpha), comp)),
                             opA, opB, complex(_rnd16(np.real(beta), prec[dc]), _rnd16(np.imag(beta), prec[dc])),
                             synth.to_c128(C0) if synth.is_complex(dc) else synth.to_c128(C0).real)
        got = synth.to_c128(Cw)
        for i in range(m):
            for j in range(n):
                er, ei = float(exp[i][j][0]), float(exp[i][j][1])
                assert out[i, j].real == er and out[i, j].imag == ei, (combo, ta, tb, i, j)
                assert got[i, j].real == _rnd16(er, prec[dc]), (combo, i, j)
                if synth.is_complex(dc):
                    assert got[i, j].imag == _rnd16(ei, prec[dc])


@pytest.mark.parametrize("combo", _SAMPLE16)
def test_identity_16bit_combos(combo):
    """The 16-bit combinations equal a complex128 numpy gemm on operands cast to the
    computation precision (numpy's float16 / the bfloat16 bit rule) and projected."""
    dc, da, db, x = combo
    prec = {"s": "s", "c": "s", "d": "d", "z": "d", "h": "h", "k": "h", "b": "b", "w": "b"}
    comp = prec[dc] if x == "c" else x
    A, B, C0 = synth.problem(21, combo, 13, 11, 17)
    cast = np.vectorize(lambda v: _rnd16(v, comp))
    Ah = cast(synth.to_c128(A).real) + 1j * cast(synth.to_c128(A).imag)
    Bh = cast(synth.to_c128(B).real) + 1j * cast(synth.to_c128(B).imag)
    case = oracle.oracle_case_of(dc, da, db)
    alpha = (1.25 - 0.5j) if case == 7 else 1.5
    ah = complex(_rnd16(np.real(alpha), comp), _rnd16(np.imag(alpha), comp))
    bh = complex(_rnd16(-0.5, prec[dc]), _rnd16(0.25, prec[dc]))
    C = synth.to_c128(C0)
    if not synth.is_complex(dc):
        if not synth.is_complex(db):
            Ah = Ah.real
        if not synth.is_complex(da):
            Bh = Bh.real
        want = bh.real * C.real + ah.real * (Ah @ Bh).real
    else:
        want = bh * C + ah * (Ah @ Bh)
    got = oracle_mxgemm("n", "n", alpha, A, B, -0.5 + 0.25j, C0.copy(), comp=x)
    scale = abs(alpha) * np.linalg.norm(Ah) * np.linalg.norm(Bh) + np.linalg.norm(C)
    assert np.linalg.norm(got - want) / scale < 1e-14


def test_complex_beta_epilogue_rounding_exceeds_two_units():
    """Pin of the tolerance's C-precision term for a complex beta: the epilogue's order of
    operations in single precision (Sec. 7.1: beta*C as a naive complex product of four
    rounded products and two rounded sums, then alpha*AB added with one more rounding)
    can be 2.9 u away from the exact value in the normwise measure -- more than the 2 u of
    a real beta, within the (1 + sqrt(5)) u of the Brent-Percival-Zimmermann bound for
    the complex product plus the final rounding. Exact rational arithmetic, numpy float32
    for the roundings."""
    from fractions import Fraction as Fr
    f = np.float32
    br, bi = f(float.fromhex("-0x1.deb1eep-1")), f(float.fromhex("0x1.a777fep-1"))
    cr, ci = f(float.fromhex("-0x1.122232p-1")), f(float.fromhex("-0x1.41cd64p-1"))
    t = f(2.0 ** -24)
    re = f(f(f(br * cr) - f(bi * ci)) + t)
    im = f(f(br * ci) + f(bi * cr))
    R = lambda x: Fr(float(x))
    ex_re = R(br) * R(cr) - R(bi) * R(ci) + R(t)
    ex_im = R(br) * R(ci) + R(bi) * R(cr)
    num = float((R(re) - ex_re) ** 2 + (R(im) - ex_im) ** 2) ** 0.5
    den = float((R(br) ** 2 + R(bi) ** 2) * (R(cr) ** 2 + R(ci) ** 2)) ** 0.5 + float(t)
    u = 2.0 ** -24
    assert 2.0 * u < num / den <= (1.0 + 5.0 ** 0.5) * u
