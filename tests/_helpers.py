"""Shared test helpers: tolerance (normwise error bound) and operand norms.

The bound is  ||C_gpu - C_ref||_F / (|alpha| ||A~||_F ||B~||_F + |beta| ||C||_F)
              <= 4 k u_x + 4 u_C
u_x is the unit roundoff of the computation precision (2^-24 single, 2^-53 double),
u_C that of C's storage precision. The 4 k u_x term bounds the length-k (or 2k, for
the 1m / 1r layouts) accumulation; the 4 u_C term bounds the epilogue's roundings in
C's storage precision (beta*C with complex beta: two products and a sum; the cast of
alpha*AB; the final sum). A~ and B~ are the operands as they enter the product:
Re(A) when C and B are real, Re(B) when C and A are real, else the full operand.
"""
import numpy as np

U = {"s": 2.0 ** -24, "d": 2.0 ** -53, "h": 2.0 ** -11, "b": 2.0 ** -8}
# unit roundoff of the summation for each computation precision: the 16-bit precisions
# round A and B to binary16 / bfloat16 (as the oracle does) and sum in FP32
U_SUM = {"s": 2.0 ** -24, "d": 2.0 ** -53, "h": 2.0 ** -24, "b": 2.0 ** -24}


def prec_of(dt):
    return {"d": "d", "z": "d", "h": "h", "k": "h", "b": "b", "w": "b"}.get(dt, "s")


def is_complex(dt):
    return dt in ("c", "z", "k", "w")


def comp_prec(combo):
    x = combo[3]
    return prec_of(combo[0]) if x == "c" else x


def op(X, trans):
    from paper_1901_06015_gb300 import synth
    X = synth.to_c128(np.asarray(X))
    if trans in ("t", "h"):
        X = X.T
    if trans in ("c", "h"):
        X = np.conj(X)
    return X


# Error floor of the split-precision products, relative to |a||b| per product. With
# unit roundoff u of the plane format (BF16: 8 significant bits, u = 2^-8; TF32: 11
# bits, u = 2^-11), X = X_hi + X_lo + r with |X - X_hi| <= u|X| and |r| <= u^2 |X|; the
# product drops lo*lo and the two residual terms, each <= u^2 |a||b|, so the error per
# product is <= 3 u^2 |a||b| (+ O(u^3)). By Cauchy-Schwarz the normwise error of the
# whole product is at most that floor: 3 * 2^-16 for BF16x3, 3 * 2^-22 for TF32x3.
U_SPLIT = {"bf16x3": 3.0 * 2.0 ** -16 * (1 + 2.0 ** -7), "tf32x3": 3.0 * 2.0 ** -22 * (1 + 2.0 ** -10)}


def tolerance(combo, k, method=None):
    tol = 4.0 * max(k, 1) * U_SUM[comp_prec(combo)] + 4.0 * U[prec_of(combo[0])]
    return tol + U_SPLIT.get(method, 0.0)


def entering_norms(combo, A, B, transa="n", transb="n"):
    dc, da, db = combo[0], combo[1], combo[2]
    Ae, Be = op(A, transa), op(B, transb)
    if not is_complex(dc) and not is_complex(db):
        Ae = Ae.real
    if not is_complex(dc) and not is_complex(da):
        Be = Be.real
    return float(np.linalg.norm(Ae)), float(np.linalg.norm(Be))


def normwise_error(combo, C_gpu, C_ref, A, B, C_in, alpha, beta, transa="n", transb="n"):
    """Return (err, bound-denominator) for C_gpu against the oracle's unrounded C_ref."""
    na, nb = entering_norms(combo, A, B, transa, transb)
    from paper_1901_06015_gb300 import synth
    den = abs(alpha) * na * nb + abs(beta) * float(np.linalg.norm(synth.to_c128(np.asarray(C_in))))
    diff = synth.to_c128(np.asarray(C_gpu)) - np.asarray(C_ref)
    num = float(np.linalg.norm(diff))
    return (num / den if den > 0 else num), den
