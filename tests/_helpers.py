"""Shared test helpers: tolerance (normwise error bound) and operand norms.

The stated bound is  ||C_gpu - C_ref||_F / (|alpha| ||A~||_F ||B~||_F + |beta| ||C||_F)
                     <= 4 k u_x
u_x is the unit roundoff of the summation in the computation precision (2^-24 single and
the 16-bit precisions, which sum in FP32; 2^-53 double). A~ and B~ are the operands as
they enter the product: Re(A) when C and B are real, Re(B) when C and A are real, else
the full operand. C_ref is the oracle's unrounded binary64 result, after the same casts
of A, B and alpha to the computation precision (so those casts cost nothing here).

What 4 k u_x has to cover: the length-K' accumulation (K' <= 2k in the 1m / 1r
layouts, at most one rounding per term: 2 k u_x), the product alpha*acc (at most sqrt(5)
u_x for a complex alpha: a naive complex product, Brent-Percival-Zimmermann) and the
epilogue's roundings in C's precision u_C (Sec. 7.1: the cast of alpha*AB, beta*C and
the sum): at most 2 u_C with a real beta, (1 + sqrt(5)) u_C with a complex beta and a
complex C. When u_C <= u_x and k >= 4 these fit in the 2 k u_x left over. A C-precision
term is added only where they cannot:
  * u_C > u_x (C stored in a lower precision than the summation: single-precision C
    after double computation, 16-bit C): storing C alone costs up to u_C >> 4 k u_x;
  * k < 4: the epilogue's fixed roundings are not covered by the 2 k u_x slack.
The split-precision methods run only where the stated bound holds for them (their k
limits, MXG_SPLIT_MIN_K_*); tolerance() refuses to give a bound below those limits.
"""
import numpy as np

U = {"s": 2.0 ** -24, "d": 2.0 ** -53, "h": 2.0 ** -11, "b": 2.0 ** -8}
# unit roundoff of the summation for each computation precision: the 16-bit precisions
# round A and B to binary16 / bfloat16 (as the oracle does) and sum in FP32
U_SUM = {"s": 2.0 ** -24, "d": 2.0 ** -53, "h": 2.0 ** -24, "b": 2.0 ** -24}
# smallest k the planner accepts for the split-precision methods (include/mxgemm.h)
SPLIT_MIN_K = {"bf16x3": 320, "tf32x3": 32}


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


def tolerance(combo, k, method=None, beta=0.0):
    """Normwise bound for combo at depth k (see the module docstring). ``beta`` only
    matters through whether it is complex (with a complex C)."""
    if method in SPLIT_MIN_K and k < SPLIT_MIN_K[method]:
        raise ValueError(f"{method} is not accepted below k = {SPLIT_MIN_K[method]}")
    x = comp_prec(combo)
    u_c = U[prec_of(combo[0])]
    tol = 4.0 * max(k, 1) * U_SUM[x]
    complex_beta = is_complex(combo[0]) and complex(beta).imag != 0.0
    e_c = (1.0 + 5.0 ** 0.5) * u_c if complex_beta else 2.0 * u_c
    if u_c > U_SUM[x]:
        tol += e_c
    elif k < 4:
        tol += e_c + 5.0 ** 0.5 * U_SUM[x]
    return tol


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
