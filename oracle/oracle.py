"""ctypes binding of the C oracle ``mxg_oracle.c`` (test infrastructure only).

The oracle states mixed-datatype gemm, C := beta*C + alpha*op(A)*op(B), directly in
binary64 / complex binary64 (arXiv 1901.06015, Fig. "mixeddom", Secs. 4.2, 5.1, 7).
This module only marshals numpy arrays into the C function; all arithmetic is in C.
Arrays are passed as they are stored: for trans T or conj-trans, A is the stored
k x m matrix (and B the stored n x k matrix).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mxg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmxg_oracle.so")

DT_CODES = {"s": 0, "d": 1, "c": 2, "z": 3, "h": 4, "k": 5, "b": 6, "w": 7}
# numpy has no complex binary16 and no bfloat16: structured dtypes of 16-bit fields
CHALF = np.dtype([("re", "<f2"), ("im", "<f2")])
BF16 = np.dtype([("bits", "<u2")])
CBF16 = np.dtype([("re", "<u2"), ("im", "<u2")])
NP_OF_DT = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128,
            "h": np.float16, "k": CHALF, "b": BF16, "w": CBF16}
PREC_CODES = {"s": 0, "d": 1, "c": 2, "h": 3, "b": 4}
TRANS_CODES = {"n": 0, "t": 1, "c": 2, "h": 3}

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__({1: "invalid argument",
                          2: "imaginary alpha in a case that forbids it"}.get(status, str(status)))
        self.status = status


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FP contraction: Dot2 needs exact
    error-free transformations)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.oracle_mxgemm.restype = i32
            lib.oracle_mxgemm.argtypes = [i32, i32, i64, i64, i64, dbl, dbl,
                                          vp, i32, i64, i64, vp, i32, i64, i64,
                                          dbl, dbl, vp, i32, i64, i64, i32, vp, i32, i32]
            lib.oracle_case_of.restype = i32
            lib.oracle_case_of.argtypes = [i32, i32, i32]
            lib.oracle_round.restype = dbl
            lib.oracle_round.argtypes = [dbl, i32]
            _lib = lib
    return _lib


def _dt_of(arr):
    for k, v in NP_OF_DT.items():
        if arr.dtype == np.dtype(v):
            return k
    raise TypeError(f"unsupported dtype {arr.dtype}")


def oracle_round(x, prec):
    """The oracle's rounding of a binary64 value to precision 's', 'd', 'h' or 'b'."""
    return _load().oracle_round(float(x), PREC_CODES[prec])


def _strides(arr):
    it = arr.dtype.itemsize
    rs, cs = arr.strides
    if rs % it or cs % it:
        raise ValueError("strides must be whole elements")
    return rs // it, cs // it


def oracle_case_of(dtc, dta, dtb):
    return _load().oracle_case_of(DT_CODES[dtc], DT_CODES[dta], DT_CODES[dtb])


def oracle_mxgemm(transa, transb, alpha, A, B, beta, C, comp="c", nthreads=None, literal_alpha=False):
    """C := beta*C + alpha*op(A)*op(B), in place on the numpy array C.

    ``transa``/``transb`` in {'n','t','c','h'} ('c' = conjugate without transpose,
    'h' = conjugate transpose); ``comp`` in {'s','d','h','b','c'} where 'c' means "the
    precision of C" (Sec. 5.1.1) and 'h' / 'b' are binary16 / bfloat16. ``alpha`` and ``beta`` are Python numbers (complex
    allowed). Returns the unrounded result C_new as a complex128 m x n array.
    """
    A = np.asarray(A); B = np.asarray(B)
    if not isinstance(C, np.ndarray):
        raise TypeError("C must be a numpy array (updated in place)")
    ta, tb = TRANS_CODES[transa], TRANS_CODES[transb]
    m, n = C.shape
    k = A.shape[0] if ta in (1, 3) else A.shape[1]
    if (A.shape[1] if ta in (1, 3) else A.shape[0]) != m:
        raise ValueError("A shape does not match C")
    if (B.shape[0] if tb in (1, 3) else B.shape[1]) != n or \
       (B.shape[1] if tb in (1, 3) else B.shape[0]) != k:
        raise ValueError("B shape does not match")
    compc = PREC_CODES[comp]
    if nthreads is None:
        nthreads = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
    out = np.zeros((m, n), dtype=np.complex128, order="F")
    al, be = complex(alpha), complex(beta)
    rsa, csa = _strides(A); rsb, csb = _strides(B); rsc, csc = _strides(C)
    st = _load().oracle_mxgemm(ta, tb, m, n, k, al.real, al.imag,
                               A.ctypes.data, DT_CODES[_dt_of(A)], rsa, csa,
                               B.ctypes.data, DT_CODES[_dt_of(B)], rsb, csb,
                               be.real, be.imag,
                               C.ctypes.data, DT_CODES[_dt_of(C)], rsc, csc,
                               compc, out.ctypes.data, int(nthreads), 1 if literal_alpha else 0)
    if st != 0:
        raise OracleError(st)
    return out
