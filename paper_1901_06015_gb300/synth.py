"""Seeded synthetic inputs for mixed-datatype gemm.

This module only draws random matrices; it holds none of the method's arithmetic.
Both the oracle-based tests and the CUDA path take their inputs from here.

Recipe (the paper's experiments use randomized, column-stored matrices with
alpha = beta = 1, Sec. 8.2.1; no dataset is involved):
  * ``numpy.random.default_rng(seed)``; fill order A.re, A.im, B.re, B.im, C.re, C.im;
    each component drawn in float64 then rounded (RN-even) to the storage type.
  * "uniform": each real component ~ U[-1, 1].
  * "loguniform": sign * 10**U(-4, 4) with a random sign (magnitudes 1e-4..1e4).
  * "smallint": integers in {-4, ..., 4}; with these, every product and partial sum
    of a gemm with k <= 1024 is an integer below 2**24, so exact in every precision.
"""
import numpy as np

# Storage datatypes: s, d, c, z (binary32/64, real/complex) and, beyond the paper's
# four, h / k (binary16 real / complex) and b / w (bfloat16 real / complex). numpy has
# no complex binary16 and no bfloat16, so those are structured dtypes of 16-bit fields
# (bfloat16 fields hold bit patterns).
CHALF = np.dtype([("re", "<f2"), ("im", "<f2")])
BF16 = np.dtype([("bits", "<u2")])
CBF16 = np.dtype([("re", "<u2"), ("im", "<u2")])
NP_OF_DT = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128,
            "h": np.float16, "k": CHALF, "b": BF16, "w": CBF16}
DTS = ("s", "d", "c", "z")
DTS_ALL = ("s", "d", "c", "z", "h", "k", "b", "w")
COMPLEX_DTS = ("c", "z", "k", "w")


def all_combos():
    """All 128 labels ``cabx`` of the paper: C, A, B storage datatypes (s, d, c, z) then
    the computation precision (s, d)."""
    return [c + a + b + x for c in DTS for a in DTS for b in DTS for x in ("s", "d")]


def all_combos_16():
    """Labels with at least one 16-bit storage datatype or a 16-bit computation
    precision (h: binary16, b: bfloat16)."""
    out = []
    for c in DTS_ALL:
        for a in DTS_ALL:
            for b in DTS_ALL:
                for x in ("s", "d", "h", "b"):
                    if x in ("h", "b") or any(t not in DTS for t in (c, a, b)):
                        out.append(c + a + b + x)
    return out


def is_complex(dt):
    return dt in COMPLEX_DTS


def _bf16_bits_from_f32(x32):
    """bfloat16 bit patterns (round-to-nearest-even) of binary32 values (input
    generation only)."""
    u = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def from_values(val, dt, order="F"):
    """Store complex128 (or real) values in datatype dt, rounding to its precision."""
    val = np.asarray(val)
    if dt in ("s", "d", "c", "z", "h"):
        v = val if is_complex(dt) else np.real(val)
        return np.asarray(v, dtype=NP_OF_DT[dt], order=order)
    out = np.empty(val.shape, dtype=NP_OF_DT[dt], order=order)
    if dt == "k":
        out["re"] = np.real(val).astype(np.float16)
        out["im"] = np.imag(val).astype(np.float16)
    elif dt == "b":
        out["bits"] = _bf16_bits_from_f32(np.real(val).astype(np.float32))
    else:
        out["re"] = _bf16_bits_from_f32(np.real(val).astype(np.float32))
        out["im"] = _bf16_bits_from_f32(np.imag(val).astype(np.float32))
    return out


def _bf16_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def to_c128(arr, dt=None):
    """Values of a stored matrix as complex128 (exact)."""
    arr = np.asarray(arr)
    if arr.dtype == CHALF:
        return arr["re"].astype(np.float64) + 1j * arr["im"].astype(np.float64)
    if arr.dtype == BF16:
        return _bf16_to_f64(arr["bits"]).astype(np.complex128)
    if arr.dtype == CBF16:
        return _bf16_to_f64(arr["re"]) + 1j * _bf16_to_f64(arr["im"])
    return arr.astype(np.complex128)


def _component(rng, shape, dist):
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=shape)
    if dist == "loguniform":
        mag = 10.0 ** rng.uniform(-4.0, 4.0, size=shape)
        sign = np.where(rng.uniform(size=shape) < 0.5, -1.0, 1.0)
        return sign * mag
    if dist == "smallint":
        return rng.integers(-4, 5, size=shape).astype(np.float64)
    raise ValueError(dist)


def matrix(rng, rows, cols, dt, dist="uniform", order="F"):
    """One rows x cols matrix of storage datatype ``dt``."""
    re = _component(rng, (rows, cols), dist)
    if is_complex(dt):
        im = _component(rng, (rows, cols), dist)
        val = re + 1j * im
    else:
        val = re
    return from_values(val, dt, order)


def problem(seed, combo, m, n, k, dist="uniform", transa="n", transb="n",
            order_a="F", order_b="F", order_c="F"):
    """Inputs of one gemm: returns (A, B, C) numpy arrays in their stored shapes.

    A is stored m x k (k x m for trans 't'/'h'); B is stored k x n (n x k for 't'/'h').
    """
    dc, da, db = combo[0], combo[1], combo[2]
    rng = np.random.default_rng(seed)
    a_shape = (k, m) if transa in ("t", "h") else (m, k)
    b_shape = (n, k) if transb in ("t", "h") else (k, n)
    # fill order A.re, A.im, B.re, B.im, C.re, C.im
    A = matrix(rng, *a_shape, da, dist, order_a)
    B = matrix(rng, *b_shape, db, dist, order_b)
    C = matrix(rng, m, n, dc, dist, order_c)
    return A, B, C


def torch_matrix(gen, rows, cols, dt, device, low=-1.0, high=1.0):
    """Device-side uniform matrix, column-major (stored as the transpose of a row-major
    cols x rows tensor). Used for the large benchmark inputs, which are checked
    against the oracle on sampled blocks copied back to the host. A complex 16-bit
    matrix is a (rows, cols, 2) float16 / bfloat16 tensor."""
    import torch
    if dt in ("h", "k", "b", "w"):
        t16 = torch.float16 if dt in ("h", "k") else torch.bfloat16
        ncomp = 2 if dt in ("k", "w") else 1
        raw = torch.empty((cols, rows, ncomp), dtype=torch.float32, device=device)
        raw.uniform_(low, high, generator=gen)
        raw = raw.to(t16)
        return raw.permute(1, 0, 2) if ncomp == 2 else raw[..., 0].t()
    tdt = {"s": torch.float32, "d": torch.float64,
           "c": torch.complex64, "z": torch.complex128}[dt]
    real = torch.float64 if dt in ("d", "z") else torch.float32
    ncomp = 2 if is_complex(dt) else 1
    raw = torch.empty((cols, rows, ncomp), dtype=real, device=device)
    raw.uniform_(low, high, generator=gen)
    if ncomp == 2:
        t = torch.view_as_complex(raw)
    else:
        t = raw[..., 0]
    assert t.dtype == tdt
    return t.t()  # rows x cols view with unit row stride
