"""GPU-test utilities: move numpy inputs to the device keeping their layout, run the
library, bring C back."""
import numpy as np


def _to_device_16(arr):
    """Device copy of a 16-bit matrix (binary16 / bfloat16, real or complex) with the
    same column- or row-major layout; complex ones become (rows, cols, 2) tensors."""
    import torch
    from paper_1901_06015_gb300 import synth
    if not (arr.flags["F_CONTIGUOUS"] or arr.flags["C_CONTIGUOUS"]):
        raise ValueError("16-bit test matrices are column- or row-major")
    col = bool(arr.flags["F_CONTIGUOUS"])
    if arr.dtype == np.float16:
        t = torch.from_numpy(np.array(arr.T if col else arr, order="C")).cuda()
        return t.t() if col else t
    if arr.dtype == synth.CHALF:
        vals = np.stack([arr["re"], arr["im"]], axis=-1)            # float16 (rows, cols, 2)
        tdt = None
    elif arr.dtype == synth.BF16:
        bits = arr["bits"]
        t = torch.from_numpy(np.array(bits.T if col else bits, order="C").view(np.int16)).cuda().view(torch.bfloat16)
        return t.t() if col else t
    else:
        vals = np.stack([arr["re"], arr["im"]], axis=-1).view(np.int16)  # bfloat16 bits
        tdt = torch.bfloat16
    v = np.ascontiguousarray(vals.transpose(1, 0, 2) if col else vals)
    t = torch.from_numpy(v).cuda()
    if tdt is not None:
        t = t.view(tdt)
    return t.permute(1, 0, 2) if col else t


def from_device(t, dt):
    """Numpy copy of a device matrix in the storage dtype of dt."""
    import torch
    from paper_1901_06015_gb300 import synth
    if dt in ("s", "d", "c", "z", "h"):
        return t.cpu().numpy()
    x = t.detach().cpu()
    if dt == "k":
        v = x.numpy()
        out = np.empty(v.shape[:2], dtype=synth.CHALF)
        out["re"], out["im"] = v[..., 0], v[..., 1]
        return out
    bits = x.view(torch.int16).numpy().view(np.uint16)
    if dt == "b":
        out = np.empty(bits.shape, dtype=synth.BF16)
        out["bits"] = bits
        return out
    out = np.empty(bits.shape[:2], dtype=synth.CBF16)
    out["re"], out["im"] = bits[..., 0], bits[..., 1]
    return out


def to_device(arr):
    """Device copy of a numpy 2-D array with the same strides (including general
    strides of a view into a larger buffer)."""
    import torch
    from paper_1901_06015_gb300 import synth
    arr = np.asarray(arr)
    if arr.dtype in (np.float16, synth.CHALF, synth.BF16, synth.CBF16):
        return _to_device_16(arr)
    it = arr.itemsize
    rs, cs = arr.strides[0] // it, arr.strides[1] // it
    if arr.flags["F_CONTIGUOUS"] or arr.flags["C_CONTIGUOUS"]:
        return torch.from_numpy(np.array(arr, order="K")).cuda()
    # general storage: copy the whole span into a flat device buffer, view with strides
    span = (arr.shape[0] - 1) * rs + (arr.shape[1] - 1) * cs + 1
    flat = np.zeros(span, dtype=arr.dtype)
    base = np.lib.stride_tricks.as_strided(flat, shape=arr.shape, strides=arr.strides)
    base[...] = arr
    dev = torch.from_numpy(flat).cuda()
    return dev.as_strided(arr.shape, (rs, cs))


def run(combo, A, B, C, alpha, beta, transa="n", transb="n", method="auto"):
    """Run one mxgemm_ex call on copies of (A, B, C); return C as numpy."""
    import torch
    from paper_1901_06015_gb300 import mxgemm_ex
    dA, dB, dC = to_device(A), to_device(B), to_device(C)
    mxgemm_ex(None, method, transa, transb, alpha, dA, dB, beta, dC, comp=combo[3])
    torch.cuda.synchronize()
    return from_device(dC, combo[0])


def methods_for(combo, k=None):
    """Methods of combo's computation precision; with k given, only those the planner
    accepts at that k (the split-precision methods have a smallest k)."""
    from tests._helpers import comp_prec, SPLIT_MIN_K
    x = comp_prec(combo)
    if x in ("h", "b"):
        return ["tc16"]
    if x == "d":
        return ["dmma", "dfma"]
    return [m for m in ("ffma", "tf32x3", "bf16x3") if k is None or k >= SPLIT_MIN_K.get(m, 0)]
