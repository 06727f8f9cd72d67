"""GPU-test utilities: move numpy inputs to the device keeping their layout, run the
library, bring C back."""
import numpy as np


def to_device(arr):
    """Device copy of a numpy 2-D array with the same strides (including general
    strides of a view into a larger buffer)."""
    import torch
    arr = np.asarray(arr)
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
    return dC.cpu().numpy()


def methods_for(combo):
    from tests._helpers import comp_prec
    return ["ffma", "tf32x3", "bf16x3"] if comp_prec(combo) == "s" else ["dmma", "dfma"]
