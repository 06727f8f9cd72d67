"""The no-allocation entry point (GPU).

mxgemm_noalloc serves callers that cannot call cudaMalloc: latency-critical loops that
cannot take cudaMalloc/cudaFree's implicit device synchronisation, and applications
whose device memory belongs to another allocator that forbids side allocations. It
packs into a fixed device array instead of an allocated workspace, and its tensor-core
kernels report a wait timeout through a fixed device error word.

This file is collected last so that a stop-at-first-failure run has already run every
other test; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import from_device, to_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (combo, (m, n, k), alpha, beta, method, seed): every contraction kernel family --
# DMMA, DFMA, FFMA, the tcgen05 split forms and the one-pass 16-bit form
CASES = [
    ("zzzd", (200, 180, 150), 1.25 - 0.5j, 0.5 + 0.25j, "dmma", 21),
    ("scds", (100, 90, 70), 1.5, -0.5, "ffma", 22),
    ("dzsd", (130, 70, 90), 2.0, 1.0, "dfma", 23),
    ("cscs", (150, 260, 330), 1.5, -0.5 + 0.5j, "bf16x3", 24),
    ("zcds", (129, 300, 64), -1.0, 0.75, "tf32x3", 25),
    ("kkhh", (140, 270, 96), 1.0, -0.5, "tc16", 26),
]


def _pair(combo, m, n, k, alpha, beta, method, seed):
    """Run the same problem through mxgemm_ex and mxgemm_noalloc (C ABI); return the
    inputs, the oracle's unrounded result and both device results."""
    import paper_1901_06015_gb300 as mx
    A, B, C0 = synth.problem(seed, combo, m, n, k)
    ref = oracle_mxgemm("n", "n", alpha, A, B, beta, C0.copy(order="F"), comp=combo[3])
    dA, dB = to_device(A), to_device(B)
    c_ex, c_na = to_device(C0), to_device(C0)
    mx.mxgemm_ex(None, method, "n", "n", alpha, dA, dB, beta, c_ex, comp=combo[3])
    mx.mxgemm_noalloc(method, "n", "n", alpha, dA, dB, beta, c_na, comp=combo[3])
    torch.cuda.synchronize()
    return A, B, C0, ref, from_device(c_ex, combo[0]), from_device(c_na, combo[0])


def test_noalloc_matches_existing_entry_point_and_oracle_twice_in_a_row():
    """Two rounds of calls back to back (the second runs on scratch the first left
    behind): the result equals mxgemm_ex's bit for bit (same kernels, same plan) and is
    within the stated bound of the oracle; the error word stays 0."""
    import paper_1901_06015_gb300 as mx
    for rnd in range(2):
        for combo, (m, n, k), alpha, beta, method, seed in CASES:
            A, B, C0, ref, got_ex, got_na = _pair(combo, m, n, k, alpha, beta, method, seed + 100 * rnd)
            assert np.array_equal(synth.to_c128(got_na), synth.to_c128(got_ex)), (combo, method, rnd)
            err, _ = normwise_error(combo, got_na, ref, A, B, C0, alpha, beta)
            assert err <= tolerance(combo, k, method, beta), (combo, method, rnd, err)
        assert mx.mxgemm_noalloc_check_device_error() == 0


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    import paper_1901_06015_gb300 as mx
    lim = 32 << 20
    n = 2048   # zzz at 2048^3: packed A' alone is 2n x 2n doubles = 128 MiB
    assert mx.mxg_plan("zzzd", n, n, n).workspace_bytes > lim
    A = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    B = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    C = torch.ones((n, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(mx.MxgError) as e:
        mx.mxgemm_noalloc("auto", "n", "n", 1.0, A.t(), B.t(), 0.0, C.t(), comp="d")
    assert e.value.status == 7
    torch.cuda.synchronize()
    assert bool((C == 1).all())
