"""The no-allocation entry point (GPU).

mxgemm_noalloc serves callers that cannot call cudaMalloc -- work enqueued inside a
CUDA graph capture, latency-critical loops that cannot take cudaMalloc/cudaFree's
implicit synchronisation, applications whose device memory belongs to another
allocator. It packs into a fixed device array instead of an allocated workspace.
This file is collected last so that a stop-at-first-failure run has already run every
other test; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import to_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(combo, m, n, k, alpha, beta, method, seed):
    """Run the same problem through mxgemm_ex and mxgemm_noalloc (C ABI)."""
    import paper_1901_06015_gb300 as mx
    A, B, C0 = synth.problem(seed, combo, m, n, k)
    dA, dB = to_device(A), to_device(B)
    ref, got = to_device(C0), to_device(C0)
    mx.mxgemm_ex(None, method, "n", "n", alpha, dA, dB, beta, ref, comp=combo[3])
    mx.mxgemm_noalloc(method, "n", "n", alpha, dA, dB, beta, got, comp=combo[3])
    torch.cuda.synchronize()
    return A, B, C0, ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_existing_entry_point_twice_in_a_row():
    # two different calls back to back: the second runs on scratch the first left behind
    for combo, (m, n, k), alpha, method, seed in [
        ("zzzd", (200, 180, 150), 1.25 - 0.5j, "dmma", 21),
        ("scds", (100, 90, 70), 1.5, "ffma", 22),
    ]:
        A, B, C0, ref, got = _pair(combo, m, n, k, alpha, -0.5, method, seed)
        err, _ = normwise_error(combo, got, ref.astype(np.complex128), A, B, C0, alpha, -0.5)
        assert err <= tolerance(combo, k), (combo, err)


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
