"""Parity at the full benchmark size (GPU): m = n = k = 8192, column-major, no
transpose, U[-1, 1], alpha = beta = 1, in the launch configuration the benchmark times
(FFMA for single, DMMA for double), for all 128 combinations. The oracle checks 4 sampled 64 x 64 blocks of C (two corners and two
seeded positions); a block obeys C_blk := alpha A(rows, :) B(:, cols) + beta C_blk, so
the bound uses the block's own operand norms."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from tests._helpers import normwise_error, tolerance
from tests.test_parity_gpu import ALL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 8192
BS = 64


@pytest.mark.parametrize("combo", ALL)
def test_full_size_sampled_blocks(combo):
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    gen = torch.Generator(device="cuda")
    gen.manual_seed(99)
    A = synth.torch_matrix(gen, N, N, combo[1], "cuda")
    B = synth.torch_matrix(gen, N, N, combo[2], "cuda")
    C = synth.torch_matrix(gen, N, N, combo[0], "cuda")
    rng = np.random.default_rng(5)
    pos = [(0, 0), (N - BS, N - BS)] + [tuple(int(v) for v in rng.integers(0, N - BS, size=2)) for _ in range(2)]
    before = [C[i:i + BS, j:j + BS].cpu().numpy() for i, j in pos]
    meth = "ffma" if combo[3] == "s" else "dmma"
    mx.mxgemm_ex(None, meth, "n", "n", 1.0, A, B, 1.0, C, comp=combo[3])
    torch.cuda.synchronize()
    for (i, j), C0 in zip(pos, before):
        Ap = np.asfortranarray(A[i:i + BS, :].cpu().numpy())
        Bp = np.asfortranarray(B[:, j:j + BS].cpu().numpy())
        ref_C = np.asfortranarray(C0.copy())
        ref = oracle_mxgemm("n", "n", 1.0, Ap, Bp, 1.0, ref_C, comp=combo[3])
        got = C[i:i + BS, j:j + BS].cpu().numpy()
        err, _ = normwise_error(combo, got, ref, Ap, Bp, C0, 1.0, 1.0)
        assert err <= tolerance(combo, N), (combo, (i, j), err)
    del A, B, C
    torch.cuda.empty_cache()
