"""16-bit storage and computation precisions (Sec. 5.3) on the GPU: binary16 and
bfloat16 storage (real and complex) for any of A, B, C, and computation precision h / b
(A and B rounded to binary16 / bfloat16, products summed in FP32 on the tensor cores,
method TC16), against the oracle."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import run, methods_for, to_device, from_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL_16 = synth.all_combos_16()   # the 1920 combinations with a 16-bit storage or precision


@pytest.mark.parametrize("combo", ALL_16)
def test_16bit_parity(combo):
    m, n, k = 67, 45, 130
    A, B, C0 = synth.problem(23, combo, m, n, k, order_c="FC"[len(combo) % 2])
    case_cplx3 = all(synth.is_complex(t) for t in combo[:3])
    alpha = (1.25 - 0.5j) if case_cplx3 else 1.5
    beta = (-0.5 + 0.25j) if synth.is_complex(combo[0]) else -0.5
    ref_C = C0.copy()
    ref = oracle_mxgemm("n", "n", alpha, A, B, beta, ref_C, comp=combo[3])
    for meth in methods_for(combo, k):
        got = run(combo, A, B, C0, alpha, beta, method=meth)
        err, _ = normwise_error(combo, got, ref, A, B, C0, alpha, beta)
        assert err <= tolerance(combo, k, meth, beta), (combo, meth, err, tolerance(combo, k, meth, beta))


@pytest.mark.parametrize("combo", ALL_16)
def test_16bit_small_integers_bit_exact(combo):
    """Integers in [-2, 2], k <= 16: every value is exact in binary16 and bfloat16, so
    the GPU result equals the oracle's rounded result bit for bit."""
    rng = np.random.default_rng(7)
    m, n, k = 40, 33, 16
    def mat(rows, cols, dt):
        re = rng.integers(-2, 3, size=(rows, cols)).astype(np.float64)
        im = rng.integers(-2, 3, size=(rows, cols)).astype(np.float64) if synth.is_complex(dt) else 0.0
        return synth.from_values(re + 1j * im, dt)
    A, B, C0 = mat(m, k, combo[1]), mat(k, n, combo[2]), mat(m, n, combo[0])
    for alpha, beta in ((1.0, 0.0), (-2.0, 1.0), (1.0, -0.5)):
        ref_C = C0.copy()
        oracle_mxgemm("n", "n", alpha, A, B, beta, ref_C, comp=combo[3])
        for meth in methods_for(combo, k):
            got = run(combo, A, B, C0, alpha, beta, method=meth)
            assert np.array_equal(synth.to_c128(got), synth.to_c128(ref_C)), (combo, meth, alpha, beta)


@pytest.mark.parametrize("combo", ["hhhh", "bbbb", "kkkh", "wbwb", "shhh", "zbbb", "ckhh"])
def test_16bit_sampled_blocks_4096(combo):
    """m = n = k = 4096 through the native tensor-core pass (TC16), two 64 x 64 blocks."""
    import paper_1901_06015_gb300 as mx
    N, BS = 4096, 64
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    A = synth.torch_matrix(gen, N, N, combo[1], "cuda")
    B = synth.torch_matrix(gen, N, N, combo[2], "cuda")
    C = synth.torch_matrix(gen, N, N, combo[0], "cuda")
    pos = [(0, 0), (N - BS, 1234)]
    before = [from_device(C[i:i + BS, j:j + BS], combo[0]) for i, j in pos]
    mx.mxgemm_ex(None, "auto", "n", "n", 1.0, A, B, 1.0, C, comp=combo[3])
    torch.cuda.synchronize()
    for (i, j), C0 in zip(pos, before):
        Ap = np.asfortranarray(from_device(A[i:i + BS, :], combo[1]))
        Bp = np.asfortranarray(from_device(B[:, j:j + BS], combo[2]))
        ref = oracle_mxgemm("n", "n", 1.0, Ap, Bp, 1.0, np.asfortranarray(C0.copy()), comp=combo[3])
        got = from_device(C[i:i + BS, j:j + BS], combo[0])
        err, _ = normwise_error(combo, got, ref, Ap, Bp, C0, 1.0, 1.0)
        assert err <= tolerance(combo, N, "tc16"), (combo, (i, j), err)


def test_16bit_storage_in_grouped_and_served_forms():
    """16-bit storage with single/double computation runs in a grouped launch; a 16-bit
    computation precision runs in the group's TC16 buckets and is served per call."""
    import paper_1901_06015_gb300 as mx
    combos = ["hsss", "sbbs", "kkcd", "wzwd", "hhhs", "bdbd"]
    probs = [synth.problem(40 + i, c, 50 + 7 * i, 40, 60) for i, c in enumerate(combos)]
    dev = [(to_device(A), to_device(B), to_device(C)) for (A, B, C) in probs]
    items = [("n", "n", 1.5, dA, dB, -0.5, dC, c[3]) for c, (dA, dB, dC) in zip(combos, dev)]
    g = mx.Group(items, tune=True, graph=True)
    g.run()
    torch.cuda.synchronize()
    for c, (A, B, C0), (_, _, dC) in zip(combos, probs, dev):
        ref = oracle_mxgemm("n", "n", 1.5, A, B, -0.5, C0.copy(), comp=c[3])
        err, _ = normwise_error(c, from_device(dC, c[0]), ref, A, B, C0, 1.5, -0.5)
        assert err <= tolerance(c, 60), (c, err)
    g.close()
    A, B, C0 = synth.problem(50, "hhhh", 30, 20, 40)
    dC = to_device(C0)
    g = mx.Group([("n", "n", 1.0, to_device(A), to_device(B), 0.0, dC, "h")], tune=False, graph=False)
    g.run()
    torch.cuda.synchronize()
    g.close()
    ref = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, C0.copy(), comp="h")
    err, _ = normwise_error("hhhh", from_device(dC, "h"), ref, A, B, C0, 1.0, 0.0)
    assert err <= tolerance("hhhh", 40, "tc16")
    srv = mx.Server(n_streams=2, hbm_budget_bytes=1 << 28)
    dA, dB, dC = to_device(A), to_device(B), to_device(C0)
    srv.submit(("n", "n", 1.0, dA, dB, 0.0, dC, "h"))
    srv.drain(30)
    assert srv.poll()[0]["status"] == 0
    srv.close()
    ref = oracle_mxgemm("n", "n", 1.0, A, B, 0.0, C0.copy(), comp="h")
    err, _ = normwise_error("hhhh", from_device(dC, "h"), ref, A, B, C0, 1.0, 0.0)
    assert err <= tolerance("hhhh", 40, "tc16")
