"""Tensor-core contraction on CTA pairs (tcgen05 cta_group::2; GPU). The pair kernel
(256 x 256 tiles over two SMs) and the single-CTA kernel (128 x 256 tiles) compute the
same products in the same order along k, so with the stream-K tail off their results
agree bit for bit; both are within the stated bound of the oracle. Shapes cover an odd
number of 128-row tiles (the last pair's second half lies past the packed operand),
ragged edges, every output mode, the one-pass 16-bit form and the split forms.

The stream-K tail (tiles of a partial last wave cut along k over every pair, partial
sums added in increasing k by the range that finishes a tile last) is forced on small
shapes with several ranges per tile, ragged edges and whole tiles before the tail: it
must stay within the stated bound of the oracle, repeat bit for bit, and differ from the
whole-tile run (so the tail really ran)."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import from_device, to_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # combo, (m, n, k), method
    ("hhhh", (300, 260, 96), "tc16"),        # Mp = 384: three 128-row tiles, odd
    ("bbbb", (128, 256, 32), "tc16"),        # one pair, half of it past Mp
    ("kkkh", (140, 270, 96), "tc16"),        # case 3, row pairs
    ("wbwb", (257, 513, 160), "tc16"),       # case 2bc, column pairs
    ("zbbb", (90, 130, 200), "tc16"),        # case 1c, Re(C) only
    ("shhh", (520, 700, 64), "tc16"),
    ("ssss", (300, 260, 320), "bf16x3"),
    ("zcds", (129, 300, 64), "tf32x3"),
    ("cscs", (150, 260, 330), "bf16x3"),
]


def _run(h, combo, method, A, B, C0, alpha, beta):
    import paper_1901_06015_gb300 as mx
    dA, dB, dC = to_device(A), to_device(B), to_device(C0)
    mx.mxgemm_ex(h, method, "n", "n", alpha, dA, dB, beta, dC, comp=combo[3])
    torch.cuda.synchronize()
    return from_device(dC, combo[0])


@pytest.mark.parametrize("combo,shape,method", CASES)
def test_pairs_equal_single_cta_and_oracle(combo, shape, method):
    import paper_1901_06015_gb300 as mx
    m, n, k = shape
    A, B, C0 = synth.problem(41, combo, m, n, k)
    alpha = (1.25 - 0.5j) if all(synth.is_complex(t) for t in combo[:3]) else 1.5
    beta = (-0.5 + 0.25j) if synth.is_complex(combo[0]) else -0.5
    hp, hs = mx.Handle(), mx.Handle()
    for h, mode in ((hp, 1), (hs, 2)):
        h.set_stream(torch.cuda.current_stream())
        h.set_cta_pairs(mode)
        h.set_stream_k(0)
    got_p = _run(hp, combo, method, A, B, C0, alpha, beta)
    got_s = _run(hs, combo, method, A, B, C0, alpha, beta)
    assert hp.check_device_error() == 0 and hs.check_device_error() == 0
    assert np.array_equal(synth.to_c128(got_p), synth.to_c128(got_s)), (combo, method)
    ref = oracle_mxgemm("n", "n", alpha, A, B, beta, C0.copy(), comp=combo[3])
    err, _ = normwise_error(combo, got_p, ref, A, B, C0, alpha, beta)
    assert err <= tolerance(combo, k, method, beta), (combo, method, err)
    hp.close(); hs.close()


@pytest.mark.parametrize("combo,method", [("ssss", "bf16x3"), ("hhhh", "tc16"), ("zcds", "tf32x3")])
def test_pairs_wide_tiles_equal_single_cta(combo, method):
    """A problem with enough 256 x 256 pair tiles to fill the device (128 pair tiles on
    76 pairs of SMs, two waves): bit-equal to the single-CTA kernel, and the first 64 x 64
    block within the bound of the oracle."""
    import paper_1901_06015_gb300 as mx
    m, n, k = 2048, 4096, 320
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    A = synth.torch_matrix(gen, m, k, combo[1], "cuda")
    B = synth.torch_matrix(gen, k, n, combo[2], "cuda")
    C0 = synth.torch_matrix(gen, m, n, combo[0], "cuda")
    outs = []
    for mode in (1, 2):
        h = mx.Handle()
        h.set_stream(torch.cuda.current_stream())
        h.set_cta_pairs(mode)
        h.set_stream_k(0)
        C = C0.clone()
        mx.mxgemm_ex(h, method, "n", "n", 1.0, A, B, 1.0, C, comp=combo[3])
        torch.cuda.synchronize()
        assert h.check_device_error() == 0
        outs.append(C)
        h.close()
    assert torch.equal(outs[0], outs[1])
    Ab = from_device(A[:64, :], combo[1])
    Bb = from_device(B[:, :64], combo[2])
    Cb = from_device(C0[:64, :64], combo[0])
    ref = oracle_mxgemm("n", "n", 1.0, np.asfortranarray(Ab), np.asfortranarray(Bb), 1.0,
                        np.asfortranarray(Cb.copy()), comp=combo[3])
    err, _ = normwise_error(combo, from_device(outs[0][:64, :64], combo[0]), ref, Ab, Bb, Cb, 1.0, 1.0)
    assert err <= tolerance(combo, k, method), (combo, err)


SK_CASES = [
    # combo, (m, n, k), method: pair tiles T, k-blocks per tile (all tiles in the tail)
    ("hhhh", (1280, 768, 1024), "tc16"),     # T = 15, 16 k-blocks: ~5 ranges per tile
    ("kkkh", (300, 520, 700), "tc16"),       # case 3, row pairs, ragged: T = 9, 22 k-blocks
    ("wbwb", (390, 700, 600), "tc16"),       # case 2bc, column pairs: T = 12, 10 k-blocks
    ("ssss", (700, 900, 640), "bf16x3"),     # T = 12, 10 k-blocks
    ("zcds", (300, 300, 512), "tf32x3"),     # case 2ac: T = 6, 16 k-blocks of 32
]


def _sk_runs(combo, method, A, B, C0, alpha, beta):
    import paper_1901_06015_gb300 as mx
    outs = []
    for mode in (2, 2, 0):
        h = mx.Handle()
        h.set_stream(torch.cuda.current_stream())
        h.set_stream_k(mode)
        outs.append(_run(h, combo, method, A, B, C0, alpha, beta))
        assert h.check_device_error() == 0
        h.close()
    return outs


@pytest.mark.parametrize("combo,shape,method", SK_CASES)
def test_stream_k_tail_within_bound_and_repeatable(combo, shape, method):
    m, n, k = shape
    A, B, C0 = synth.problem(43, combo, m, n, k)
    alpha = (1.25 - 0.5j) if all(synth.is_complex(t) for t in combo[:3]) else 1.5
    beta = (-0.5 + 0.25j) if synth.is_complex(combo[0]) else -0.5
    sk1, sk2, whole = _sk_runs(combo, method, A, B, C0, alpha, beta)
    assert np.array_equal(synth.to_c128(sk1), synth.to_c128(sk2)), combo
    assert not np.array_equal(synth.to_c128(sk1), synth.to_c128(whole)), combo
    ref = oracle_mxgemm("n", "n", alpha, A, B, beta, C0.copy(), comp=combo[3])
    for got in (sk1, whole):
        err, _ = normwise_error(combo, got, ref, A, B, C0, alpha, beta)
        assert err <= tolerance(combo, k, method, beta), (combo, method, err)


def test_stream_k_tail_after_whole_tiles():
    """81 pair tiles on 76 pairs: one wave of whole tiles per pair after its range of the
    5-tile tail (16 k-blocks each: 80 steps over 76 pairs). Every block of C sampled
    along the diagonal and in the tail's corner is within the bound of the oracle."""
    import paper_1901_06015_gb300 as mx
    combo, method = "hhhh", "tc16"
    m = n = 2304
    k = 1024
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    A = synth.torch_matrix(gen, m, k, combo[1], "cuda")
    B = synth.torch_matrix(gen, k, n, combo[2], "cuda")
    C0 = synth.torch_matrix(gen, m, n, combo[0], "cuda")
    outs = []
    for mode in (2, 2, 0):
        h = mx.Handle()
        h.set_stream(torch.cuda.current_stream())
        h.set_stream_k(mode)
        C = C0.clone()
        mx.mxgemm_ex(h, method, "n", "n", 1.0, A, B, 1.0, C, comp=combo[3])
        torch.cuda.synchronize()
        assert h.check_device_error() == 0
        outs.append(C)
        h.close()
    assert torch.equal(outs[0], outs[1])
    assert not torch.equal(outs[0], outs[2])
    for r0, c0 in ((0, 0), (1024, 1024), (2240, 2240), (2240, 1792), (1792, 2240)):
        Ab = from_device(A[r0:r0 + 64, :], combo[1])
        Bb = from_device(B[:, c0:c0 + 64], combo[2])
        Cb = from_device(C0[r0:r0 + 64, c0:c0 + 64], combo[0])
        ref = oracle_mxgemm("n", "n", 1.0, np.asfortranarray(Ab), np.asfortranarray(Bb), 1.0,
                            np.asfortranarray(Cb.copy()), comp=combo[3])
        got = from_device(outs[0][r0:r0 + 64, c0:c0 + 64], combo[0])
        err, _ = normwise_error(combo, got, ref, Ab, Bb, Cb, 1.0, 1.0)
        assert err <= tolerance(combo, k, method), (r0, c0, err)


PF_CASES = [
    # combo, (m, n, k), method: C types s, c (row and column pairs), z (16-byte elements), d
    ("shhh", (300, 520, 96), "tc16"),
    ("ckkh", (140, 270, 96), "tc16"),
    ("zkkh", (150, 260, 64), "tc16"),
    ("zbbb", (90, 130, 200), "tc16"),        # case 1c: Re(C) only
    ("dhhh", (260, 300, 128), "tc16"),
    ("cscs", (150, 260, 330), "bf16x3"),
    ("ssss", (300, 600, 320), "bf16x3"),
]


@pytest.mark.parametrize("combo,shape,method", PF_CASES)
def test_c_prefetch_equals_direct_loads(combo, shape, method):
    """The pair kernel takes old C from its TMA prefetch ring when C has unit row stride
    and reads it straight from global memory otherwise. The same C stored both ways
    (column-major, and every other row of a larger buffer) gives the same result bit for
    bit, ragged edges and every output mode included, within the bound of the oracle."""
    from tests.gpu_util import run
    m, n, k = shape
    A, B, C0 = synth.problem(47, combo, m, n, k)
    alpha = (1.25 - 0.5j) if all(synth.is_complex(t) for t in combo[:3]) else 1.5
    beta = (-0.5 + 0.25j) if synth.is_complex(combo[0]) else -0.5
    big = np.zeros((2 * m + 1, n), dtype=C0.dtype, order="F")
    Cg = big[::2, :][:m, :]
    Cg[...] = C0
    assert Cg.strides[0] != Cg.itemsize           # no unit row stride: direct loads
    got_col = run(combo, A, B, np.asfortranarray(C0), alpha, beta, method=method)
    got_gen = run(combo, A, B, Cg, alpha, beta, method=method)
    assert np.array_equal(synth.to_c128(got_col), synth.to_c128(got_gen)), combo
    ref = oracle_mxgemm("n", "n", alpha, A, B, beta, C0.copy(), comp=combo[3])
    err, _ = normwise_error(combo, got_col, ref, A, B, C0, alpha, beta)
    assert err <= tolerance(combo, k, method, beta), (combo, method, err)
