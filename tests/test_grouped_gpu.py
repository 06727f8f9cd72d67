"""Grouped persistent launch (GPU): many problems of mixed datatype combinations and
uneven shapes in one grouped pack launch + one persistent contraction launch per
computation precision, optionally autotuned and captured in a CUDA graph. Each result
must equal the same problem run alone (bit for bit, same method family) and the oracle
within tolerance."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import to_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems(seed, count, lo=1, hi=300, trans=True):
    rng = np.random.default_rng(seed)
    combos = synth.all_combos()
    out = []
    for i in range(count):
        combo = combos[int(rng.integers(len(combos)))]
        m, n, k = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
        ta = "ntch"[int(rng.integers(4))] if trans else "n"
        tb = "ntch"[int(rng.integers(4))] if trans else "n"
        A, B, C = synth.problem(int(rng.integers(1 << 30)), combo, m, n, k, transa=ta, transb=tb,
                                order_c="FC"[int(rng.integers(2))])
        alpha = complex(1.25, -0.5) if all(c in "cz" for c in combo[:3]) else 1.5
        out.append(dict(combo=combo, ta=ta, tb=tb, alpha=alpha, beta=-0.5, A=A, B=B, C=C))
    return out


def _device_items(probs):
    items, dev = [], []
    for p in probs:
        dA, dB, dC = to_device(p["A"]), to_device(p["B"]), to_device(p["C"])
        dev.append((dA, dB, dC))
        items.append((p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, p["combo"][3]))
    return items, dev


def _solo(p, method_s="ffma", method_d="dmma"):
    import paper_1901_06015_gb300 as mx
    dA, dB, dC = to_device(p["A"]), to_device(p["B"]), to_device(p["C"])
    from tests._helpers import comp_prec
    meth = method_s if comp_prec(p["combo"]) == "s" else method_d
    mx.mxgemm_ex(None, meth, p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, comp=p["combo"][3])
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("tune,graph", [(False, False), (True, True)])
def test_grouped_equals_solo_and_oracle(tune, graph):
    import paper_1901_06015_gb300 as mx
    probs = _problems(1, 96)
    items, dev = _device_items(probs)
    g = mx.Group(items, method_d="dmma", tune=tune, graph=graph)
    g.run()
    torch.cuda.synchronize()
    desc = g.describe()
    assert desc["graph"] == graph
    for p, (_, _, dC) in zip(probs, dev):
        got = dC.cpu().numpy()
        assert np.array_equal(got, _solo(p)), p["combo"]
        ref_C = np.array(p["C"], order="K")
        ref = oracle_mxgemm(p["ta"], p["tb"], p["alpha"], p["A"], p["B"], p["beta"], ref_C, comp=p["combo"][3])
        k = p["A"].shape[0] if p["ta"] in "th" else p["A"].shape[1]
        err, _ = normwise_error(p["combo"], got, ref, p["A"], p["B"], p["C"], p["alpha"], p["beta"], p["ta"], p["tb"])
        assert err <= tolerance(p["combo"], k), (p["combo"], err)
    g.close()


def test_grouped_auto_double_kernel_within_tolerance_and_replay():
    """method_d = auto (DFMA kernels, tile chosen by the tuner); two graph replays equal
    two solo applications (beta != 0, so each run changes C)."""
    import paper_1901_06015_gb300 as mx
    probs = _problems(2, 64, trans=False)
    items, dev = _device_items(probs)
    g = mx.Group(items, tune=True, graph=True)
    g.run()
    g.run()
    torch.cuda.synchronize()
    for p, (_, _, dC) in zip(probs, dev):
        once = dict(p)
        ref_C = np.array(p["C"], order="K")
        oracle_mxgemm("n", "n", p["alpha"], p["A"], p["B"], p["beta"], ref_C, comp=p["combo"][3])
        C1 = ref_C.copy()
        ref2 = oracle_mxgemm("n", "n", p["alpha"], p["A"], p["B"], p["beta"], ref_C, comp=p["combo"][3])
        got = dC.cpu().numpy()
        err, _ = normwise_error(p["combo"], got, ref2, p["A"], p["B"], C1, p["alpha"], p["beta"])
        assert err <= 2 * tolerance(p["combo"], p["A"].shape[1]), (p["combo"], err)
    g.close()


def test_grouped_scale_and_noop_problems():
    import paper_1901_06015_gb300 as mx
    probs = _problems(3, 8, trans=False)
    # k == 0 (scale only) and m == 0 (nothing) entries
    A0 = np.zeros((5, 0), dtype=np.complex128); B0 = np.zeros((0, 4), dtype=np.float32)
    C0 = synth.matrix(np.random.default_rng(0), 5, 4, "z")
    probs.append(dict(combo="zdsd", ta="n", tb="n", alpha=1.0, beta=-0.5, A=A0, B=B0, C=C0))
    items, dev = _device_items(probs)
    Cm = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    items.append(("n", "n", 1.0, torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                  torch.zeros((2, 3), dtype=torch.float64, device="cuda"), 1.0, Cm, "d"))
    g = mx.Group(items, tune=False, graph=True)
    g.run()
    torch.cuda.synchronize()
    assert np.array_equal(dev[-1][2].cpu().numpy(), (-0.5 * C0).astype(C0.dtype))
    for p, (_, _, dC) in list(zip(probs, dev))[:-1]:
        assert np.array_equal(dC.cpu().numpy(), _solo(p))
    g.close()


def test_grouped_reports_first_invalid_problem():
    import paper_1901_06015_gb300 as mx
    probs = _problems(4, 5, trans=False)
    items, _ = _device_items(probs)
    # problem 3: case 1b (C, A real; B complex) with a complex alpha -> status 2
    A = torch.zeros((4, 3), dtype=torch.float32, device="cuda").t().contiguous().t()
    B = torch.zeros((3, 2), dtype=torch.complex64, device="cuda").t().contiguous().t()
    C = torch.zeros((4, 2), dtype=torch.float32, device="cuda").t().contiguous().t()
    items[3] = ("n", "n", 1.0 + 1.0j, A, B, 0.0, C, "s")
    with pytest.raises(mx.MxgError) as e:
        mx.Group(items, tune=False, graph=False)
    assert e.value.status == 2 and "problem 3" in str(e.value)


def test_one_shot_grouped_call():
    import paper_1901_06015_gb300 as mx
    probs = _problems(5, 16, trans=False)
    items, dev = _device_items(probs)
    mx.mxgemm_grouped(items)
    torch.cuda.synchronize()
    for p, (_, _, dC) in zip(probs, dev):
        ref_C = np.array(p["C"], order="K")
        ref = oracle_mxgemm("n", "n", p["alpha"], p["A"], p["B"], p["beta"], ref_C, comp=p["combo"][3])
        err, _ = normwise_error(p["combo"], dC.cpu().numpy(), ref, p["A"], p["B"], p["C"], p["alpha"], p["beta"])
        assert err <= tolerance(p["combo"], p["A"].shape[1])


@pytest.mark.parametrize("method_d,variant,solo_d", [
    ("dmma", 4, "dmma"),   # DMMA 64 x 64
    ("dfma", 2, "dfma"),   # DFMA 64 x 64
    ("dfma", 3, "dfma"),   # DFMA 32 x 32 (adjacent row pairs per thread)
    ("dfma", 6, "dfma"),   # DFMA 16 x 16 (64-thread CTAs)
])
@pytest.mark.parametrize("variant_s", [0, 1, 5])   # FFMA 128, 64, 32
def test_every_grouped_kernel_equals_solo(tmp_path, method_d, variant, solo_d, variant_s):
    """Each contraction kernel of the grouped launch, forced through a loaded tuning
    file, gives every problem bit for bit the result of the same problem run alone with
    the same method family (each element is accumulated by one thread in increasing k,
    whatever the tile). Shapes, transposes and storage orders are mixed, so ragged
    edges, complex row/column pairs and every output mode occur."""
    import paper_1901_06015_gb300 as mx
    probs = _problems(11, 48, lo=1, hi=140)
    items, _ = _device_items(probs)
    probe = mx.Group(items, method_d=method_d, tune=False, graph=False)
    sigs = {b["precision"]: b["signature"] for b in probe.describe()["buckets"]}
    probe.close()
    path = tmp_path / "tune.txt"
    path.write_text("".join(f"{sigs[p]} {v} 0 1.0\n" for p, v in (("s", variant_s), ("d", variant)) if p in sigs))
    assert mx.mxg_tune_load(str(path)) == 0
    items, dev = _device_items(probs)
    g = mx.Group(items, method_d=method_d, tune=False, graph=True)
    kernels = {b["precision"]: b["kernel"] for b in g.describe()["buckets"]}
    names = {0: "ffma_128", 1: "ffma_64", 5: "ffma_32", 2: "dfma_64", 3: "dfma_32", 4: "dmma_64", 6: "dfma_16"}
    assert kernels.get("s", names[variant_s]) == names[variant_s]
    assert kernels.get("d", names[variant]) == names[variant]
    g.run()
    torch.cuda.synchronize()
    for p, (_, _, dC) in zip(probs, dev):
        assert np.array_equal(dC.cpu().numpy(), _solo(p, method_d=solo_d)), (p["combo"], p["ta"], p["tb"])
    g.close()


def test_grouped_batching_configuration_sampled_blocks():
    """The batching configuration at its full size, in the launch configuration the
    benchmark times: 2048 problems, m, n, k = round(exp(U(ln 16, ln 1024))), combination
    uniform over the 128, entries U[-1, 1], alpha = 1.5, beta = -0.5, one autotuned,
    graph-captured grouped launch. Every problem is checked against the oracle on a
    block of up to 16 x 16 entries of C at seeded rows and columns (the block obeys
    C_blk := alpha A(rows, :) B(:, cols) + beta C_blk, so the bound uses its own norms)."""
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    rng = np.random.default_rng(0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    combos = synth.all_combos()
    items, metas = [], []
    for _ in range(2048):
        combo = combos[int(rng.integers(len(combos)))]
        m, n, k = (int(round(float(np.exp(rng.uniform(np.log(16), np.log(1024)))))) for _ in range(3))
        A = synth.torch_matrix(gen, m, k, combo[1], "cuda")
        B = synth.torch_matrix(gen, k, n, combo[2], "cuda")
        C = synth.torch_matrix(gen, m, n, combo[0], "cuda")
        items.append(("n", "n", 1.5, A, B, -0.5, C, combo[3]))
        rows = torch.as_tensor(np.sort(rng.choice(m, size=min(m, 16), replace=False)), device="cuda")
        cols = torch.as_tensor(np.sort(rng.choice(n, size=min(n, 16), replace=False)), device="cuda")
        metas.append((combo, k, rows, cols, C[rows][:, cols].cpu().numpy()))
    g = mx.Group(items, tune=True, graph=True)
    g.run()
    torch.cuda.synchronize()
    assert {b["precision"] for b in g.describe()["buckets"]} == {"s", "d"}
    for (_, _, _, A, B, _, C, _), (combo, k, rows, cols, C0) in zip(items, metas):
        Ab = A[rows].cpu().numpy()
        Bb = B[:, cols].cpu().numpy()
        got = C[rows][:, cols].cpu().numpy()
        ref = oracle_mxgemm("n", "n", 1.5, Ab, Bb, -0.5, np.array(C0, order="F"), comp=combo[3])
        err, _ = normwise_error(combo, got, ref, Ab, Bb, C0, 1.5, -0.5)
        assert err <= tolerance(combo, k), (combo, k, err)
    g.close()


def _solo16(p, meth):
    """p run alone through mxgemm_ex with method meth and whole tiles (the grouped
    launch has no stream-K tail); C as numpy (16-bit aware)."""
    import paper_1901_06015_gb300 as mx
    from tests.gpu_util import from_device
    dA, dB, dC = to_device(p["A"]), to_device(p["B"]), to_device(p["C"])
    h = mx.Handle()
    h.set_stream(torch.cuda.current_stream())
    h.set_stream_k(0)
    mx.mxgemm_ex(h, meth, p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, comp=p["combo"][3])
    torch.cuda.synchronize()
    h.close()
    return from_device(dC, p["combo"][0])


@pytest.mark.parametrize("method_s", ["bf16x3", "tf32x3"])
def test_grouped_tensor_core_buckets(method_s):
    """Tensor-core buckets of a grouped launch: single-precision problems on the split
    method (those below its smallest k fall back to the FFMA bucket), the 16-bit
    computation precisions on TC16, next to the plain buckets, graph-captured and timed.
    Every result equals the same problem run alone with its method bit for bit and is
    within the stated bound of the oracle."""
    import paper_1901_06015_gb300 as mx
    from tests.gpu_util import from_device
    from tests._helpers import SPLIT_MIN_K, comp_prec
    rng = np.random.default_rng(5)
    combos = ["ssss", "cscs", "zcds", "dsss", "zzzs", "czcs", "hhhh", "kkkh", "bbbb", "wbwb", "shhh", "zbbb",
              "dddd", "zzzd", "ccsd"]
    probs = []
    for i in range(45):
        combo = combos[i % len(combos)]
        m, n = (int(x) for x in rng.integers(20, 300, size=2))
        k = int(rng.choice([40, 200, 330, 700]))
        ta, tb = "ntch"[i % 4], "nt"[i % 2]
        A, B, C = synth.problem(700 + i, combo, m, n, k, transa=ta, transb=tb, order_c="FC"[i % 2])
        alpha = complex(1.25, -0.5) if all(synth.is_complex(c) for c in combo[:3]) else 1.5
        beta = (0.5 - 0.25j) if synth.is_complex(combo[0]) else -0.5
        probs.append(dict(combo=combo, ta=ta, tb=tb, alpha=alpha, beta=beta, A=A, B=B, C=C, k=k))
    dev = [(to_device(p["A"]), to_device(p["B"]), to_device(p["C"])) for p in probs]
    items = [(p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, p["combo"][3]) for p, (dA, dB, dC) in zip(probs, dev)]
    g = mx.Group(items, method_s=method_s, tune=True, graph=True)
    g.run()
    torch.cuda.synchronize()
    kernels = {b["kernel"] for b in g.describe()["buckets"]}
    assert {"tc16_f16", "tc16_bf16", "tc_" + method_s} <= kernels, kernels
    h = mx.Handle()
    h.set_stream(torch.cuda.current_stream())
    assert h.check_device_error() == 0
    for p, (_, _, dC) in zip(probs, dev):
        x = comp_prec(p["combo"])
        meth = "tc16" if x in "hb" else ("dfma" if x == "d" else (method_s if p["k"] >= SPLIT_MIN_K[method_s] else "ffma"))
        got = from_device(dC, p["combo"][0])
        assert np.array_equal(synth.to_c128(got), synth.to_c128(_solo16(p, meth))), (p["combo"], meth)
        ref = oracle_mxgemm(p["ta"], p["tb"], p["alpha"], p["A"], p["B"], p["beta"], np.array(p["C"], order="K"),
                            comp=p["combo"][3])
        err, _ = normwise_error(p["combo"], got, ref, p["A"], p["B"], p["C"], p["alpha"], p["beta"], p["ta"], p["tb"])
        assert err <= tolerance(p["combo"], p["k"], meth, p["beta"]), (p["combo"], meth, err)
    g.close()
    h.close()
