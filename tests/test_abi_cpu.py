"""CPU-only checks of the C ABI library: it builds, loads, exports every function the
header declares, and its host-side planner classifies and sizes calls as the paper's
case table says (no CUDA call is made)."""
import json
import os
import re

import pytest

import paper_1901_06015_gb300 as mx
from paper_1901_06015_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                                txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = mx.lib()
    names = _declared_functions()
    assert "mxgemm" in names and "mxg_plan" in names
    for n in names:
        assert hasattr(L, n), n
    assert L.mxg_version() >= 10000


def test_strerror_codes():
    for st in range(9):
        assert mx.mxg_strerror(st) and "unknown" not in mx.mxg_strerror(st)


def test_case_table_and_real_products_match_figure():
    g = json.load(open(os.path.join(GOLDEN, "mixeddom.json")))
    for row in g["cases"]:
        dc = "z" if row["C"] == "C" else "d"
        da = "z" if row["A"] == "C" else "d"
        db = "z" if row["B"] == "C" else "d"
        for x in "sd":
            info = mx.mxg_plan(dc + da + db + x, 64, 48, 32)
            assert mx.CASE_NAMES[info.domain_case] == row["case"]
            assert 2 * info.real_products == row["flops_per_mnk"]
            assert info.flops == row["flops_per_mnk"] * 64 * 48 * 32
            assert info.Mr * info.Nr * info.Kr == info.real_products * 64 * 48 * 32
            assert info.comp_prec == (0 if x == "s" else 1)


def test_comp_precision_defaults_to_C():
    assert mx.mxg_plan("sddc", 8, 8, 8).comp_prec == 0
    assert mx.mxg_plan("zccc", 8, 8, 8).comp_prec == 1


@pytest.mark.parametrize("combo", synth.all_combos())
def test_every_combo_plans(combo):
    info = mx.mxg_plan(combo, 100, 90, 80)
    assert info.workspace_bytes > 0
    assert info.method in (1, 5)   # AUTO: FFMA for single, DFMA for double


def test_stream_k_tail_workspace_follows_the_automatic_rule():
    """The CTA-pair kernel's stream-K tail: the plan reserves its workspace (76 pairs of
    a 152-SM device x 512 KB of FP32 partial slots, plus 76 x 8 tile counters rounded
    to 256 bytes) exactly when the automatic rule would run it: the pairs idle in the
    partial last wave are at least 6% of the run, and each pair's range holds at least
    16 k-blocks (64 elements of a 16-bit format each)."""
    sk = 76 * 512 * 1024 + 2560

    def ws(combo, m, n, k, method):
        return mx.mxg_plan(combo, m, n, k, method=method).workspace_bytes

    def planes(m, n, k, count):                       # 2-byte planes: count per operand
        return count * 2 * (m * k + n * k)

    # BF16x3 4096^3: 256 pair tiles, last wave 28 of 76 (48 idle over 4 waves: 16%) -> tail
    assert ws("ssss", 4096, 4096, 4096, "bf16x3") == planes(4096, 4096, 4096, 2) + sk
    # TC16 2048^3: 64 tiles, one partial wave (16% idle), 64 x 32 k-blocks -> tail
    assert ws("hhhh", 2048, 2048, 2048, "tc16") == planes(2048, 2048, 2048, 1) + sk
    # TC16 8192^3: 40 idle pairs over 14 waves (4%) -> none
    assert ws("hhhh", 8192, 8192, 8192, "tc16") == planes(8192, 8192, 8192, 1)
    # 2048 x 2048 x 512: 64 x 8 k-blocks, fewer than 16 per pair -> none
    assert ws("hhhh", 2048, 2048, 512, "tc16") == planes(2048, 2048, 512, 1)
    # 152 tiles fill two waves exactly -> none
    assert ws("hhhh", 256 * 8, 256 * 19, 4096, "tc16") == planes(2048, 4864, 4096, 1)


def test_whole_op_transpose_for_row_major_C():
    info = mx.mxg_plan("zzsd", 50, 40, 30, strides=((1, 50), (1, 30), (40, 1)))
    assert info.whole_op_transposed == 1
    assert mx.CASE_NAMES[info.domain_case] == "2ac"   # reported for the call as given
    assert (info.Mr, info.Nr, info.Kr) == (40, 100, 30)  # computed as 2bc on C^T
    info = mx.mxg_plan("zzsd", 50, 40, 30)
    assert info.whole_op_transposed == 0 and (info.Mr, info.Nr, info.Kr) == (100, 40, 30)


@pytest.mark.parametrize("bad", [
    dict(m=-1), dict(transa="x"), dict(strides=((0, 5), (1, 5), (1, 5))),
    dict(strides=((1, 5), (1, 5), (1, 1))),        # C overlaps itself
    dict(method="ffma", comp="d"), dict(method="dmma", comp="s"),
])
def test_invalid_arguments(bad):
    kw = dict(m=5, n=5, k=5, transa="n", transb="n", method="auto", strides=None, comp=None)
    kw.update(bad)
    with pytest.raises((mx.MxgError, KeyError)) as e:
        mx.mxg_plan("dddd", kw["m"], kw["n"], kw["k"], transa=kw["transa"], transb=kw["transb"],
                    method=kw["method"], strides=kw["strides"], comp=kw["comp"])
    if isinstance(e.value, mx.MxgError):
        assert e.value.status == 1


@pytest.mark.parametrize("combo", ["sscs", "scss", "zdds", "dzzd", "zszd", "zzsd"])
def test_imaginary_alpha_status(combo):
    with pytest.raises(mx.MxgError) as e:
        mx.mxg_plan(combo, 4, 4, 4, alpha=1 + 1j)
    assert e.value.status == 2
    mx.mxg_plan(combo[:3] + combo[3], 4, 4, 4, alpha=2.0)
    mx.mxg_plan("zzzd", 4, 4, 4, alpha=1 + 1j)
    mx.mxg_plan("dddd", 4, 4, 4, alpha=1 + 1j)


def test_split_methods_have_a_smallest_k():
    """The split-precision methods are planned only where their error floor (3 u_p^2
    per product) leaves the stated bound 4 k u_s room for the accumulation and the
    epilogue: BF16x3 from k = 320, TF32x3 from k = 32 (MXG_EACCURACY = 8 below). The
    header's numbers follow from the floor: 2.5 k >= 3 * 2^8 (1 + 2^-7) + 5.5 and
    k >= 12 (1 + 2^-10) + 5.5 in units of 2^-24, rounded up."""
    floor_bf16 = 3 * 2 ** 8 * (1 + 2 ** -7)
    floor_tf32 = 3 * 2 ** 2 * (1 + 2 ** -10)
    assert 2.5 * 320 >= floor_bf16 + 5.5 > 2.5 * 300
    assert 32 >= floor_tf32 + 5.5
    for combo in ("ssss", "zzzs", "dsss", "csss", "zcds"):
        for meth, kmin in (("bf16x3", 320), ("tf32x3", 32)):
            with pytest.raises(mx.MxgError) as e:
                mx.mxg_plan(combo, 64, 64, kmin - 1, method=meth)
            assert e.value.status == 8
            assert mx.mxg_plan(combo, 64, 64, kmin, method=meth).method == mx.METHODS[meth]
        # quick returns need no accuracy: k == 0 is C := beta C
        assert mx.mxg_plan(combo, 64, 64, 0, method="bf16x3").flops == 0
        assert mx.mxg_plan(combo, 64, 64, 1, method="ffma").flops > 0


def test_empty_operands_accept_any_strides():
    # k == 0: A is m x 0 and B is 0 x n; their strides are never used
    info = mx.mxg_plan("dddd", 5, 4, 0, strides=((1, 0), (0, 0), (1, 5)))
    assert info.flops == 0


def test_empty_C_accepts_any_strides():
    info = mx.mxg_plan("dddd", 0, 4, 3, strides=((0, 0), (1, 3), (0, 0)))
    assert info.flops == 0


def test_tune_file_round_trip(tmp_path):
    """The autotuner's decision file (host only, no CUDA call): mxg_tune_load keeps the
    lines with a known kernel variant (0..6) and schedule (0 dynamic, 1 static) and drops
    the rest; mxg_tune_save writes back exactly what is held."""
    src = tmp_path / "in.txt"
    src.write_text("\n".join([
        "d1-m5-c0-n20-f71-k16 3 0 48.6",     # DFMA 32 x 32, dynamic
        "d0-m1-c0-n20-f71-k16 1 1 1.78",     # FFMA 64 x 64, static
        "d0-m1-c0-n9-f40-k10 5 0 0.25",      # FFMA 32 x 32
        "bad-variant 9 0 1.0",               # no such kernel
        "bad-schedule 2 7 1.0",              # no such schedule
    ]) + "\n")
    assert mx.mxg_tune_load(str(src)) == 0
    out = tmp_path / "out.txt"
    assert mx.mxg_tune_save(str(out)) == 0
    held = {}
    for line in out.read_text().splitlines():
        sig, v, sch, ms = line.split()
        held[sig] = (int(v), int(sch), float(ms))
    assert held["d1-m5-c0-n20-f71-k16"] == (3, 0, pytest.approx(48.6))
    assert held["d0-m1-c0-n20-f71-k16"] == (1, 1, pytest.approx(1.78))
    assert held["d0-m1-c0-n9-f40-k10"] == (5, 0, pytest.approx(0.25))
    assert "bad-variant" not in held and "bad-schedule" not in held


def test_tune_file_errors(tmp_path):
    assert mx.mxg_tune_load(str(tmp_path / "missing.txt")) == 1     # MXG_EINVAL
    assert mx.mxg_tune_save(str(tmp_path / "no-such-dir" / "x.txt")) == 1


def test_binding_marshals_layouts_and_datatypes():
    """The Python binding only marshals: a tensor becomes (pointer, datatype code,
    row stride, column stride) in elements of its datatype; a (rows, cols, 2) binary16 /
    bfloat16 tensor is one complex matrix with halved strides; m, n, k come from C and
    op(A). Checked on CPU tensors (no CUDA call)."""
    torch = pytest.importorskip("torch")
    A = torch.zeros(6, 4, dtype=torch.complex64)                      # row-major c
    B = torch.zeros(5, 6, dtype=torch.float64).t()                    # column-major d, 6 x 5
    C = torch.zeros(9, 13, dtype=torch.float32)[::2, ::3]             # general s, 5 x 5
    arr, n = mx.make_problems([("t", "c", 1.5 - 0.5j, A, B, -0.25, C, "d")])
    p = arr[0]
    assert n == 1
    assert (p.transa, p.transb, p.m, p.n, p.k) == (1, 2, 5, 5, 6)
    assert (p.alpha_re, p.alpha_im, p.beta_re, p.beta_im) == (1.5, -0.5, -0.25, 0.0)
    assert (p.dtA, p.rsA, p.csA) == (2, 4, 1)
    assert (p.dtB, p.rsB, p.csB) == (1, 1, 6)
    assert (p.dtC, p.rsC, p.csC) == (0, 26, 3)
    assert p.A == A.data_ptr() and p.B == B.data_ptr() and p.C == C.data_ptr()
    assert p.comp_prec == 1
    # complex binary16 / bfloat16 as (rows, cols, 2), column-major over (rows, cols)
    K = torch.zeros(7, 3, 2, dtype=torch.float16).permute(1, 0, 2)    # 3 x 7 complex, strides (2, 6, 1)
    W = torch.zeros(3, 7, 2, dtype=torch.bfloat16)                    # 3 x 7 complex, row-major
    H = torch.zeros(7, 7, dtype=torch.float16)
    arr, _ = mx.make_problems([("n", "n", 1.0, K, H, 0.0, W, "h")])
    p = arr[0]
    assert (p.dtA, p.rsA, p.csA) == (5, 1, 3)
    assert (p.dtC, p.rsC, p.csC) == (7, 7, 1)
    assert (p.dtB, p.m, p.n, p.k, p.comp_prec) == (4, 3, 7, 7, 3)
    with pytest.raises(TypeError):
        mx.make_problems([("n", "n", 1.0, torch.zeros(2, 2, dtype=torch.int32), H, 0.0, H, "s")])
