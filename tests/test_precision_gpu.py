"""Precision form (GPU): the split-precision tensor-core products (TF32x3, BF16x3) and
the plain FFMA form, on the benchmark's precision inputs (combos sss, dss, csc, zcd,
ccs with computation precision single; m = n = k in {4096, 8192, 16384}; U[-1, 1] and
log-uniform sign*10^U(-4, 4)). Each result is compared with the FP64 oracle on two
sampled 32 x 32 blocks. With MXG_REPORT=<file>, every error is appended to that file
as one JSON line."""
import json
import os

import numpy as np
import pytest

from oracle import oracle_mxgemm
from tests._helpers import normwise_error, tolerance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [int(x) for x in os.environ.get("MXG_PRECISION_SIZES", "4096,8192,16384").split(",")]


@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
@pytest.mark.parametrize("n", SIZES)
def test_precision_form_errors(n, dist):
    import bench
    import paper_1901_06015_gb300 as mx
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    report = os.environ.get("MXG_REPORT")
    for combo in bench.PRECISION_COMBOS:
        gen.manual_seed(bench.precision_seed(combo, n, dist))
        A, B, C0 = bench.precision_inputs(gen, combo, n, dist, dev)
        bs = 32
        rng = np.random.default_rng(n)
        pos = [(0, 0), tuple(int(v) for v in rng.integers(0, n - bs, size=2))]
        refs = []
        for (i, j) in pos:
            Ap = np.asfortranarray(A[i:i + bs, :].cpu().numpy())
            Bp = np.asfortranarray(B[:, j:j + bs].cpu().numpy())
            Cb = np.asfortranarray(C0[i:i + bs, j:j + bs].cpu().numpy())
            refs.append((Ap, Bp, Cb, oracle_mxgemm("n", "n", 1.0, Ap, Bp, 1.0, Cb.copy(order="F"), comp="s")))
        for meth in ("ffma", "tf32x3", "bf16x3"):
            C = C0.clone()
            mx.mxgemm_ex(None, meth, "n", "n", 1.0, A, B, 1.0, C, comp="s")
            torch.cuda.synchronize()
            errs = []
            for (i, j), (Ap, Bp, Cb, ref) in zip(pos, refs):
                got = C[i:i + bs, j:j + bs].cpu().numpy()
                errs.append(normwise_error(combo, got, ref, Ap, Bp, Cb, 1.0, 1.0)[0])
            tol = tolerance(combo, n, meth)
            if report:
                with open(report, "a") as f:
                    f.write(json.dumps({"combo": combo, "n": n, "dist": dist, "method": meth,
                                        "err": max(errs), "tol": tol}) + "\n")
            assert max(errs) <= tol, (combo, n, dist, meth, errs, tol)
            del C
        del A, B, C0
        torch.cuda.empty_cache()
