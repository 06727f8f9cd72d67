"""The bounds-checking debug build (GPU). Built with MXG_DEBUG_BOUNDS, every pack
kernel and epilogue checks each element address it computes against the extent its
arguments describe, and a violation sets bit 1 of the device error word instead of
touching memory. On valid calls the word stays 0 and the results equal the normal
build's bit for bit (the checks change no arithmetic). Runs in a subprocess, since one
process loads one build of the library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# every pack pattern and output mode, general / row / column storage, all four method
# families, split-K, and a 16-bit combination; the child prints C's bytes as hex
CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1901_06015_gb300 as mx
from paper_1901_06015_gb300 import synth
from tests.gpu_util import to_device, from_device
cases = [("zzzd", "dmma", "n", "t", "F"), ("cscs", "bf16x3", "h", "n", "C"), ("zcds", "tf32x3", "t", "c", "F"),
         ("dzzs", "ffma", "c", "h", "C"), ("zddd", "dfma", "n", "n", "F"), ("kkkh", "tc16", "n", "t", "F"),
         ("sdzs", "ffma", "t", "n", "F")]
h = mx.Handle(); h.set_stream(torch.cuda.current_stream())
hk = mx.Handle(); hk.set_stream(torch.cuda.current_stream()); hk.set_split_k(3)
out = {"debug": int(mx.lib().mxg_debug_bounds()), "results": []}
for i, (combo, meth, ta, tb, oc) in enumerate(cases):
    k = 330 if meth in ("bf16x3", "tf32x3") else 97
    A, B, C0 = synth.problem(80 + i, combo, 70, 150, k, transa=ta, transb=tb, order_c=oc)
    alpha = (1.25 - 0.5j) if all(synth.is_complex(t) for t in combo[:3]) else 1.5
    beta = (0.5 + 0.25j) if synth.is_complex(combo[0]) else -0.5
    for handle in ((h, hk) if meth in ("ffma", "dfma", "dmma") else (h,)):
        dA, dB, dC = to_device(A), to_device(B), to_device(C0)
        mx.mxgemm_ex(handle, meth, ta, tb, alpha, dA, dB, beta, dC, comp=combo[3])
        torch.cuda.synchronize()
        out["results"].append(np.ascontiguousarray(from_device(dC, combo[0])).tobytes().hex())
out["word"] = h.check_device_error() | hk.check_device_error()
print(json.dumps(out))
"""


def _run(debug):
    env = dict(os.environ)
    env["MXG_DEBUG_BOUNDS"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_bounds_build_is_silent_on_valid_calls_and_changes_no_result():
    dbg = _run(True)
    ref = _run(False)
    assert dbg["debug"] == 1 and ref["debug"] == 0
    assert dbg["word"] == 0 and ref["word"] == 0
    assert dbg["results"] == ref["results"]
