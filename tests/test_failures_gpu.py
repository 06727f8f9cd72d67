"""Resource failures made on the host (GPU tests; nothing here faults or hangs the GPU):
a caller workspace smaller than the plan needs, and a served request whose packed
operands can never fit the server's arena. Each must come back as MXG_ENOMEM (3) for
that call or request alone, with C untouched and the other work unaffected."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from paper_1901_06015_gb300 import synth
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import from_device, to_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_caller_workspace_too_small_is_enomem_and_c_unchanged():
    import paper_1901_06015_gb300 as mx
    combo, (m, n, k) = "zzzd", (100, 90, 80)
    need = mx.mxg_plan(combo, m, n, k).workspace_bytes
    A, B, C0 = synth.problem(60, combo, m, n, k)
    dA, dB = to_device(A), to_device(B)
    h = mx.Handle()
    h.set_stream(torch.cuda.current_stream())
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    h.set_workspace(small)
    dC = to_device(C0)
    with pytest.raises(mx.MxgError) as e:
        mx.mxgemm_ex(h, "auto", "n", "n", 1.5, dA, dB, -0.5, dC, comp="d")
    assert e.value.status == 3
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), C0)
    # exactly the planned size is enough, and gives the library-workspace result
    exact = torch.empty(need, dtype=torch.uint8, device="cuda")
    h.set_workspace(exact)
    mx.mxgemm_ex(h, "auto", "n", "n", 1.5, dA, dB, -0.5, dC, comp="d")
    h.set_workspace(None)
    dC2 = to_device(C0)
    mx.mxgemm_ex(h, "auto", "n", "n", 1.5, dA, dB, -0.5, dC2, comp="d")
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), dC2.cpu().numpy())
    h.close()


def test_server_request_beyond_the_arena_fails_alone():
    """A 1 MiB arena: one request needs more packed-operand space than the whole arena
    and completes with MXG_ENOMEM, C untouched; the small requests around it complete
    and match the oracle."""
    import paper_1901_06015_gb300 as mx
    budget = 1 << 20
    big = ("zzzd", 300, 300, 300)
    assert mx.mxg_plan(*big).workspace_bytes > budget
    specs = [("dsdd", 40, 30, 20), big, ("cscs", 33, 20, 17), ("sdds", 25, 25, 25)]
    srv = mx.Server(n_streams=2, hbm_budget_bytes=budget, small_flops=1e6)
    probs, ids = [], []
    for i, (combo, m, n, k) in enumerate(specs):
        A, B, C0 = synth.problem(70 + i, combo, m, n, k)
        dA, dB, dC = to_device(A), to_device(B), to_device(C0)
        ids.append(srv.submit(("n", "n", 1.5, dA, dB, -0.5, dC, combo[3]), keep=(dA, dB, dC)))
        probs.append((combo, k, A, B, C0, dC))
    srv.drain(60)
    status = {c["id"]: c["status"] for c in srv.poll()}
    srv.close()
    for rid, (combo, k, A, B, C0, dC) in zip(ids, probs):
        got = from_device(dC, combo[0])
        if (combo, A.shape[0]) == (big[0], big[1]):
            assert status[rid] == 3
            assert np.array_equal(got, C0)
        else:
            assert status[rid] == 0
            ref = oracle_mxgemm("n", "n", 1.5, A, B, -0.5, C0.copy(order="F"), comp=combo[3])
            err, _ = normwise_error(combo, got, ref, A, B, C0, 1.5, -0.5)
            assert err <= tolerance(combo, k), (combo, err)
