"""Serving loop (GPU): requests submitted while others run are admitted by HBM
footprint and overlap on several streams; every result is the same as the request run
alone (bit for bit, same kernels) and within tolerance of the oracle."""
import numpy as np
import pytest

from oracle import oracle_mxgemm
from tests._helpers import normwise_error, tolerance
from tests.gpu_util import to_device
from tests.test_grouped_gpu import _problems, _solo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_and_oracle():
    import paper_1901_06015_gb300 as mx
    probs = _problems(11, 160, lo=8, hi=400)
    budget = 48 << 20    # small enough that admission has to wait for memory
    srv = mx.Server(n_streams=4, hbm_budget_bytes=budget, small_flops=2e6)
    dev = []
    for p in probs:
        dA, dB, dC = to_device(p["A"]), to_device(p["B"]), to_device(p["C"])
        dev.append(dC)
        srv.submit((p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, p["combo"][3]), keep=(dA, dB))
    srv.drain(120)
    comps = srv.poll(10000)
    st = srv.stats()
    derr = srv.check_device_error()    # no device-side wait ran out
    srv.close()
    assert derr == 0
    assert len(comps) == len(probs) and all(c["status"] == 0 for c in comps)
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert st["peak_bytes_in_flight"] <= budget or st["max_in_flight"] == 1
    assert st["max_in_flight"] > 1                     # work overlapped
    assert len({c["stream"] for c in comps}) > 1       # more than one stream used
    for c in comps:
        assert c["arrival"] <= c["admit"] + 1e-6 and c["admit"] <= c["done"] + 1e-3
    torch.cuda.synchronize()
    for p, dC in zip(probs, dev):
        got = dC.cpu().numpy()
        assert np.array_equal(got, _solo(p, "ffma", "dmma")), p["combo"]
        ref_C = np.array(p["C"], order="K")
        ref = oracle_mxgemm(p["ta"], p["tb"], p["alpha"], p["A"], p["B"], p["beta"], ref_C, comp=p["combo"][3])
        k = p["A"].shape[0] if p["ta"] in "th" else p["A"].shape[1]
        err, _ = normwise_error(p["combo"], got, ref, p["A"], p["B"], p["C"], p["alpha"], p["beta"], p["ta"], p["tb"])
        assert err <= tolerance(p["combo"], k)


def test_fifo_baseline_runs_in_order_on_one_stream():
    import paper_1901_06015_gb300 as mx
    probs = _problems(12, 40, lo=8, hi=200, trans=False)
    srv = mx.Server(n_streams=1, hbm_budget_bytes=1 << 30, fifo=True)
    keep = []
    for p in probs:
        dA, dB, dC = to_device(p["A"]), to_device(p["B"]), to_device(p["C"])
        keep.append((dA, dB, dC))
        srv.submit(("n", "n", p["alpha"], dA, dB, p["beta"], dC, p["combo"][3]))
    srv.drain(60)
    comps = sorted(srv.poll(1000), key=lambda c: c["id"])
    srv.close()
    assert all(c["stream"] == 0 and c["status"] == 0 for c in comps)
    done = [c["done"] for c in comps]
    assert all(a <= b + 1e-6 for a, b in zip(done, done[1:]))


def test_invalid_request_completes_with_its_status():
    import paper_1901_06015_gb300 as mx
    srv = mx.Server(n_streams=2, hbm_budget_bytes=1 << 26)
    A = torch.zeros((4, 3), dtype=torch.float32, device="cuda").t().contiguous().t()
    B = torch.zeros((3, 2), dtype=torch.complex64, device="cuda").t().contiguous().t()
    C = torch.zeros((4, 2), dtype=torch.float32, device="cuda").t().contiguous().t()
    rid = srv.submit(("n", "n", 1.0 + 1.0j, A, B, 0.0, C, "s"))   # case 1b with complex alpha
    srv.drain(10)
    comps = srv.poll()
    srv.close()
    assert comps[0]["id"] == rid and comps[0]["status"] == 2


def test_serving_configuration_sampled_blocks():
    """Requests drawn as the serving configuration draws them (m, n, k log-uniform in
    [32, 4096], combination uniform over the 128, alpha and beta uniform in [-2, 2]),
    submitted back to back to a 4-stream server with admission by HBM footprint; A and
    B are views of shared operand pools, every request has its own C. Each result is
    checked against the oracle on a block of up to 16 x 16 entries of C."""
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    rng = np.random.default_rng(2)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    pool_a = {dt: synth.torch_matrix(gen, 4096, 4096, dt, "cuda") for dt in "sdcz"}
    pool_b = {dt: synth.torch_matrix(gen, 4096, 4096, dt, "cuda") for dt in "sdcz"}
    combos = synth.all_combos()
    srv = mx.Server(n_streams=4, hbm_budget_bytes=8 << 30, small_flops=2e8)
    reqs = []
    for _ in range(300):
        combo = combos[int(rng.integers(len(combos)))]
        m, n, k = (int(round(float(np.exp(rng.uniform(np.log(32), np.log(4096)))))) for _ in range(3))
        al, be = float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2))
        A, B = pool_a[combo[1]][:m, :k], pool_b[combo[2]][:k, :n]
        C = synth.torch_matrix(gen, m, n, combo[0], "cuda")
        rows = torch.as_tensor(np.sort(rng.choice(m, size=min(m, 16), replace=False)), device="cuda")
        cols = torch.as_tensor(np.sort(rng.choice(n, size=min(n, 16), replace=False)), device="cuda")
        C0 = C[rows][:, cols].cpu().numpy()
        srv.submit(("n", "n", al, A, B, be, C, combo[3]), keep=(A, B))
        reqs.append((combo, k, al, be, A, B, C, rows, cols, C0))
    srv.drain(600)
    comps = srv.poll(1000)
    derr = srv.check_device_error()
    srv.close()
    assert derr == 0 and len(comps) == len(reqs) and all(c["status"] == 0 for c in comps)
    torch.cuda.synchronize()
    for combo, k, al, be, A, B, C, rows, cols, C0 in reqs:
        Ab, Bb = A[rows].cpu().numpy(), B[:, cols].cpu().numpy()
        got = C[rows][:, cols].cpu().numpy()
        ref = oracle_mxgemm("n", "n", al, Ab, Bb, be, np.array(C0, order="F"), comp=combo[3])
        err, _ = normwise_error(combo, got, ref, Ab, Bb, C0, al, be)
        assert err <= tolerance(combo, k), (combo, k, err)


def test_small_requests_batched_into_waves_equal_solo():
    """A burst of small requests (all combinations, transposes, both computation
    precisions): those admitted while a wave runs on the high-priority stream are
    batched into the next wave (one grouped launch); every result still equals the same
    request run alone bit for bit and is within the bound of the oracle."""
    import paper_1901_06015_gb300 as mx
    probs = _problems(13, 240, lo=4, hi=64)
    dev = [(to_device(p["A"]), to_device(p["B"]), to_device(p["C"])) for p in probs]
    torch.cuda.synchronize()
    srv = mx.Server(n_streams=3, hbm_budget_bytes=1 << 30, small_flops=1e7)
    for p, (dA, dB, dC) in zip(probs, dev):
        srv.submit((p["ta"], p["tb"], p["alpha"], dA, dB, p["beta"], dC, p["combo"][3]))
    srv.drain(120)
    comps = srv.poll(1000)
    st = srv.stats()
    derr = srv.check_device_error()
    srv.close()
    assert derr == 0 and all(c["status"] == 0 for c in comps) and len(comps) == len(probs)
    assert st["waves"] >= 1 and st["wave_requests"] >= 2 * st["waves"]
    torch.cuda.synchronize()
    for p, (_, _, dC) in zip(probs, dev):
        got = dC.cpu().numpy()
        assert np.array_equal(got, _solo(p, "ffma", "dfma")), p["combo"]
        ref = oracle_mxgemm(p["ta"], p["tb"], p["alpha"], p["A"], p["B"], p["beta"], np.array(p["C"], order="K"),
                            comp=p["combo"][3])
        k = p["A"].shape[0] if p["ta"] in "th" else p["A"].shape[1]
        err, _ = normwise_error(p["combo"], got, ref, p["A"], p["B"], p["C"], p["alpha"], p["beta"], p["ta"], p["tb"])
        assert err <= tolerance(p["combo"], k), (p["combo"], err)
