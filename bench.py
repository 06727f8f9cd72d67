#!/usr/bin/env python
"""Benchmark of mixed-datatype gemm on GB300: C := beta*C + alpha*A*B.

Default workload ("plain_large"): m = n = k = 8192, column-major, no transpose,
entries U[-1, 1], alpha = beta = 1, the plain cast-then-gemm form (FP32 FFMA for
single computation precision, FP64 DMMA for double). One step = 16 gemms: the 8
domain cases of Fig. "mixeddom" x the 2 computation precisions, with the storage
precisions of (C, A, B) = pattern (step mod 8), so 8 consecutive steps cover all
128 combinations. Flops are counted as 2mnk x R (R = real products of the case).

Prints ONE JSON line (rank 0). --impl reference times the oracle (CPU) instead.
"""
import argparse
import hashlib
import itertools
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mixed-dt gemm GFLOPS & %peak per combo; grouped/served req/s, p99 vs plain"
CASES = list(itertools.product([0, 1], repeat=3))           # (C, A, B) complex?
PATTERNS = list(itertools.product("sd", repeat=3))           # (C, A, B) precision
R_OF = {(0, 0, 0): 1, (0, 0, 1): 1, (0, 1, 0): 1, (0, 1, 1): 2,
        (1, 0, 0): 1, (1, 0, 1): 2, (1, 1, 0): 2, (1, 1, 1): 4}


def real_products(combo):
    """R of the domain case of combo (C, A, B datatypes, then the computation precision)."""
    from paper_1901_06015_gb300.synth import is_complex
    return R_OF[tuple(int(is_complex(dt)) for dt in combo[:3])]
NOMINAL_BF16_TFLOPS = 2250.0
NOMINAL_FP64_TFLOPS = 1.25


def dt_of(cplx, prec):
    return ("c" if prec == "s" else "z") if cplx else prec


def step_combos(step):
    pc, pa, pb = PATTERNS[step % 8]
    out = []
    for (cc, ac, bc) in CASES:
        for x in "sd":
            out.append((dt_of(cc, pc) + dt_of(ac, pa) + dt_of(bc, pb) + x, R_OF[(cc, ac, bc)]))
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            try:
                power.append(float(f[3].split()[0]))
            except (ValueError, IndexError):
                pass
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        srt = sorted(sm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "sm_mhz_p10": srt[len(srt) // 10] if srt else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json), if
    the counters were taken on the kernel's current source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kernel)
        if not d or d.get("source_hash") != kernel_source_hash(d["source_files"]):
            return None
    except Exception:
        return None
    return d.get("dram_bytes_per_launch_at_bench_size")


def aggregate_over_ranks(dist, t_ms, flops, device=None):
    """Whole-job numbers of a replicas-only run: the slowest rank's time and the sum of
    the ranks' useful flops (no data-path collective: only this reduction of two
    scalars). Works with any torch.distributed backend (NCCL on GPUs, gloo in tests)."""
    import torch
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    f = torch.tensor([float(flops)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t[0]), float(f[0])


# ------------------------------------------------------------------ CPU (oracle) arm
def oracle_sample(step, n, bm, bn, seed=123):
    """Time the oracle on one bm x bn block of C (full k = n) for each of the step's
    16 combos. Returns (useful flops, seconds, threads)."""
    import numpy as np
    import oracle
    from paper_1901_06015_gb300 import synth
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed + step)
    flops, secs = 0.0, 0.0
    for combo, R in step_combos(step):
        A = synth.matrix(rng, bm, n, combo[1])
        B = synth.matrix(rng, n, bn, combo[2])
        C = synth.matrix(rng, bm, bn, combo[0])
        t0 = time.perf_counter()
        oracle.oracle_mxgemm("n", "n", 1.0, A, B, 1.0, C, comp=combo[3], nthreads=threads)
        secs += time.perf_counter() - t0
        flops += 2.0 * bm * bn * n * R
    return flops, secs, threads


def adhoc_sample(step, n, bm, bn, seed=123):
    """The paper's "Ad-hoc" baseline on the host cores (Sec. 8.2): copy-cast A, B and C
    to one common datatype (complex if any operand is complex, in the computation
    precision), call a same-type gemm (torch.matmul on the CPU, all threads), apply alpha
    and beta, and cast C back -- on the same bm x bn blocks of C as oracle_sample.
    Returns (useful flops 2mnkR, seconds, threads)."""
    import numpy as np
    import torch
    from paper_1901_06015_gb300 import synth
    threads = os.cpu_count() or 1
    torch.set_num_threads(threads)
    rng = np.random.default_rng(seed + step)
    flops, secs = 0.0, 0.0
    for combo, R in step_combos(step):
        A = synth.matrix(rng, bm, n, combo[1])
        B = synth.matrix(rng, n, bn, combo[2])
        C = synth.matrix(rng, bm, bn, combo[0])
        cplx = any(synth.is_complex(dt) for dt in combo[:3])
        dt = {("s", False): torch.float32, ("s", True): torch.complex64,
              ("d", False): torch.float64, ("d", True): torch.complex128}[(combo[3], cplx)]
        At, Bt, Ct = (torch.from_numpy(np.ascontiguousarray(x)) for x in (A, B, C))
        t0 = time.perf_counter()
        Ac, Bc, Cc = At.to(dt), Bt.to(dt), Ct.to(dt)
        P = torch.matmul(Ac, Bc)
        Cn = 1.0 * Cc + 1.0 * P
        out = Cn if Ct.is_complex() else (Cn.real if Cn.is_complex() else Cn)
        out = out.to(Ct.dtype)
        secs += time.perf_counter() - t0
        flops += 2.0 * bm * bn * n * R
    return flops, secs, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.size
    bm = bn = 256 if n >= 4096 else 64
    for w in range(args.warmup):
        oracle_sample(w, n, bm, bn)
    fl, secs = 0.0, 0.0
    for s in range(args.steps):
        f, t, threads = oracle_sample(s, n, bm, bn)
        fl += f
        secs += t
    gf = fl / secs / 1e9
    sample = (f"one {bm}x{bn} block of C (k={n}) per gemm of each step (16 gemms: the step's 8 domain cases x 2 "
              f"computation precisions), oracle in binary64 with compensated sums, {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": gf, "unit": "GFLOPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": gf, "unit": "GFLOPS", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": gf, "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(args):
    return {"workload": f"plain_large: 16 mixed-datatype gemms per step (8 domain cases x 2 computation "
                        f"precisions; storage precisions rotate with the step, 8 steps = all 128 combos), "
                        f"m=n=k={args.size}, column-major, no transpose, U[-1,1], alpha=beta=1",
            "m": args.size, "n": args.size, "k": args.size,
            "single_method": "ffma", "double_method": args.double_method,
            "l2": "inputs larger than L2 (every operand >= 268 MB at 8192^2), no flush"}


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    n = args.size
    stream = torch.cuda.current_stream()

    # one handle per computation precision so the contraction time of each method is
    # measured separately (same stream)
    hs, hd = mx.Handle(), mx.Handle()
    for h in (hs, hd):
        h.set_stream(stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    mats = {}

    def mat(role, dt):
        if (role, dt) not in mats:
            mats[(role, dt)] = synth.torch_matrix(gen, n, n, dt, dev)
        return mats[(role, dt)]

    for s in range(8):
        for combo, _ in step_combos(s):
            mat("A", combo[1]); mat("B", combo[2]); mat("C", combo[0])

    # load every kernel once on a small problem (lazy module loading stays out of the timing)
    small = {dt: synth.torch_matrix(gen, 64, 64, dt, dev) for dt in "sdcz"}
    for s in range(8):
        for combo, _ in step_combos(s):
            h, meth = (hs, "ffma") if combo[3] == "s" else (hd, args.double_method)
            mx.mxgemm_ex(h, meth, "n", "n", 1.0, small[combo[1]], small[combo[2]], 1.0,
                         small[combo[0]].clone(), comp=combo[3])
    torch.cuda.synchronize()

    def run_step(step, per_call=None):
        launches = 0
        for combo, R in step_combos(step):
            h, meth = (hs, "ffma") if combo[3] == "s" else (hd, args.double_method)
            if per_call is not None:
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            mx.mxgemm_ex(h, meth, "n", "n", 1.0, mat("A", combo[1]), mat("B", combo[2]), 1.0,
                         mat("C", combo[0]), comp=combo[3])
            launches += 3
            if per_call is not None:
                e1.record(stream)
                per_call.append((combo, R, e0, e1))
        return launches

    for w in range(args.warmup):
        run_step(w)
    torch.cuda.synchronize()
    for h in (hs, hd):
        h.set_phase_timing(True)

    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    per_call = []
    ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    for t in range(args.steps):
        launches += run_step(t, per_call)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    pack_s, con_s, nl_s = hs.phase_times()
    pack_d, con_d, nl_d = hd.phase_times()
    for h in (hs, hd):
        h.set_phase_timing(False)

    flops_step = sum(2.0 * n ** 3 * R for _, R in step_combos(0))
    my_flops = flops_step * args.steps
    t_max, tot_flops = aggregate_over_ranks(dist, ms, my_flops, dev)
    value = tot_flops / (t_max / 1e3) / 1e9

    # per-combo GFLOPS (this rank)
    per_combo = {}
    for combo, R, e0, e1 in per_call:
        cms = e0.elapsed_time(e1)
        per_combo[combo] = round(2.0 * n ** 3 * R / (cms / 1e3) / 1e9, 1)

    peaks, peak_src = measured_peaks()
    # dominant kernel: the double-precision contraction (nearly all of the step's time)
    d_flops = sum(2.0 * n ** 3 * R for c, R in step_combos(0) if c[3] == "d") * args.steps
    s_flops = sum(2.0 * n ** 3 * R for c, R in step_combos(0) if c[3] == "s") * args.steps
    fp64_peak = peaks["bf16_tflops_sustained"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
    ach_d = d_flops / nl_d / (con_d / nl_d / 1e3) / 1e12 if nl_d else None
    ach_s = s_flops / nl_s / (con_s / nl_s / 1e3) / 1e12 if nl_s else None
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    ffma_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    kname = "dmma_gemm" if args.double_method == "dmma" else "simt_gemm<double>"
    roofline = {
        "kernel": kname, "bound": "tensor", "achieved": ach_d, "peak": fp64_peak, "unit": "TFLOP/s",
        "frac": (ach_d / fp64_peak) if ach_d else None,
        "traffic": traffic_per_launch(kname),
        "traffic_note": "scaled, not captured at this size: DRAM bytes of one ncu capture of the kernel at "
                        "4096^3 (dddd, profiles/traffic.json) times the useful-flop ratio of the mean launch here "
                        "(2*8192^3*1.75 flops); null once the kernel's source changes",
        "peak_source": f"{peak_src} bf16_tflops_sustained x nominal FP64/BF16 ratio (1.25/2250); "
                       "kernel timed inside a long step",
        "share_of_step": con_d / ms if ms else None,
        "per_launch": "achieved = mean useful flops (2mnk R) per launch / mean contraction-kernel "
                      "duration, CUDA events around each contraction launch on its stream",
        "note": "the nominal-ratio peak understates this chip's FP64 pipe: chains of independent DMMA / DFMA "
                "measured 1.05 / 1.20 TF/s at 2002 MHz, and ncu shows the DMMA kernel's FP64 pipe 97% active",
        "frac_of_nominal_fp64": (ach_d / NOMINAL_FP64_TFLOPS) if ach_d else None,
    }
    secondary = {"kernel": "simt_gemm<float> (FFMA)", "bound": "alu", "achieved": ach_s, "peak": ffma_peak,
                 "unit": "TFLOP/s", "frac": (ach_s / ffma_peak) if ach_s else None,
                 "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x max SM clock",
                 "share_of_step": con_s / ms if ms else None}
    pack_share = (pack_s + pack_d) / ms if ms else None

    # e2e through the public API with host buffers (pinned), copies inside the timed region.
    # Pipelined as a user's loop would be: inputs go host -> device on one copy stream into
    # three rotating device buffer sets (so the inputs of gemms i+1 and i+2 load while gemm
    # i computes), and each result goes device -> host on another copy stream.
    e2e = None
    if not args.no_e2e:
        host = {key: t.cpu().pin_memory() for key, t in mats.items()}
        out = {dt: torch.empty_like(mats[("C", dt)], device="cpu").pin_memory() for dt in "sdcz"
               if ("C", dt) in mats}
        nsets = 3
        sets = [dict(mats)] + [{key: torch.empty_like(t) for key, t in mats.items()} for _ in range(nsets - 1)]
        cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        h2d = d2h = 0
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs_in.wait_stream(stream)
        cs_out.wait_stream(stream)
        free = [None] * nsets    # event: the set's last result has been read back
        last = None
        i = 0
        for t in range(args.steps):
            for combo, R in step_combos(t):
                bs = sets[i % nsets]
                dA, dB, dC = bs[("A", combo[1])], bs[("B", combo[2])], bs[("C", combo[0])]
                with torch.cuda.stream(cs_in):
                    if free[i % nsets] is not None:
                        cs_in.wait_event(free[i % nsets])
                    dA.copy_(host[("A", combo[1])], non_blocking=True)
                    dB.copy_(host[("B", combo[2])], non_blocking=True)
                    dC.copy_(host[("C", combo[0])], non_blocking=True)
                    ev_in = torch.cuda.Event()
                    ev_in.record(cs_in)
                h2d += sum(x.numel() * x.element_size() for x in (dA, dB, dC))
                stream.wait_event(ev_in)
                h, meth = (hs, "ffma") if combo[3] == "s" else (hd, args.double_method)
                mx.mxgemm_ex(h, meth, "n", "n", 1.0, dA, dB, 1.0, dC, comp=combo[3])
                ev_c = torch.cuda.Event()
                ev_c.record(stream)
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(ev_c)
                    out[combo[0]].copy_(dC, non_blocking=True)
                    last = torch.cuda.Event()
                    last.record(cs_out)
                free[i % nsets] = last
                d2h += dC.numel() * dC.element_size()
                i += 1
        if last is not None:
            stream.wait_event(last)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = e0.elapsed_time(e1)
        ems, _ = aggregate_over_ranks(dist, ems, 0.0, dev)
        e2e = {"value": tot_flops / (ems / 1e3) / 1e9, "unit": "GFLOPS",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "overlap": "inputs copied on a side stream into three rotating device buffer sets (up to "
                          "two gemms ahead) while the current gemm computes; results read back on a third stream"}
        del sets, host, out

    cpu = adhoc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f, t, threads = oracle_sample(0, n, 512, 256)
        cpu = {"value": f / t / 1e9, "unit": "GFLOPS", "cores": threads, "kind": "oracle",
               "sample": f"one 512x256 block of C (k={n}) for each of the step's 16 gemms; "
                         f"{t:.1f} s of oracle time"}
        adhoc_sample(1, n, 512, 256)   # warm-up (thread pool, allocator)
        f, t, threads = adhoc_sample(0, n, 512, 256)
        adhoc = {"value": f / t / 1e9, "unit": "GFLOPS", "cores": threads,
                 "kind": "the paper's Ad-hoc (copy-cast to one datatype + same-type torch.matmul on the CPU)",
                 "sample": f"the same 512x256 blocks of C (k={n}) as cpu_baseline; useful flops 2mnkR"}

    # %peak per combo: each call's useful GFLOPS (packs + contraction, CUDA events around
    # the call) against the pipe its contraction runs on
    # (theoretical peaks, as the paper's percentages are: FP32 lanes x 2 x max clock, and
    # the FP64 pipe's nominal rate)
    pct_peak = {c: round(100.0 * gf / (1e3 * (ffma_peak if c[3] == "s" else NOMINAL_FP64_TFLOPS)), 2)
                for c, gf in per_combo.items()}
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        del mats
        torch.cuda.empty_cache()
        forms = {}
        for name, fn in (("plain_small", plain_small_form), ("grouped", grouped_form), ("serving", serving_form)):
            try:   # a form that fails is reported in the line; the plain_large result stands
                forms[name] = fn(args)
            except Exception as exc:   # noqa: BLE001
                forms[name] = {"error": f"{type(exc).__name__}: {exc}"}
                torch.cuda.synchronize()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic", "config": workload_config(args),
            "roofline": roofline, "roofline_single": secondary, "pack_share_of_step": pack_share,
            "cpu_baseline": cpu, "adhoc_cpu": adhoc, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "per_combo_gflops": per_combo, "per_combo_pct_peak": pct_peak,
            "per_combo_peaks": {"single": {"tflops": ffma_peak, "source": secondary["peak_source"]},
                                "double": {"tflops": NOMINAL_FP64_TFLOPS,
                                           "source": "nominal FP64 rate of GB300 (theoretical peak)"}},
        }
        if forms is not None:
            g = forms["grouped"]
            line["grouped"] = {k: v for k, v in g.items() if k not in ("group",)}
            if "group" in g:
                line["grouped"]["kernels"] = [(b["precision"], b["kernel"], b["schedule"])
                                              for b in g["group"].get("buckets", [])]
            line["serving"] = forms["serving"]
            line["plain_small"] = forms["plain_small"]
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ precision workload
PRECISION_COMBOS = ["ssss", "dsss", "cscs", "zcds", "ccss"]   # (C,A,B) sss, dss, csc, zcd, ccs + comp s


def precision_seed(combo, n, dist):
    return (n * 131 + PRECISION_COMBOS.index(combo) * 7 + (dist == "loguniform")) & 0x7fffffff


def loguniform_(gen, X):
    """Overwrite X in place with sign * 10^U(-4, 4) per real component (sign kept)."""
    import torch
    rv = torch.view_as_real(X) if X.is_complex() else X
    u = torch.rand(rv.shape, generator=gen, device=rv.device, dtype=rv.dtype)
    rv.copy_(torch.sign(rv) * torch.pow(10.0, 8.0 * u - 4.0))


def precision_inputs(gen, combo, n, dist, dev):
    from paper_1901_06015_gb300 import synth
    A = synth.torch_matrix(gen, n, n, combo[1], dev)
    B = synth.torch_matrix(gen, n, n, combo[2], dev)
    C0 = synth.torch_matrix(gen, n, n, combo[0], dev)
    if dist == "loguniform":
        for X in (A, B, C0):
            loguniform_(gen, X)
    return A, B, C0


def run_precision(args):
    """Split-precision tensor-core forms vs the plain FP32 FFMA form (GFLOPS). The error
    of every result against the FP64 oracle is checked and reported by
    tests/test_precision_gpu.py on the same inputs."""
    import numpy as np
    import torch
    import paper_1901_06015_gb300 as mx

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    h = mx.Handle(); h.set_stream(stream)
    h.set_stream_k(args.stream_k)
    sizes = [int(x) for x in args.sizes.split(",")]
    methods = ["ffma", "tf32x3", "bf16x3"]
    results = []
    gen = torch.Generator(device=dev)
    sampler = ClockSampler(0)
    sampler.start()
    for dist in ("uniform", "loguniform"):
        for n in sizes:
            for combo in PRECISION_COMBOS:
                gen.manual_seed(precision_seed(combo, n, dist))
                A, B, C0 = precision_inputs(gen, combo, n, dist, dev)
                R = real_products(combo)
                for meth in methods:
                    C = C0.clone()
                    mx.mxgemm_ex(h, meth, "n", "n", 1.0, A, B, 1.0, C, comp="s")   # warm
                    times = []
                    for _ in range(args.reps):
                        C.copy_(C0)
                        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        mx.mxgemm_ex(h, meth, "n", "n", 1.0, A, B, 1.0, C, comp="s")
                        e1.record(stream)
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
                    best = min(times)
                    results.append({"combo": combo, "n": n, "dist": dist, "method": meth,
                                    "gflops": round(2.0 * n ** 3 * R / best / 1e6, 1), "ms": round(best, 3)})
                    print(json.dumps(results[-1]), file=sys.stderr, flush=True)
                del A, B, C0, C
                torch.cuda.empty_cache()
    clocks = sampler.stop()
    speed = {}
    for r in results:
        speed.setdefault(r["method"], []).append(r["gflops"])
    gm = {m: float(np.exp(np.mean(np.log(v)))) for m, v in speed.items()}
    line = {"metric": METRIC, "workload": "precision", "value": gm.get("bf16x3"), "unit": "GFLOPS",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32 (bf16/tf32 split planes)", "data": "synthetic",
            "config": {"workload": "precision form: combos sss, dss, csc, zcd, ccs (comp single), m=n=k in "
                       + args.sizes + ", uniform U[-1,1] and log-uniform sign*10^U(-4,4); best of "
                       + str(args.reps) + " (the call includes its pack kernels)"},
            "geomean_gflops": gm, "speedup_vs_ffma": {m: gm[m] / gm["ffma"] for m in gm},
            "clocks": clocks, "results": results}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ plain small form
def plain_small_form(args, reps=20):
    """The plain method on small problems: one mxgemm_ex call (AUTO: FFMA single, DFMA
    double) for each of the 128 combinations at m = n = k = 128, column-major, no
    transpose, U[-1, 1], alpha = 1.5, beta = -0.5 -- launch-latency bound. Per combo: the
    mean of `reps` back-to-back calls (CUDA events around them on the stream)."""
    import torch
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    h = mx.Handle(); h.set_stream(stream)
    gen = torch.Generator(device=dev); gen.manual_seed(0)
    n = 128
    per, dev_us = {}, {}
    for combo in synth.all_combos():
        A = synth.torch_matrix(gen, n, n, combo[1], dev)
        B = synth.torch_matrix(gen, n, n, combo[2], dev)
        C = synth.torch_matrix(gen, n, n, combo[0], dev)
        for _ in range(3):
            mx.mxgemm_ex(h, "auto", "n", "n", 1.5, A, B, -0.5, C, comp=combo[3])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            mx.mxgemm_ex(h, "auto", "n", "n", 1.5, A, B, -0.5, C, comp=combo[3])
        e1.record(stream)
        torch.cuda.synchronize()
        per[combo] = e0.elapsed_time(e1) / reps * 1e3            # microseconds per call
        # a second pass with the library's phase timing: the call's kernels alone (its
        # events between the launches add a little)
        h.set_phase_timing(True)
        for _ in range(reps):
            mx.mxgemm_ex(h, "auto", "n", "n", 1.5, A, B, -0.5, C, comp=combo[3])
        pk, ct, nl = h.phase_times()
        h.set_phase_timing(False)
        dev_us[combo] = (pk + ct) / max(nl, 1) * 1e3
    h.close()
    us = sorted(per.values())
    du = sorted(dev_us.values())
    flops = {c: 2.0 * n ** 3 * real_products(c) for c in per}
    return {"workload": "plain small: one call per combination, m=n=k=128, column-major, U[-1,1], alpha=1.5, "
                        "beta=-0.5, method AUTO (FFMA single, DFMA double); mean of %d back-to-back calls" % reps,
            "us_per_call_median": us[len(us) // 2], "us_per_call_min": us[0], "us_per_call_max": us[-1],
            "device_us_per_call_median": du[len(du) // 2], "device_us_per_call_min": du[0],
            "device_us_per_call_max": du[-1],
            "timing": "us_per_call: CUDA events around 20 back-to-back calls from Python (host planning, the "
                      "ctypes call and three launches); device_us: a second pass of 20 calls with the library's "
                      "phase timing (events before, between and after its launches)",
            "gflops_all_combos": sum(flops.values()) / (sum(per.values()) / 1e6) / 1e9,
            "per_combo_us": {c: round(v, 2) for c, v in per.items()}}


# ------------------------------------------------------------------ grouped workload
def grouped_problems(count, seed, lo, hi, dev):
    """count independent problems: m, n, k = round(exp(U(ln lo, ln hi))), combination
    uniform over the 128, entries U[-1, 1], alpha = 1.5, beta = -0.5."""
    import numpy as np
    import torch
    from paper_1901_06015_gb300 import synth
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    combos = synth.all_combos()
    items, flops = [], 0.0
    for _ in range(count):
        combo = combos[int(rng.integers(len(combos)))]
        m, n, k = (int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi)))))) for _ in range(3))
        A = synth.torch_matrix(gen, m, k, combo[1], dev)
        B = synth.torch_matrix(gen, k, n, combo[2], dev)
        C = synth.torch_matrix(gen, m, n, combo[0], dev)
        items.append(("n", "n", 1.5, A, B, -0.5, C, combo[3]))
        R = real_products(combo)
        flops += 2.0 * m * n * k * R
    return items, flops


def grouped_form(args):
    """One graph-captured grouped launch of args.count problems (autotuned) vs the same
    problems as separate plain calls. Returns the measurement as a dict."""
    import torch
    import paper_1901_06015_gb300 as mx
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    items, flops = grouped_problems(args.count, 0, 16, 1024, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = mx.Group(items, tune=True, graph=True, stream=stream, method_s=args.method_s)
    create_s = time.perf_counter() - t0
    desc = g.describe()
    h = mx.Handle(); h.set_stream(stream)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    k_of = [(A.shape[0] if ta in "th" else A.shape[1]) for (ta, tb, al, A, B, be, C, x) in items]
    min_k = {"bf16x3": 320, "tf32x3": 32}.get(args.method_s, 0)

    def separate():
        for (ta, tb, al, A, B, be, C, x), k in zip(items, k_of):
            meth = args.method_s if (x == "s" and k >= min_k and args.method_s != "auto") else "auto"
            mx.mxgemm_ex(h, meth, ta, tb, al, A, B, be, C, comp=x)

    steps, warmup = max(args.steps, 5), max(args.warmup, 3)
    sampler = ClockSampler(0)
    sampler.start()
    ms_g = timed(g.run, steps, warmup)
    ms_s = timed(separate, steps, warmup)
    clocks = sampler.stop()
    # the same grouped run without the tuner (first candidate, dynamic schedule)
    g2 = mx.Group(items, tune=False, graph=True, stream=stream, method_s=args.method_s)
    ms_g2 = timed(g2.run, steps, warmup)
    g.close(); g2.close(); h.close()
    del items
    torch.cuda.empty_cache()
    return {"problems": args.count, "steps": steps, "warmup": warmup, "ms": ms_g,
            "problems_per_s": args.count / (ms_g / 1e3), "gflops": flops / (ms_g / 1e3) / 1e9,
            "separate_ms": ms_s, "separate_problems_per_s": args.count / (ms_s / 1e3),
            "separate_gflops": flops / (ms_s / 1e3) / 1e9, "speedup_vs_separate": ms_s / ms_g,
            "untuned_grouped_ms": ms_g2, "useful_gflop_per_run": flops / 1e9, "create_s": create_s,
            "group": desc, "clocks": clocks,
            "workload": f"batching: {args.count} independent gemms, m,n,k = round(exp(U(ln16, ln1024))), "
                        "combination uniform over the 128, U[-1,1], alpha=1.5, beta=-0.5, seed 0; one "
                        "graph-captured grouped persistent launch (autotuned) vs separate plain calls on one stream"}


def run_grouped(args):
    """The batching form alone (one JSON line)."""
    r = grouped_form(args)
    line = {"metric": METRIC, "workload": "grouped", "value": r["problems_per_s"], "unit": "problems/s",
            "n_gpus": 1, "steps": r["steps"], "warmup": r["warmup"], "ms_per_step": r["ms"],
            "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": r["workload"]}, **{k: v for k, v in r.items() if k not in ("workload",)}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ serving workload
def serving_form(args):
    """Poisson arrivals of mixed-datatype requests (m, n, k log-uniform in [32, 4096],
    combination uniform over the 128, alpha, beta ~ U[-2, 2]) served with continuous
    batching vs the same trace as serial plain calls on one stream. Returns a dict."""
    import numpy as np
    import torch
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(0)
    combos = synth.all_combos()
    N = args.requests
    mmax = 4096
    # operand pools: every request reads views of these (column-major, leading dim 4096)
    gen = torch.Generator(device=dev); gen.manual_seed(7)
    poolA = {dt: synth.torch_matrix(gen, mmax, mmax, dt, dev) for dt in "sdcz"}
    poolB = {dt: synth.torch_matrix(gen, mmax, mmax, dt, dev) for dt in "sdcz"}
    poolC = {dt: synth.torch_matrix(gen, mmax, mmax, dt, dev) for dt in "sdcz"}
    reqs = []
    for i in range(N):
        combo = combos[int(rng.integers(len(combos)))]
        m, n, k = (int(round(float(np.exp(rng.uniform(np.log(32), np.log(4096)))))) for _ in range(3))
        al, be = float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2))
        R = real_products(combo)
        reqs.append((combo, m, n, k, al, be, 2.0 * m * n * k * R))
    total_flops = sum(r[6] for r in reqs)

    def item(r):
        combo, m, n, k, al, be, _ = r
        return ("n", "n", al, poolA[combo[1]][:m, :k], poolB[combo[2]][:k, :n], be, poolC[combo[0]][:m, :n], combo[3])

    # offline capacity: serial service time of a seeded sample, back to back on one stream
    h = mx.Handle(); h.set_stream(torch.cuda.current_stream())
    sample = [reqs[int(j)] for j in rng.choice(N, size=min(args.capacity_sample, N), replace=False)]
    for r in sample[:50]:
        it = item(r); mx.mxgemm_ex(h, "auto", *it[:7], comp=it[7])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in sample:
        it = item(r); mx.mxgemm_ex(h, "auto", *it[:7], comp=it[7])
    torch.cuda.synchronize()
    mean_service = (time.perf_counter() - t0) / len(sample)
    sample_flops = sum(r[6] for r in sample) / len(sample)
    capacity = 1.0 / mean_service                      # requests / s
    lam = args.load * capacity
    gaps = rng.exponential(1.0 / lam, size=N)
    arrivals = np.cumsum(gaps)

    def serve(fifo, burst=0):
        """Serve the trace (Poisson arrivals), or with burst > 0 its first `burst` requests
        submitted at once (saturation: the completion rate is the form's capacity)."""
        srv = mx.Server(n_streams=1 if fifo else args.streams, hbm_budget_bytes=args.budget_gb << 30,
                        small_flops=args.small_flops, fifo=fifo)
        todo = reqs[:burst] if burst else reqs
        arr = [mx.make_problems([item(r)])[0] for r in todo]
        base = srv.now()
        for i in range(len(todo)):
            target = base + (0.0 if burst else arrivals[i])
            while True:
                d = target - srv.now()
                if d <= 0:
                    break
                time.sleep(min(d, 0.002) if d > 0.0005 else 0)
            rid = __import__("ctypes").c_uint64(0)
            mx.lib().mxg_server_submit(srv.s, arr[i], __import__("ctypes").byref(rid))
        srv.drain(3600)
        comps = srv.poll(len(todo) + 10)
        st = srv.stats()
        srv.close()
        lat = np.array([c["done"] - c["arrival"] for c in comps if c["status"] == 0])
        t_first = min(c["arrival"] for c in comps); t_last = max(c["done"] for c in comps)
        fl = sum(r[6] for r in todo)
        large_wait = [c["admit"] - c["arrival"] for c in comps if c["flops"] > args.small_flops]
        return {"requests_per_s": len(lat) / (t_last - t_first), "gflops": fl / (t_last - t_first) / 1e9,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p90_ms": float(np.percentile(lat, 90) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "failed": int(st["failed"]), "max_in_flight": int(st["max_in_flight"]),
                "peak_bytes_in_flight": int(st["peak_bytes_in_flight"]), "span_s": t_last - t_first,
                "waves": int(st["waves"]), "wave_requests": int(st["wave_requests"]),
                "max_queue_ms_large": float(max(large_wait) * 1e3) if large_wait else None}

    sampler = ClockSampler(0)
    sampler.start()
    served = serve(False)
    serial = serve(True)
    sat = None
    if args.saturation > 0:
        b = min(args.saturation, N)
        sat_served, sat_serial = serve(False, b), serve(True, b)
        sat = {"requests": b, "served_requests_per_s": sat_served["requests_per_s"],
               "serial_requests_per_s": sat_serial["requests_per_s"],
               "served_gflops": sat_served["gflops"], "serial_gflops": sat_serial["gflops"],
               "capacity_ratio": sat_served["requests_per_s"] / sat_serial["requests_per_s"],
               "served_failed": sat_served["failed"], "serial_failed": sat_serial["failed"]}
    clocks = sampler.stop()
    del poolA, poolB, poolC
    torch.cuda.empty_cache()
    # the FP64 pipe bounds both forms: the double-precision requests' flops at the nominal
    # FP64 rate, per request of the trace
    fp64_s = sum(r[6] for r in reqs if r[0][3] == "d" or (r[0][3] == "c" and r[0][0] in "dz")) / (
        NOMINAL_FP64_TFLOPS * 1e12)
    return {"requests": N, "load": args.load, "arrival_rate": lam, "capacity_requests_per_s": capacity,
            "fp64_bound_requests_per_s": N / fp64_s if fp64_s > 0 else None,
            "mean_service_ms": mean_service * 1e3, "mean_request_gflop": total_flops / N / 1e9,
            "served": served, "serial": serial,
            "p99_speedup_vs_serial": serial["p99_ms"] / served["p99_ms"],
            "p50_speedup_vs_serial": serial["p50_ms"] / served["p50_ms"], "saturation": sat, "clocks": clocks,
            "workload": f"serving: {N} requests, Poisson arrivals at {args.load} x offline capacity, "
                        "m,n,k log-uniform in [32,4096], combination uniform over the 128, alpha,beta ~ U[-2,2]; "
                        f"continuous batching over {args.streams} streams (small <= {args.small_flops:g} flops on "
                        f"a high-priority stream), HBM budget {args.budget_gb} GiB, vs serial plain calls on one "
                        "stream"}


def run_serving(args):
    """The serving form alone (one JSON line)."""
    r = serving_form(args)
    line = {"metric": METRIC, "workload": "serving", "value": r["served"]["requests_per_s"], "unit": "requests/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": r["workload"], "requests": r["requests"], "load": r["load"]},
            **{k: v for k, v in r.items() if k not in ("workload",)}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ single-call workload
def run_single(args):
    """Repeated calls of one combination with one method (micro-benchmark, and the
    small case the ncu captures run)."""
    import torch
    import paper_1901_06015_gb300 as mx
    from paper_1901_06015_gb300 import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    combo, n = args.combo, args.size
    mm, nn, kk = (int(x) for x in args.mnk.split(",")) if args.mnk else (n, n, n)
    gen = torch.Generator(device=dev); gen.manual_seed(3)

    def operand(dt, layout, rows, cols):
        X = synth.torch_matrix(gen, rows, cols, dt, dev)      # column-major
        if layout == "row":
            return X.contiguous()                             # row-major copy
        if layout == "gen":                                   # general storage: stride 2 in both
            big = torch.zeros((2 * rows, 2 * cols), dtype=X.dtype, device=dev)
            v = big[::2, ::2]
            v.copy_(X)
            return v
        return X

    la, lb, lc = (args.layout.split(",") + ["col"] * 3)[:3]
    A = operand(combo[1], la, *((kk, mm) if args.transa in "th" else (mm, kk)))
    B = operand(combo[2], lb, *((nn, kk) if args.transb in "th" else (kk, nn)))
    C = operand(combo[0], lc, mm, nn)
    h = mx.Handle(); h.set_stream(stream)
    h.set_split_k(args.split_k)
    h.set_cta_pairs(args.cta_pairs)
    h.set_stream_k(args.stream_k)
    R = real_products(combo)
    times = []
    h.set_phase_timing(True)
    sampler = ClockSampler(0)
    sampler.start()
    for i in range(args.warmup + args.reps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mx.mxgemm_ex(h, args.method, args.transa, args.transb, 1.0, A, B, 1.0, C, comp=combo[3])
        e1.record(stream)
        torch.cuda.synchronize()
        if i == args.warmup - 1 or (args.warmup == 0 and i == 0):
            h.phase_times()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    pack_ms, con_ms, nl = h.phase_times()
    fl = 2.0 * mm * nn * kk * R
    # C is read and written once in its storage type (beta = 1): with k = 0 the call is the
    # stand-alone C := beta*C launch, with a small k the contraction kernel's time is
    # dominated by its fused epilogue, so this is the epilogue's HBM rate
    c_bytes = 2.0 * mm * nn * C.element_size() * (2 if C.dim() == 3 else 1)
    c_ms = (con_ms / nl) if nl else min(times)
    line = {"workload": "single", "combo": combo, "method": args.method, "m_n_k": [mm, nn, kk], "reps": args.reps,
            "split_k": args.split_k, "cta_pairs": args.cta_pairs, "stream_k": args.stream_k,
            "layout": [la, lb, lc], "trans": [args.transa, args.transb],
            "best_ms": min(times), "gflops": fl / min(times) / 1e6,
            "contraction_ms_mean": con_ms / max(nl, 1), "pack_ms_mean": pack_ms / max(nl, 1),
            "contraction_tflops": fl / (con_ms / max(nl, 1)) / 1e9 if nl else None,
            "c_bytes": c_bytes, "c_gbs": c_bytes / c_ms / 1e6 if c_ms > 0 else None, "clocks": clocks}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--double-method", default="dmma", choices=["dmma", "dfma"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the plain-small, grouped and serving forms that follow plain_large")
    ap.add_argument("--workload", default="plain_large", choices=["plain_large", "plain_small", "precision", "grouped", "serving", "single"])
    ap.add_argument("--count", type=int, default=2048)
    ap.add_argument("--method-s", default="auto", choices=["auto", "ffma", "tf32x3", "bf16x3"],
                    help="grouped workload: method of the single-precision problems")
    ap.add_argument("--combo", default="dddd")
    ap.add_argument("--method", default="auto")
    ap.add_argument("--layout", default="col,col,col", help="storage of A,B,C: col | row | gen")
    ap.add_argument("--transa", default="n")
    ap.add_argument("--transb", default="n")
    ap.add_argument("--mnk", default="", help="m,n,k for --workload single (default: --size cubed)")
    ap.add_argument("--split-k", type=int, default=0)
    ap.add_argument("--cta-pairs", type=int, default=0, help="tensor-core methods: 0 auto, 1 pairs, 2 single CTAs")
    ap.add_argument("--stream-k", type=int, default=1,
                    help="stream-K tail of the CTA-pair kernel: 0 off, 1 auto, 2 whenever the last wave is partial")
    ap.add_argument("--requests", type=int, default=100000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--budget-gb", type=int, default=48)
    ap.add_argument("--small-flops", type=float, default=2e8)
    ap.add_argument("--capacity-sample", type=int, default=3000)
    ap.add_argument("--saturation", type=int, default=5000,
                    help="serving: also submit this many requests at once to each form (0: skip)")
    ap.add_argument("--sizes", default="4096,8192,16384")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "grouped":
        return run_grouped(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload == "plain_small":
        r = plain_small_form(args)
        print(json.dumps({"metric": METRIC, "workload": "plain_small", "value": r["gflops_all_combos"],
                          "unit": "GFLOPS", "n_gpus": 1, "higher_is_better": True, "dtype": "f64+f32",
                          "data": "synthetic", "config": {"workload": r["workload"]},
                          **{k: v for k, v in r.items() if k != "workload"}}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
