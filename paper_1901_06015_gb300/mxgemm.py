"""ctypes binding of the C ABI in ``include/mxgemm.h`` (argument marshalling only).

Every computation happens in the CUDA library; this module turns torch tensors into
(pointer, datatype code, row stride, column stride) and Python scalars into
(re, im) pairs. Tensors are passed as stored: for trans 't'/'h', A is the stored
k x m matrix and B the stored n x k matrix.
"""
import ctypes
import os
import threading

from . import build as _build

# storage datatypes: s, d, c, z; h / k = binary16 real / complex; b / w = bfloat16
# real / complex
DT_CODES = {"s": 0, "d": 1, "c": 2, "z": 3, "h": 4, "k": 5, "b": 6, "w": 7}
TRANS_CODES = {"n": 0, "t": 1, "c": 2, "h": 3}
PREC_CODES = {"s": 0, "d": 1, "c": 2, "h": 3, "b": 4}  # 'c': the precision of C
METHODS = {"auto": 0, "ffma": 1, "tf32x3": 2, "bf16x3": 3, "dmma": 4, "dfma": 5, "tc16": 6}
CASE_NAMES = ["0", "1b", "1a", "2ab", "1c", "2bc", "2ac", "3"]

_i32, _i64, _dbl, _vp, _sz = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_lock = threading.Lock()
_lib = None


class PlanInfo(ctypes.Structure):
    _fields_ = [("domain_case", _i32), ("comp_prec", _i32), ("method", _i32),
                ("whole_op_transposed", _i32), ("Mr", _i64), ("Nr", _i64), ("Kr", _i64),
                ("real_products", _i32), ("flops", _dbl), ("workspace_bytes", _sz), ("k_splits", _i32)]


class Problem(ctypes.Structure):
    """mxg_problem of include/mxgemm.h."""
    _fields_ = [("transa", _i32), ("transb", _i32), ("m", _i64), ("n", _i64), ("k", _i64),
                ("alpha_re", _dbl), ("alpha_im", _dbl), ("beta_re", _dbl), ("beta_im", _dbl),
                ("A", _vp), ("dtA", _i32), ("rsA", _i64), ("csA", _i64),
                ("B", _vp), ("dtB", _i32), ("rsB", _i64), ("csB", _i64),
                ("C", _vp), ("dtC", _i32), ("rsC", _i64), ("csC", _i64), ("comp_prec", _i32)]


class Completion(ctypes.Structure):
    """mxg_completion of include/mxgemm.h."""
    _fields_ = [("id", ctypes.c_uint64), ("status", _i32), ("stream", _i32), ("arrival", _dbl),
                ("admit", _dbl), ("done", _dbl), ("flops", _dbl), ("footprint", _sz)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("bytes_in_flight", _sz), ("peak_bytes_in_flight", _sz),
                ("budget", _sz), ("max_in_flight", _i64), ("queue_len", _i64),
                ("waves", ctypes.c_uint64), ("wave_requests", ctypes.c_uint64)]


class MxgError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {mxg_strerror(status)} (status {status})")


_GEMM_TAIL = [_i32, _i32, _i64, _i64, _i64, _dbl, _dbl, _vp, _i32, _i64, _i64,
              _vp, _i32, _i64, _i64, _dbl, _dbl, _vp, _i32, _i64, _i64, _i32]


def lib():
    """Load the CUDA library, building it in-tree first if it is missing or stale.
    MXG_DEBUG_BOUNDS=1 in the environment loads (and builds) the bounds-checking debug
    build instead."""
    global _lib
    with _lock:
        if _lib is None:
            debug = os.environ.get("MXG_DEBUG_BOUNDS", "") == "1"
            path = _build.LIB_DEBUG if debug else _build.LIB
            if not _build.up_to_date(debug):
                path = _build.build(debug_bounds=debug)
            L = ctypes.CDLL(path)
            L.mxgemm.restype = _i32
            L.mxgemm.argtypes = _GEMM_TAIL
            L.mxgemm_ex.restype = _i32
            L.mxgemm_ex.argtypes = [_vp, _i32] + _GEMM_TAIL
            L.mxg_plan.restype = _i32
            L.mxg_plan.argtypes = [_i32, _i32, _i32, _i64, _i64, _i64, _dbl, _dbl,
                                   _i32, _i64, _i64, _i32, _i64, _i64, _i32, _i64, _i64,
                                   _i32, ctypes.POINTER(PlanInfo)]
            L.mxg_create.restype = _i32
            L.mxg_create.argtypes = [ctypes.POINTER(_vp)]
            L.mxg_destroy.restype = _i32
            L.mxg_destroy.argtypes = [_vp]
            L.mxg_set_split_k.restype = _i32
            L.mxg_set_split_k.argtypes = [_vp, _i32]
            L.mxg_set_cta_pairs.restype = _i32
            L.mxg_set_cta_pairs.argtypes = [_vp, _i32]
            L.mxg_set_stream_k.restype = _i32
            L.mxg_set_stream_k.argtypes = [_vp, _i32]
            L.mxg_set_literal_alpha.restype = _i32
            L.mxg_set_literal_alpha.argtypes = [_vp, _i32]
            L.mxg_set_stream.restype = _i32
            L.mxg_set_stream.argtypes = [_vp, _vp]
            L.mxg_set_workspace.restype = _i32
            L.mxg_set_workspace.argtypes = [_vp, _vp, _sz]
            L.mxg_check_device_error.restype = _i32
            L.mxg_check_device_error.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.mxgemm_noalloc.restype = _i32
            L.mxgemm_noalloc.argtypes = [_vp, _i32] + _GEMM_TAIL
            L.mxgemm_noalloc_check_device_error.restype = _i32
            L.mxgemm_noalloc_check_device_error.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.mxg_group_create.restype = _i32
            L.mxg_group_create.argtypes = [_vp, _i64, ctypes.POINTER(Problem), _i32, _i32, _i32,
                                           ctypes.POINTER(_vp), ctypes.POINTER(_i64)]
            L.mxg_group_run.restype = _i32
            L.mxg_group_run.argtypes = [_vp]
            L.mxg_group_describe.restype = _i32
            L.mxg_group_describe.argtypes = [_vp, ctypes.c_char_p, _sz]
            L.mxg_group_destroy.restype = _i32
            L.mxg_group_destroy.argtypes = [_vp]
            L.mxgemm_grouped.restype = _i32
            L.mxgemm_grouped.argtypes = [_vp, _i64, ctypes.POINTER(Problem)]
            L.mxg_tune_save.restype = _i32
            L.mxg_tune_save.argtypes = [ctypes.c_char_p]
            L.mxg_tune_load.restype = _i32
            L.mxg_tune_load.argtypes = [ctypes.c_char_p]
            L.mxg_server_create.restype = _i32
            L.mxg_server_create.argtypes = [_i32, _sz, _dbl, _i32, _i32, _i32, ctypes.POINTER(_vp)]
            L.mxg_server_submit.restype = _i32
            L.mxg_server_submit.argtypes = [_vp, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_uint64)]
            L.mxg_server_poll.restype = _i32
            L.mxg_server_poll.argtypes = [_vp, ctypes.POINTER(Completion), _i32, ctypes.POINTER(_i32)]
            L.mxg_server_drain.restype = _i32
            L.mxg_server_drain.argtypes = [_vp, _dbl]
            L.mxg_server_get_stats.restype = _i32
            L.mxg_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
            L.mxg_server_now.restype = _dbl
            L.mxg_server_now.argtypes = [_vp]
            L.mxg_server_check_device_error.restype = _i32
            L.mxg_server_check_device_error.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.mxg_server_destroy.restype = _i32
            L.mxg_server_destroy.argtypes = [_vp]
            L.mxg_set_phase_timing.restype = _i32
            L.mxg_set_phase_timing.argtypes = [_vp, _i32]
            L.mxg_phase_times.restype = _i32
            L.mxg_phase_times.argtypes = [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]
            L.mxg_selftest_wait_timeout.restype = _i32
            L.mxg_selftest_wait_timeout.argtypes = [_vp, _dbl]
            L.mxg_strerror.restype = ctypes.c_char_p
            L.mxg_strerror.argtypes = [_i32]
            L.mxg_last_cuda_error.restype = _i32
            L.mxg_version.restype = _i32
            L.mxg_debug_bounds.restype = _i32
            _lib = L
    return _lib


def mxg_strerror(status):
    return lib().mxg_strerror(int(status)).decode()


def dt_of(t):
    """Storage datatype of a tensor. A 3-D float16 / bfloat16 tensor of shape
    (rows, cols, 2) with unit last stride is a complex binary16 / bfloat16 matrix
    (torch has no complex bfloat16)."""
    import torch
    m = {torch.float32: "s", torch.float64: "d", torch.complex64: "c", torch.complex128: "z",
         torch.float16: "h", torch.complex32: "k", torch.bfloat16: "b"}
    if t.dim() == 3 and t.shape[2] == 2 and t.stride(2) == 1 and t.dtype in (torch.float16, torch.bfloat16):
        return "k" if t.dtype == torch.float16 else "w"
    if t.dim() != 2 or t.dtype not in m:
        raise TypeError(f"unsupported matrix {tuple(t.shape)} of {t.dtype}")
    return m[t.dtype]


def _mat(t):
    dt = dt_of(t)
    if t.dim() == 3:
        rs, cs = t.stride(0), t.stride(1)
        if rs % 2 or cs % 2:
            raise ValueError("a (rows, cols, 2) complex matrix needs even row and column strides")
        return ctypes.c_void_p(t.data_ptr()), DT_CODES[dt], int(rs // 2), int(cs // 2)
    rs, cs = t.stride()
    return ctypes.c_void_p(t.data_ptr()), DT_CODES[dt], int(rs), int(cs)


def _dims(transa, transb, A, C):
    m, n = C.shape[0], C.shape[1]
    k = A.shape[0] if transa in ("t", "h") else A.shape[1]
    return int(m), int(n), int(k)


def _scalars(alpha, beta):
    a, b = complex(alpha), complex(beta)
    return a.real, a.imag, b.real, b.imag


def _args(transa, transb, alpha, A, B, beta, C, comp):
    m, n, k = _dims(transa, transb, A, C)
    ar, ai, br, bi = _scalars(alpha, beta)
    pa, da, rsa, csa = _mat(A)
    pb, db, rsb, csb = _mat(B)
    pc, dc, rsc, csc = _mat(C)
    return (TRANS_CODES[transa], TRANS_CODES[transb], m, n, k, ar, ai,
            pa, da, rsa, csa, pb, db, rsb, csb, br, bi, pc, dc, rsc, csc, PREC_CODES[comp])


def mxgemm(transa, transb, alpha, A, B, beta, C, comp="c"):
    """C := beta*C + alpha*op(A)*op(B) through the C entry point ``mxgemm`` (current
    device, legacy default stream, library-owned workspace). Raises MxgError."""
    st = lib().mxgemm(*_args(transa, transb, alpha, A, B, beta, C, comp))
    if st:
        raise MxgError(st, "mxgemm")
    return C


class Handle:
    """An ``mxg_handle``: device, stream and workspace for ``mxgemm_ex``."""

    def __init__(self):
        h = ctypes.c_void_p()
        st = lib().mxg_create(ctypes.byref(h))
        if st:
            raise MxgError(st, "mxg_create")
        self.h = h
        self._ws = None

    def set_split_k(self, mode):
        """Split-K: 0 off, 1 automatic, n >= 2 slices (see mxg_set_split_k)."""
        st = lib().mxg_set_split_k(self.h, int(mode))
        if st:
            raise MxgError(st, "mxg_set_split_k")

    def set_cta_pairs(self, mode):
        """Tensor-core methods on CTA pairs: 0 automatic, 1 always, 2 never."""
        st = lib().mxg_set_cta_pairs(self.h, int(mode))
        if st:
            raise MxgError(st, "mxg_set_cta_pairs")

    def set_stream_k(self, mode):
        """Stream-K tail of the CTA-pair kernel: 0 off, 1 automatic, 2 whenever the last
        wave is partial (see mxg_set_stream_k)."""
        st = lib().mxg_set_stream_k(self.h, int(mode))
        if st:
            raise MxgError(st, "mxg_set_stream_k")

    def set_literal_alpha(self, on):
        """Sec. 7.2's literal reading of a complex alpha for calls on this handle."""
        st = lib().mxg_set_literal_alpha(self.h, 1 if on else 0)
        if st:
            raise MxgError(st, "mxg_set_literal_alpha")

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        st = lib().mxg_set_stream(self.h, ctypes.c_void_p(ptr or 0))
        if st:
            raise MxgError(st, "mxg_set_stream")

    def set_workspace(self, tensor):
        """Caller-owned workspace (a CUDA tensor kept alive by the handle), or None."""
        if tensor is None:
            st = lib().mxg_set_workspace(self.h, None, 0)
        else:
            st = lib().mxg_set_workspace(self.h, ctypes.c_void_p(tensor.data_ptr()),
                                         tensor.numel() * tensor.element_size())
        if st:
            raise MxgError(st, "mxg_set_workspace")
        self._ws = tensor

    def check_device_error(self):
        f = _i32(0)
        st = lib().mxg_check_device_error(self.h, ctypes.byref(f))
        if st:
            raise MxgError(st, "mxg_check_device_error")
        return int(f.value)

    def selftest_wait_timeout(self, seconds=0.05):
        """Status of the bounded-wait self-test (MXG_ETIMEOUT = 5 is the expected one)."""
        return lib().mxg_selftest_wait_timeout(self.h, float(seconds))

    def set_phase_timing(self, on):
        st = lib().mxg_set_phase_timing(self.h, 1 if on else 0)
        if st:
            raise MxgError(st, "mxg_set_phase_timing")

    def phase_times(self):
        """(pack_ms, contraction_ms, contraction_launches) since the last query."""
        a, b, n = _dbl(0), _dbl(0), _i64(0)
        st = lib().mxg_phase_times(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n))
        if st:
            raise MxgError(st, "mxg_phase_times")
        return a.value, b.value, int(n.value)

    def close(self):
        if self.h:
            lib().mxg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles = {}


def _handle_for_current():
    import torch
    dev = torch.cuda.current_device()
    h = _handles.get(dev)
    if h is None:
        h = _handles[dev] = Handle()
    return h


def mxgemm_ex(handle, method, transa, transb, alpha, A, B, beta, C, comp="c", stream=None):
    """C := beta*C + alpha*op(A)*op(B) through ``mxgemm_ex`` with an explicit method.
    handle=None uses a per-device handle bound to torch's current stream (or
    ``stream`` if given)."""
    import torch
    if handle is None:
        handle = _handle_for_current()
        handle.set_stream(stream if stream is not None else torch.cuda.current_stream())
    st = lib().mxgemm_ex(handle.h, METHODS[method] if isinstance(method, str) else int(method),
                         *_args(transa, transb, alpha, A, B, beta, C, comp))
    if st:
        raise MxgError(st, "mxgemm_ex")
    return C


def mxgemm_noalloc(method, transa, transb, alpha, A, B, beta, C, comp="c", stream=None):
    """C := beta*C + alpha*op(A)*op(B) through ``mxgemm_noalloc``: no device allocation;
    the packed operands use the library's fixed scratch array. ``stream`` defaults to
    torch's current stream. Raises MxgError (status 7 when the problem needs more
    scratch than the fixed array holds)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    ptr = getattr(s, "cuda_stream", s)
    st = lib().mxgemm_noalloc(ctypes.c_void_p(ptr or 0),
                              METHODS[method] if isinstance(method, str) else int(method),
                              *_args(transa, transb, alpha, A, B, beta, C, comp))
    if st:
        raise MxgError(st, "mxgemm_noalloc")
    return C


def mxgemm_noalloc_check_device_error(stream=None):
    """Read and clear mxgemm_noalloc's device error word on the current device after
    synchronising ``stream`` (default: torch's current stream); nonzero means a
    device-side wait of some call ran out of its limit."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    ptr = getattr(s, "cuda_stream", s)
    flag = _i32(0)
    st = lib().mxgemm_noalloc_check_device_error(ctypes.c_void_p(ptr or 0), ctypes.byref(flag))
    if st:
        raise MxgError(st, "mxgemm_noalloc_check_device_error")
    return int(flag.value)


def make_problems(items):
    """items: iterable of (transa, transb, alpha, A, B, beta, C, comp) on torch tensors.
    Returns a ctypes array of mxg_problem."""
    items = list(items)
    arr = (Problem * max(len(items), 1))()
    for i, (ta, tb, alpha, A, B, beta, C, comp) in enumerate(items):
        v = _args(ta, tb, alpha, A, B, beta, C, comp)
        p = arr[i]
        (p.transa, p.transb, p.m, p.n, p.k, p.alpha_re, p.alpha_im, p.A, p.dtA, p.rsA, p.csA,
         p.B, p.dtB, p.rsB, p.csB, p.beta_re, p.beta_im, p.C, p.dtC, p.rsC, p.csC, p.comp_prec) = \
            (v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7].value or 0, v[8], v[9], v[10],
             v[11].value or 0, v[12], v[13], v[14], v[15], v[16], v[17].value or 0, v[18], v[19], v[20], v[21])
    return arr, len(items)


class Group:
    """An mxg_group: a grouped persistent launch over many problems (see
    mxg_group_create). ``tune``: autotune kernels and schedules per bucket; ``graph``:
    capture the run in a CUDA graph."""

    def __init__(self, items, handle=None, method_s="auto", method_d="auto", tune=True, graph=True, stream=None):
        import torch
        if handle is None:
            handle = Handle()
            handle.set_stream(stream if stream is not None else torch.cuda.current_stream())
        self.handle = handle
        self._arr, n = make_problems(items)
        g = ctypes.c_void_p()
        bad = _i64(-1)
        flags = (1 if tune else 0) | (2 if graph else 0)
        st = lib().mxg_group_create(handle.h, n, self._arr, METHODS[method_s], METHODS[method_d], flags,
                                    ctypes.byref(g), ctypes.byref(bad))
        if st:
            raise MxgError(st, f"mxg_group_create (problem {bad.value})")
        self.g = g

    def run(self):
        st = lib().mxg_group_run(self.g)
        if st:
            raise MxgError(st, "mxg_group_run")

    def describe(self):
        import json
        buf = ctypes.create_string_buffer(8192)
        lib().mxg_group_describe(self.g, buf, 8192)
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "g", None):
            lib().mxg_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """An mxg_server: continuous-batching request server (see mxg_server_create).
    ``fifo=True`` gives the serial baseline (one stream, submission order)."""

    def __init__(self, n_streams=4, hbm_budget_bytes=16 << 30, small_flops=5e7, method_s="auto",
                 method_d="auto", fifo=False):
        s = ctypes.c_void_p()
        st = lib().mxg_server_create(int(n_streams), int(hbm_budget_bytes), float(small_flops), METHODS[method_s],
                                     METHODS[method_d], 1 if fifo else 0, ctypes.byref(s))
        if st:
            raise MxgError(st, "mxg_server_create")
        self.s = s
        self._keep = {}

    def submit(self, item, keep=None):
        """item: (transa, transb, alpha, A, B, beta, C, comp) on device tensors. ``keep``
        (optional) is held until the request completes (e.g. the tensors)."""
        arr, _ = make_problems([item])
        rid = ctypes.c_uint64(0)
        st = lib().mxg_server_submit(self.s, arr, ctypes.byref(rid))
        if st:
            raise MxgError(st, "mxg_server_submit")
        if keep is not None:
            self._keep[rid.value] = keep
        return rid.value

    def poll(self, max_items=4096):
        buf = (Completion * max_items)()
        n = _i32(0)
        lib().mxg_server_poll(self.s, buf, max_items, ctypes.byref(n))
        out = []
        for i in range(n.value):
            c = buf[i]
            self._keep.pop(c.id, None)
            out.append({"id": c.id, "status": c.status, "stream": c.stream, "arrival": c.arrival,
                        "admit": c.admit, "done": c.done, "flops": c.flops, "footprint": c.footprint})
        return out

    def drain(self, timeout_s=600.0):
        st = lib().mxg_server_drain(self.s, float(timeout_s))
        if st:
            raise MxgError(st, "mxg_server_drain")

    def stats(self):
        st = ServerStats()
        lib().mxg_server_get_stats(self.s, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def now(self):
        return lib().mxg_server_now(self.s)

    def check_device_error(self):
        """The server's device error word (nonzero: a device-side wait of a served
        request ran out), cleared by the read."""
        flag = _i32(0)
        st = lib().mxg_server_check_device_error(self.s, ctypes.byref(flag))
        if st:
            raise MxgError(st, "mxg_server_check_device_error")
        return flag.value

    def close(self):
        if getattr(self, "s", None):
            lib().mxg_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mxgemm_grouped(items, handle=None, stream=None):
    """One-shot grouped call (no tuning, no graph); synchronises the stream."""
    import torch
    if handle is None:
        handle = _handle_for_current()
        handle.set_stream(stream if stream is not None else torch.cuda.current_stream())
    arr, n = make_problems(items)
    st = lib().mxgemm_grouped(handle.h, n, arr)
    if st:
        raise MxgError(st, "mxgemm_grouped")


def mxg_tune_save(path):
    return lib().mxg_tune_save(path.encode())


def mxg_tune_load(path):
    return lib().mxg_tune_load(path.encode())


def mxg_plan(combo_or_dts, m, n, k, transa="n", transb="n", alpha=1.0, method="auto",
             strides=None, comp=None):
    """Host-only planning (no CUDA call): returns PlanInfo or raises MxgError.

    ``combo_or_dts`` is a label 'cabx' (C, A, B datatypes, computation precision
    's'/'d', or 'c' = precision of C). ``strides`` = ((rsA, csA), (rsB, csB),
    (rsC, csC)); default column-major."""
    dc, da, db = combo_or_dts[0], combo_or_dts[1], combo_or_dts[2]
    x = comp or (combo_or_dts[3] if len(combo_or_dts) > 3 else "c")
    if strides is None:
        a_rows = k if transa in ("t", "h") else m
        b_rows = n if transb in ("t", "h") else k
        strides = ((1, max(a_rows, 1)), (1, max(b_rows, 1)), (1, max(m, 1)))
    (rsa, csa), (rsb, csb), (rsc, csc) = strides
    a = complex(alpha)
    info = PlanInfo()
    st = lib().mxg_plan(METHODS[method] if isinstance(method, str) else int(method),
                        TRANS_CODES[transa], TRANS_CODES[transb], m, n, k, a.real, a.imag,
                        DT_CODES[da], rsa, csa, DT_CODES[db], rsb, csb, DT_CODES[dc], rsc, csc,
                        PREC_CODES[x], ctypes.byref(info))
    if st:
        raise MxgError(st, "mxg_plan")
    return info
