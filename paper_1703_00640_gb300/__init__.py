"""Python binding of libtruncmul (include/truncmul.h): argument marshalling only.

Every step of a product runs in the library's CUDA kernels. Operands and
results are little-endian uint64 limb arrays; torch tensors (any 8-byte dtype,
contiguous, on the current CUDA device) supply device memory and streams. The
library must be built (``build()`` or ``__graft_entry__.build()``); importing
fails loudly when it is missing, and there is no CPU fallback.
"""
import ctypes
import os

from . import build as _build

KIND = {"full": 0, "lo": 1, "hi": 2}
STATUS = {0: "TM_OK", 1: "TM_UNCERTIFIED", -1: "TM_EINVAL", -2: "TM_ENOMEM", -3: "TM_EPRECISION", -4: "TM_ETIMEOUT",
          -5: "TM_ECUDA", -6: "TM_ERANGE", -7: "TM_EALIAS"}
TM_OK, TM_EINVAL, TM_ENOMEM, TM_EPRECISION, TM_ETIMEOUT, TM_ECUDA, TM_ERANGE, TM_EALIAS = (
    0, -1, -2, -3, -4, -5, -6, -7)
TM_UNCERTIFIED = 1


class Report(ctypes.Structure):
    """tm_report (include/truncmul.h)."""
    _fields_ = [("kind", ctypes.c_int32), ("status", ctypes.c_int32), ("b", ctypes.c_uint32),
                ("N", ctypes.c_uint32), ("n_digits", ctypes.c_uint32),
                ("lam_fwd", ctypes.c_uint32), ("lam_bwd", ctypes.c_uint32),
                ("fft_passes", ctypes.c_uint32), ("fwd_streams", ctypes.c_uint32),
                ("margin", ctypes.c_double),
                ("e_max", ctypes.c_double), ("workspace_bytes", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Desc(ctypes.Structure):
    """tm_desc (include/truncmul.h)."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_bits", ctypes.c_uint64),
                ("out", ctypes.c_void_p), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    """tm_completion (include/truncmul.h)."""
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("b", ctypes.c_uint32), ("N", ctypes.c_uint32), ("limit", ctypes.c_double)]


class PlanTune(ctypes.Structure):
    _fields_ = [("b", ctypes.c_uint32), ("N", ctypes.c_uint32), ("candidates", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("ms_default", ctypes.c_double),
                ("ms_best", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Tune(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("points", ctypes.c_int32),
                ("split", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("npass", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class TruncMulError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({strerror(code)})")
        self.code = code


NPHASES = 6
PHASES = ["fwd_map", "fwd_fft", "twist_pointwise", "inv_fft", "back_round", "carry"]
STATIC_MAX_BITS = 65536
EXPORTS = ["tm_mul", "tm_mul_params", "tm_mul_adaptive", "tm_mul_full", "tm_mul_lo", "tm_mul_hi", "tm_mul_host", "tm_mul_events",
           "tm_mul_static", "tm_batch_create", "tm_batch_launch", "tm_batch_status",
           "tm_batch_destroy", "tm_mul_batch", "tm_server_create", "tm_server_submit",
           "tm_server_progress", "tm_server_pending", "tm_server_destroy",
           "tm_autotune", "tm_set_layout", "tm_autotune_plan", "tm_plan_set", "tm_operand_create", "tm_mul_operand", "tm_operand_destroy",
           "tm_reciprocal",
           "tm_barrett_create", "tm_barrett_divrem", "tm_barrett_reciprocal",
           "tm_barrett_destroy", "tm_coeffs",
           "tm_plan_query", "tm_stream_status", "tm_release", "tm_strerror", "tm_probe_dfma", "tm_table_values", "tm_convolution", "tm_set_fused"]

_lib = None


def library_path() -> str:
    return _build.OUT


def load(path: str = None):
    """Loads libtruncmul.so (no build; raises OSError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: run paper_1703_00640_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    R = ctypes.POINTER(Report)
    for name in ("tm_mul_full", "tm_mul_lo", "tm_mul_hi"):
        getattr(lib, name).argtypes = [P, P, P, ctypes.c_uint64, P, R]
        getattr(lib, name).restype = ctypes.c_int
    lib.tm_mul.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P, R]
    lib.tm_mul_params.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64,
                                  ctypes.POINTER(Params), P, R]
    lib.tm_mul_params.restype = ctypes.c_int
    lib.tm_mul_adaptive.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P, R]
    lib.tm_mul_adaptive.restype = ctypes.c_int
    lib.tm_mul_host.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P, R]
    lib.tm_mul_static.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P, R]
    lib.tm_coeffs.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P, R]
    lib.tm_mul_events.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, P,
                                  ctypes.POINTER(ctypes.c_void_p), R]
    lib.tm_plan_query.argtypes = [ctypes.c_int, ctypes.c_uint64, R]
    lib.tm_probe_dfma.argtypes = [ctypes.c_int, P, ctypes.POINTER(ctypes.c_double)]
    lib.tm_probe_dfma.restype = ctypes.c_int
    lib.tm_table_values.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, P]
    lib.tm_table_values.restype = ctypes.c_int
    lib.tm_convolution.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.POINTER(ctypes.c_double)]
    lib.tm_convolution.restype = ctypes.c_int
    lib.tm_set_fused.argtypes = [ctypes.c_int]
    lib.tm_set_fused.restype = ctypes.c_int
    D = ctypes.POINTER(Desc)
    lib.tm_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), D, ctypes.c_uint32, P]
    lib.tm_batch_launch.argtypes = [P, P]
    lib.tm_batch_status.argtypes = [P, P, R]
    lib.tm_batch_destroy.argtypes = [P]
    lib.tm_mul_batch.argtypes = [D, ctypes.c_uint32, P, R]
    lib.tm_server_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64, ctypes.c_int]
    lib.tm_server_create.restype = ctypes.c_int
    lib.tm_server_submit.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_uint64]
    lib.tm_server_submit.restype = ctypes.c_int64
    lib.tm_server_progress.argtypes = [P, ctypes.POINTER(Completion), ctypes.c_int]
    lib.tm_server_progress.restype = ctypes.c_int
    lib.tm_server_pending.argtypes = [P]
    lib.tm_server_pending.restype = ctypes.c_int
    lib.tm_server_destroy.argtypes = [P]
    lib.tm_server_destroy.restype = ctypes.c_int
    lib.tm_operand_create.argtypes = [ctypes.c_int, ctypes.c_uint64, P, P,
                                      ctypes.POINTER(ctypes.c_void_p)]
    lib.tm_mul_operand.argtypes = [P, P, P, P, R]
    lib.tm_operand_destroy.argtypes = [P]
    lib.tm_autotune.argtypes = [ctypes.c_int, ctypes.c_uint64, P, ctypes.POINTER(Tune)]
    lib.tm_autotune.restype = ctypes.c_int
    lib.tm_set_layout.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(Tune)]
    lib.tm_set_layout.restype = ctypes.c_int
    lib.tm_autotune_plan.argtypes = [ctypes.c_int, ctypes.c_uint64, P, ctypes.POINTER(PlanTune)]
    lib.tm_autotune_plan.restype = ctypes.c_int
    lib.tm_plan_set.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.tm_plan_set.restype = ctypes.c_int
    lib.tm_reciprocal.argtypes = [P, P, ctypes.c_uint64, P]
    lib.tm_barrett_create.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.tm_barrett_divrem.argtypes = [P, P, P, P, P, R]
    lib.tm_barrett_reciprocal.argtypes = [P, P, P]
    lib.tm_barrett_destroy.argtypes = [P]
    for name in ("tm_operand_create", "tm_mul_operand", "tm_operand_destroy", "tm_reciprocal",
                 "tm_barrett_create", "tm_barrett_divrem", "tm_barrett_reciprocal",
                 "tm_barrett_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    lib.tm_stream_status.argtypes = [P, R]
    lib.tm_release.argtypes = []
    lib.tm_strerror.argtypes = [ctypes.c_int]
    lib.tm_strerror.restype = ctypes.c_char_p
    for name in ("tm_batch_create", "tm_batch_launch", "tm_batch_status", "tm_batch_destroy",
                 "tm_mul_batch"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("tm_mul", "tm_mul_host", "tm_mul_events", "tm_mul_static", "tm_coeffs", "tm_plan_query", "tm_stream_status",
                 "tm_release"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def build(force: bool = False) -> str:
    return _build.build(force=force)


def strerror(code: int) -> str:
    return load().tm_strerror(int(code)).decode()


def _kind(kind) -> int:
    return KIND[kind] if isinstance(kind, str) else int(kind)


def out_limbs(kind, n_bits: int) -> int:
    k = _kind(kind)
    nl = (n_bits + 63) // 64
    return 2 * nl if k == 0 else (nl if k == 1 else n_bits // 64 + 1)


def _ptr(t):
    if t is None:
        return None
    assert t.is_contiguous() and t.element_size() == 8, "limb tensors must be contiguous 8-byte"
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def plan(kind, n_bits: int) -> dict:
    """tm_plan_query: the library's plan for (kind, n) (host only, no GPU needed)."""
    rep = Report()
    rc = load().tm_plan_query(_kind(kind), int(n_bits), ctypes.byref(rep))
    if rc:
        raise TruncMulError(rc, "tm_plan_query")
    return rep.as_dict()


def mul(kind, u, v, n_bits: int, out=None, stream=None, report: bool = True, check: bool = True):
    """tm_mul on device tensors. Returns (out, report dict or None)."""
    import torch
    k = _kind(kind)
    if out is None:
        out = torch.empty(out_limbs(k, n_bits), dtype=torch.int64, device=u.device)
    rep = Report() if report else None
    rc = load().tm_mul(k, _ptr(out), _ptr(u), _ptr(v), int(n_bits), _stream_ptr(stream),
                       ctypes.byref(rep) if rep is not None else None)
    if check and rc:
        raise TruncMulError(rc, "tm_mul")
    return out, (rep.as_dict() if rep is not None else None)


def mul_params(kind, u, v, n_bits: int, b: int, N: int, limit: float = 0.0, out=None,
               stream=None, report: bool = True, check: bool = True):
    """tm_mul_params: the product with the caller's digit size b and transform
    length N (the paper's empirical parameters). Returns (out, report dict or None);
    report["status"] is TM_UNCERTIFIED when (b, N) is outside the worst-case bound."""
    import torch
    k = _kind(kind)
    if out is None:
        out = torch.empty(out_limbs(k, n_bits), dtype=torch.int64, device=u.device)
    prm = Params(b=int(b), N=int(N), limit=float(limit))
    rep = Report() if report else None
    rc = load().tm_mul_params(k, _ptr(out), _ptr(u), _ptr(v), int(n_bits), ctypes.byref(prm),
                              _stream_ptr(stream),
                              ctypes.byref(rep) if rep is not None else None)
    if check and rc < 0:             # TM_UNCERTIFIED (> 0) is a result, not an error
        raise TruncMulError(rc, "tm_mul_params")
    return out, (rep.as_dict() if rep is not None else None)


def mul_adaptive(kind, u, v, n_bits: int, out=None, stream=None, report: bool = True,
                 check: bool = True):
    """tm_mul_adaptive: the product with the digit size chosen from the operands'
    measured digit norms. Returns (out, report dict or None)."""
    import torch
    k = _kind(kind)
    if out is None:
        out = torch.empty(out_limbs(k, n_bits), dtype=torch.int64, device=u.device)
    rep = Report() if report else None
    rc = load().tm_mul_adaptive(k, _ptr(out), _ptr(u), _ptr(v), int(n_bits),
                                _stream_ptr(stream), ctypes.byref(rep) if rep is not None else None)
    if check and rc:
        raise TruncMulError(rc, "tm_mul_adaptive")
    return out, (rep.as_dict() if rep is not None else None)


def mul_events(kind, u, v, n_bits: int, events, out=None, stream=None):
    """tm_mul_events: enqueue one product recording torch.cuda.Event objects
    (NPHASES + 1 of them, enable_timing=True) between its phases. Asynchronous."""
    import torch
    k = _kind(kind)
    assert len(events) == NPHASES + 1
    if out is None:
        out = torch.empty(out_limbs(k, n_bits), dtype=torch.int64, device=u.device)
    arr = (ctypes.c_void_p * (NPHASES + 1))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    rc = load().tm_mul_events(k, _ptr(out), _ptr(u), _ptr(v), int(n_bits), _stream_ptr(stream),
                              arr, None)
    if rc:
        raise TruncMulError(rc, "tm_mul_events")
    return out


FUSED_AUTO, FUSED_NEVER, FUSED_ALWAYS = 0, 1, 2


def set_fused(mode: int) -> None:
    """tm_set_fused: 0 automatic, 1 per-phase launches only, 2 one cooperative
    launch per product wherever the layout allows."""
    rc = load().tm_set_fused(int(mode))
    if rc:
        raise TruncMulError(rc, "tm_set_fused")


def convolution(x, y, out=None, stream=None):
    """tm_convolution: the FP64 cyclic convolution of the real float64 device
    tensors x and y (length N). Returns (out, eta) with |out_k - (x*y)_k| <=
    eta ||x||_2 ||y||_2."""
    import torch
    if out is None:
        out = torch.empty_like(x)
    eta = ctypes.c_double()
    rc = load().tm_convolution(_ptr(out), _ptr(x), _ptr(y), int(x.numel()), _stream_ptr(stream),
                               ctypes.byref(eta))
    if rc:
        raise TruncMulError(rc, "tm_convolution")
    return out, eta.value


def table_values(which: int, length: int, count: int):
    """tm_table_values: the FFT kernels' twiddle table `which` (0 twiddles, 1
    tangent-form radix-4 records, 2 twist coefficients, 3 four-step twiddles of
    Mp = length in the output order of count sequences) as a float64 numpy array."""
    import numpy as np
    import torch
    per = 4 if which == 1 else 2
    entries = length if which == 3 else count
    out = torch.empty(per * max(entries, 0), dtype=torch.float64, device="cuda")
    rc = load().tm_table_values(int(which), int(length), int(count), _ptr(out), _stream_ptr(None))
    if rc:
        raise TruncMulError(rc, "tm_table_values")
    return out.cpu().numpy().astype(np.float64)


def probe_dfma(iters: int, stream=None) -> float:
    """tm_probe_dfma: enqueues the FP64 FMA issue-rate probe on `stream` and
    returns the flops it performs (time it with events on the same stream)."""
    fl = ctypes.c_double()
    rc = load().tm_probe_dfma(int(iters), _stream_ptr(stream), ctypes.byref(fl))
    if rc:
        raise TruncMulError(rc, "tm_probe_dfma")
    return fl.value


def mul_static(kind, u, v, n_bits: int, out, stream=None, report: bool = True):
    """tm_mul_static: the product with no device allocation (n_bits <= STATIC_MAX_BITS).
    `out` must be supplied by the caller. Returns (status code, report dict or None)."""
    rep = Report() if report else None
    rc = load().tm_mul_static(_kind(kind), _ptr(out), _ptr(u), _ptr(v), int(n_bits),
                              _stream_ptr(stream), ctypes.byref(rep) if rep is not None else None)
    return rc, (rep.as_dict() if rep is not None else None)


def _descs(items):
    arr = (Desc * len(items))()
    for i, (kind, n_bits, out, u, v) in enumerate(items):
        arr[i].kind = _kind(kind)
        arr[i].reserved = 0
        arr[i].n_bits = int(n_bits)
        arr[i].out = out.data_ptr()
        arr[i].u = u.data_ptr()
        arr[i].v = v.data_ptr()
    return arr


class Batch:
    """tm_batch: many products recorded once as a CUDA graph, relaunched at will.
    items: list of (kind, n_bits, out, u, v) with device tensors (kept alive here)."""

    def __init__(self, items, stream=None):
        self._items = list(items)          # keep the tensors alive
        self._h = ctypes.c_void_p()
        arr = _descs(self._items)
        rc = load().tm_batch_create(ctypes.byref(self._h), arr, len(arr), _stream_ptr(stream))
        if rc:
            self._h = None
            raise TruncMulError(rc, "tm_batch_create")

    def launch(self, stream=None):
        rc = load().tm_batch_launch(self._h, _stream_ptr(stream))
        if rc:
            raise TruncMulError(rc, "tm_batch_launch")

    def status(self, stream=None) -> dict:
        rep = Report()
        rc = load().tm_batch_status(self._h, _stream_ptr(stream), ctypes.byref(rep))
        d = rep.as_dict()
        d["rc"] = rc
        return d

    def close(self):
        if self._h:
            load().tm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mul_batch(items, stream=None) -> dict:
    """tm_mul_batch (one shot). items as for Batch. Returns the report."""
    arr = _descs(items)
    rep = Report()
    rc = load().tm_mul_batch(arr, len(arr), _stream_ptr(stream), ctypes.byref(rep))
    if rc:
        raise TruncMulError(rc, "tm_mul_batch")
    return rep.as_dict()


class Operand:
    """tm_operand: the forward transform of a fixed operand v, kept on the device.
    mul(u) then computes the product of this kind and n_bits with two transforms
    instead of three; results are bit-identical to mul(kind, u, v, n_bits)."""

    def __init__(self, kind, v, n_bits: int, stream=None):
        self.kind = _kind(kind)
        self.n_bits = int(n_bits)
        self.device = v.device
        self._h = ctypes.c_void_p()
        rc = load().tm_operand_create(self.kind, self.n_bits, _ptr(v), _stream_ptr(stream),
                                      ctypes.byref(self._h))
        if rc:
            self._h = None
            raise TruncMulError(rc, "tm_operand_create")

    def mul(self, u, out=None, stream=None, report: bool = True, check: bool = True):
        """tm_mul_operand. Returns (out, report dict or None)."""
        import torch
        if out is None:
            out = torch.empty(out_limbs(self.kind, self.n_bits), dtype=torch.int64,
                              device=u.device)
        rep = Report() if report else None
        rc = load().tm_mul_operand(_ptr(out), _ptr(u), self._h, _stream_ptr(stream),
                                   ctypes.byref(rep) if rep is not None else None)
        if check and rc:
            raise TruncMulError(rc, "tm_mul_operand")
        return out, (rep.as_dict() if rep is not None else None)

    def close(self):
        if self._h:
            load().tm_operand_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(kind, n_bits: int, stream=None) -> dict:
    """tm_autotune: time the FFT layouts for (kind, n) and keep the fastest."""
    t = Tune()
    rc = load().tm_autotune(_kind(kind), int(n_bits), _stream_ptr(stream), ctypes.byref(t))
    if rc:
        raise TruncMulError(rc, "tm_autotune")
    return t.as_dict()


def autotune_plan(kind, n_bits: int, stream=None) -> dict:
    """tm_autotune_plan: time the certified plans (b, N) of (kind, n) near the
    planner's and keep the fastest for later calls."""
    t = PlanTune()
    rc = load().tm_autotune_plan(_kind(kind), int(n_bits), _stream_ptr(stream), ctypes.byref(t))
    if rc:
        raise TruncMulError(rc, "tm_autotune_plan")
    return t.as_dict()


def plan_set(kind, n_bits: int, b: int = 0, N: int = 0):
    """tm_plan_set: make the certified (b, N) the plan of (kind, n); b = N = 0
    restores the planner's choice."""
    rc = load().tm_plan_set(_kind(kind), int(n_bits), int(b), int(N))
    if rc:
        raise TruncMulError(rc, "tm_plan_set")


def set_layout(kind, n_bits: int, points: int = 1024, split: int = 0, passes: int = 0):
    """tm_set_layout: make a layout (as autotune reports it) the FFT pass layout of
    later plans with the transform length of (kind, n); the defaults restore the
    default layout."""
    t = Tune(points=points, split=split, passes=passes)
    rc = load().tm_set_layout(_kind(kind), int(n_bits), ctypes.byref(t))
    if rc:
        raise TruncMulError(rc, "tm_set_layout")


def reciprocal(m, k_bits: int, out=None, stream=None):
    """tm_reciprocal: floor((2^(2k) - 1) / m) for a k-bit m (bit k-1 set), as a
    device tensor of ceil((k+1)/64) limbs. Waits for the stream."""
    import torch
    if out is None:
        out = torch.empty((k_bits + 1 + 63) // 64, dtype=torch.int64, device=m.device)
    rc = load().tm_reciprocal(_ptr(out), _ptr(m), int(k_bits), _stream_ptr(stream))
    if rc:
        raise TruncMulError(rc, "tm_reciprocal")
    return out


class Barrett:
    """tm_barrett: division by a fixed k-bit divisor m (bit k-1 set) with its
    reciprocal and the kept transforms of the reciprocal and of m."""

    def __init__(self, m, k_bits: int, stream=None):
        self.k_bits = int(k_bits)
        self._h = ctypes.c_void_p()
        rc = load().tm_barrett_create(_ptr(m), self.k_bits, _stream_ptr(stream),
                                      ctypes.byref(self._h))
        if rc:
            self._h = None
            raise TruncMulError(rc, "tm_barrett_create")

    def divrem(self, x, q=None, r=None, stream=None, report: bool = True, want=("q", "r")):
        """q = floor(x / m), r = x mod m for x < 2^(2k) (ceil(2k/64) limbs).
        Returns (q or None, r or None, report dict or None)."""
        import torch
        k = self.k_bits
        if q is None and "q" in want:
            q = torch.empty((k + 1 + 63) // 64, dtype=torch.int64, device=x.device)
        if r is None and "r" in want:
            r = torch.empty((k + 63) // 64, dtype=torch.int64, device=x.device)
        rep = Report() if report else None
        rc = load().tm_barrett_divrem(self._h, _ptr(q), _ptr(r), _ptr(x), _stream_ptr(stream),
                                      ctypes.byref(rep) if rep is not None else None)
        if rc:
            raise TruncMulError(rc, "tm_barrett_divrem")
        return q, r, (rep.as_dict() if rep is not None else None)

    def reciprocal(self, stream=None):
        import torch
        out = torch.empty((self.k_bits + 1 + 63) // 64, dtype=torch.int64, device="cuda")
        rc = load().tm_barrett_reciprocal(self._h, _ptr(out), _stream_ptr(stream))
        if rc:
            raise TruncMulError(rc, "tm_barrett_reciprocal")
        return out

    def close(self):
        if self._h:
            load().tm_barrett_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """tm_server: queued requests with continuous batching under a memory budget.
    submit() queues (device tensors must stay alive until completion);
    progress() retires finished work and admits queued requests, never blocking."""

    def __init__(self, budget_bytes: int, slots: int = 4):
        self._h = ctypes.c_void_p()
        rc = load().tm_server_create(ctypes.byref(self._h), int(budget_bytes), int(slots))
        if rc:
            self._h = None
            raise TruncMulError(rc, "tm_server_create")
        self._buf = (Completion * 4096)()
        self._keep = {}

    def submit(self, kind, out, u, v, n_bits: int) -> int:
        t = load().tm_server_submit(self._h, _kind(kind), _ptr(out), _ptr(u), _ptr(v), int(n_bits))
        if t < 0:
            raise TruncMulError(int(t), "tm_server_submit")
        self._keep[t] = (out, u, v)
        return t

    def progress(self):
        rc = load().tm_server_progress(self._h, self._buf, len(self._buf))
        if rc < 0:
            raise TruncMulError(rc, "tm_server_progress")
        done = [(self._buf[i].ticket, self._buf[i].status) for i in range(rc)]
        for t, _ in done:
            self._keep.pop(t, None)
        return done

    def pending(self) -> int:
        return load().tm_server_pending(self._h)

    def close(self):
        if self._h:
            load().tm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mul_lo(u, v, n_bits, **kw):
    return mul("lo", u, v, n_bits, **kw)


def mul_hi(u, v, n_bits, **kw):
    return mul("hi", u, v, n_bits, **kw)


def mul_full(u, v, n_bits, **kw):
    return mul("full", u, v, n_bits, **kw)


def mul_host(kind, u, v, n_bits: int, out=None, stream=None):
    """tm_mul_host on host (CPU) tensors or numpy arrays; returns (out, report)."""
    import numpy as np
    k = _kind(kind)
    if out is None:
        out = np.zeros(out_limbs(k, n_bits), dtype=np.uint64)

    def p(a):
        if hasattr(a, "data_ptr"):
            assert a.is_contiguous() and a.element_size() == 8
            return ctypes.c_void_p(a.data_ptr())
        assert a.dtype.itemsize == 8 and a.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(a.ctypes.data)
    rep = Report()
    rc = load().tm_mul_host(k, p(out), p(u), p(v), int(n_bits), _stream_ptr(stream),
                            ctypes.byref(rep))
    if rc:
        raise TruncMulError(rc, "tm_mul_host")
    return out, rep.as_dict()


def coeffs(kind, u, v, n_bits: int, stream=None):
    """tm_coeffs: the rounded coefficients c_i (int64 device tensor) and the report."""
    import torch
    k = _kind(kind)
    pl = plan(k, n_bits)
    count = pl["N"] + 1 if k == 2 else pl["N"]
    c = torch.empty(count, dtype=torch.int64, device=u.device)
    rep = Report()
    rc = load().tm_coeffs(k, _ptr(c), _ptr(u), _ptr(v), int(n_bits), _stream_ptr(stream),
                          ctypes.byref(rep))
    if rc and rc != TM_EPRECISION:
        raise TruncMulError(rc, "tm_coeffs")
    return c, rep.as_dict()


def stream_status(stream=None) -> dict:
    rep = Report()
    rc = load().tm_stream_status(_stream_ptr(stream), ctypes.byref(rep))
    d = rep.as_dict()
    d["rc"] = rc
    return d


def release():
    rc = load().tm_release()
    if rc:
        raise TruncMulError(rc, "tm_release")
