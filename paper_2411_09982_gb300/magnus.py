"""Thin ctypes binding of libmagnus.so (the C ABI declared in include/magnus.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Functions keep the C names; tensors are passed as device pointers
(`torch.Tensor.data_ptr()`), complex matrices as complex128 tensors (the
interleaved (re, im) FP64 layout of the ABI).  There is no CPU fallback: if
the library cannot be loaded or no sm_103a device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmagnus.so")

MG_OK = 0
MG_EINVAL = -1
MG_ENOMEM = -2
MG_ECUDA = -3
MG_ENONFINITE = -4
MG_ENOTHERM = -5
MG_ETIMEOUT = -6
MG_EAGAIN = -7
MG_EUNSUPPORTED = -8

MG_PREC_FP64 = 0
MG_PREC_SPLIT = 1
MG_PREC_AUTO = 2
MG_TAYLOR_AUTO = 0
MG_TAYLOR_PS = 1
MG_OUT_STATE = 0
MG_OUT_PROPAGATOR = 1
MG_OUT_TRAJECTORY = 2
MG_FLAG_HOST_PTRS = 1
MG_FLAG_CHECK_HERMITIAN = 2
MG_FLAG_NO_TRACE_SHIFT = 4
MG_FLAG_STATE_ACTION = 8


class MagnusError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {code} ({detail})")


class mg_report(ctypes.Structure):
    _fields_ = [
        ("intervals", ctypes.c_int32),
        ("taylor_degree", ctypes.c_int32),
        ("max_squarings", ctypes.c_int32),
        ("min_squarings", ctypes.c_int32),
        ("max_norm1", ctypes.c_double),
        ("unitarity_defect", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("matrix_products", ctypes.c_int64),
        ("sparse_matvecs", ctypes.c_int64),
        ("sparse_nnz", ctypes.c_int64),
        ("action_ctas", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mg_job(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("K", ctypes.c_int),
        ("H0", ctypes.c_void_p), ("Hk", ctypes.c_void_p),
        ("N", ctypes.c_int), ("P", ctypes.c_int),
        ("t0", ctypes.c_double), ("dt", ctypes.c_double),
        ("w", ctypes.c_void_p), ("samples", ctypes.c_void_p),
        ("output", ctypes.c_int), ("input", ctypes.c_void_p), ("out", ctypes.c_void_p),
        ("precision", ctypes.c_int), ("slices", ctypes.c_int), ("flags", ctypes.c_int),
        ("tolerance", ctypes.c_double),
    ]


class mg_tune_entry(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("slices", ctypes.c_int32), ("taylor", ctypes.c_int32),
                ("action", ctypes.c_int32), ("error", ctypes.c_double), ("us_per_interval", ctypes.c_double),
                ("taylor_target", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mg_job_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("intervals", ctypes.c_int64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); mirrors include/magnus.h
SIGNATURES = {
    "mg_ctx_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "mg_ctx_destroy": (_I, [_P]),
    "mg_ctx_set_workspace_limit": (_I, [_P, ctypes.c_size_t]),
    "mg_quadrature_nodes": (_I, [_I, _P, _P]),
    "mg_taylor_choice": (_I, [_D, _I, _I, _I, _P, _P, _P]),
    "mg_split_digits": (_I, [_I, _I, _P, _P]),
    "mg_second_order_weights": (_I, [_I, _P]),
    "mg_csr_pattern": (_I, [_I, _I, _P, _P, _P, _P, _P, _P]),
    "mg_plan_create": (_I, [_P, ctypes.POINTER(_P), _I, _I, _P, _P, _I, _I, _I]),
    "mg_plan_destroy": (_I, [_P]),
    "mg_plan_set_magnus_order": (_I, [_P, _I]),
    "mg_set_controls": (_I, [_P, _I, _I, _D, _D, _P, _P, _I]),
    "mg_evolve": (_I, [_P, _I, _P, _P, _I, _I, ctypes.POINTER(mg_report)]),
    "mg_evolve_batch": (_I, [_P, _I, _P, _P, _P, _P, _I, _I, _P]),
    "mg_coefficients": (_I, [_P, _I, _I, _I, _D, _P, _P, _P]),
    "mg_build_omega": (_I, [_P, _I, _I, _I, _D, _P, _P, _P, _P, _P, _P]),
    "mg_expm": (_I, [_P, _I, _I, _P, _P, _I, _I, _P]),
    "mg_cgemm": (_I, [_P, _I, _I, _P, _P, _P, _I, _I]),
    "mg_propagate": (_I, [_P, _I, _I, _P, _I, _P, _P, _I, _I, _I]),
    "mg_ctx_enable_gemm_timing": (_I, [_P, _I]),
    "mg_ctx_set_wait_limit": (_I, [_P, _D, _I]),
    "mg_ctx_set_stage_k": (_I, [_P, _I]),
    "mg_ctx_set_digit_pairs": (_I, [_P, _I]),
    "mg_ctx_set_cta_pairs": (_I, [_P, _I]),
    "mg_ctx_set_structure": (_I, [_P, _I]),
    "mg_ctx_gemm_stats": (_I, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_D), ctypes.POINTER(_D), _I]),
    "mg_cgemm_split_static": (_I, [_I, _P, _I, _I, _P, _P, _P, _I]),
    "mg_tune_select": (_I, [_I, ctypes.POINTER(mg_tune_entry), _D, _D, ctypes.POINTER(_I)]),
    "mg_tune_cache_store": (_I, [ctypes.c_char_p, ctypes.c_char_p, _I, ctypes.POINTER(mg_tune_entry), _I]),
    "mg_tune_cache_lookup": (_I, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(mg_tune_entry)]),
    "mg_plan_autotune": (_I, [_P, _I, _D, ctypes.c_char_p, ctypes.POINTER(mg_tune_entry)]),
    "mg_plan_set_taylor": (_I, [_P, _I]),
    "mg_plan_set_taylor_target": (_I, [_P, ctypes.c_double]),
    "mg_ctx_set_tune_cache": (_I, [_P, ctypes.c_char_p]),
    "mg_batch_graph_create": (_I, [_P, _I, _P, _P, _P, _P, _I, ctypes.POINTER(_P)]),
    "mg_batch_graph_launch": (_I, [_P, _P]),
    "mg_batch_graph_stats": (_I, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "mg_batch_graph_destroy": (_I, [_P]),
    "mg_server_create": (_I, [_P, ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "mg_submit": (_I, [_P, ctypes.POINTER(mg_job), ctypes.POINTER(ctypes.c_uint64)]),
    "mg_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(mg_job_report)]),
    "mg_server_stats": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                             ctypes.POINTER(ctypes.c_int64)]),
    "mg_server_destroy": (_I, [_P]),
    "mg_strerror": (ctypes.c_char_p, [_I]),
    "mg_last_error_message": (ctypes.c_char_p, []),
    "mg_kernel_launch_count": (ctypes.c_int64, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmagnus.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code, where):
    if code != MG_OK:
        lib = load()
        raise MagnusError(code, where, (lib.mg_strerror(code) or b"").decode() + "; " +
                          (lib.mg_last_error_message() or b"").decode())
    return code


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(stream.cuda_stream))


# ----------------------------------------------------------------------------
# object wrappers
# ----------------------------------------------------------------------------
class Context:
    """An mg_ctx bound to one device and one CUDA stream (torch stream or None)."""

    def __init__(self, device: int = 0, stream=None, workspace_limit: int | None = None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.mg_ctx_create(ctypes.byref(h), device, _stream_ptr(stream)), "mg_ctx_create")
        self.h = h
        self.device = device
        self.stream = stream
        if workspace_limit is not None:
            _check(lib.mg_ctx_set_workspace_limit(self.h, int(workspace_limit)), "mg_ctx_set_workspace_limit")

    def set_workspace_limit(self, nbytes):
        _check(load().mg_ctx_set_workspace_limit(self.h, int(nbytes)), "mg_ctx_set_workspace_limit")

    def enable_gemm_timing(self, on=True):
        _check(load().mg_ctx_enable_gemm_timing(self.h, 1 if on else 0), "mg_ctx_enable_gemm_timing")

    def set_tune_cache(self, path):
        _check(load().mg_ctx_set_tune_cache(self.h, path.encode() if path else None), "mg_ctx_set_tune_cache")

    def set_stage_k(self, stage_k):
        _check(load().mg_ctx_set_stage_k(self.h, int(stage_k)), "mg_ctx_set_stage_k")

    def set_digit_pairs(self, on):
        """False/0: digit-major; True/1: paired, 16-deep stages; 2: paired, 32-deep stages."""
        _check(load().mg_ctx_set_digit_pairs(self.h, int(on)), "mg_ctx_set_digit_pairs")

    def set_cta_pairs(self, on):
        """True / False, or None for the library's choice by digit count."""
        _check(load().mg_ctx_set_cta_pairs(self.h, -1 if on is None else (1 if on else 0)), "mg_ctx_set_cta_pairs")

    def set_structure(self, mode):
        """Split products of real operators: bit 0 skips the exactly-zero parts of X's powers,
        bit 1 the tiles above the diagonal of symmetric results; True = 3 (default), False = 0."""
        mode = 3 if mode is True else (0 if mode is False else int(mode))
        _check(load().mg_ctx_set_structure(self.h, mode), "mg_ctx_set_structure")

    def set_wait_limit(self, seconds=4.0, stall_test=False):
        _check(load().mg_ctx_set_wait_limit(self.h, float(seconds), 1 if stall_test else 0), "mg_ctx_set_wait_limit")

    def gemm_stats(self, reset=True):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        fl = ctypes.c_double()
        _check(load().mg_ctx_gemm_stats(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                        1 if reset else 0), "mg_ctx_gemm_stats")
        return dict(launches=n.value, ms=ms.value, flops=fl.value)

    def close(self):
        if self.h:
            load().mg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """An mg_plan: resident H0 / H_k on the device, a precision mode and controls."""

    def __init__(self, ctx: Context, H0, Hk, precision=MG_PREC_FP64, slices=6, flags=0):
        import torch
        lib = load()
        self.ctx = ctx
        self.d = int(H0.shape[0])
        self.K = int(Hk.shape[0]) if Hk is not None else 0
        H0 = torch.as_tensor(H0, dtype=torch.complex128).contiguous()
        Hk_t = torch.as_tensor(Hk, dtype=torch.complex128).contiguous() if self.K else None
        host = not H0.is_cuda
        h = ctypes.c_void_p()
        _check(lib.mg_plan_create(ctx.h, ctypes.byref(h), self.d, self.K, _ptr(H0), _ptr(Hk_t), precision,
                                  slices, flags | (MG_FLAG_HOST_PTRS if host else 0)), "mg_plan_create")
        self.h = h

    def autotune(self, output, tolerance, cache_path=None):
        """Measure and set the fastest configuration within `tolerance` (mg_plan_autotune)."""
        e = mg_tune_entry()
        _check(load().mg_plan_autotune(self.h, output, float(tolerance),
                                       cache_path.encode() if cache_path else None, ctypes.byref(e)),
               "mg_plan_autotune")
        return e.as_dict()

    def set_taylor(self, taylor):
        _check(load().mg_plan_set_taylor(self.h, int(taylor)), "mg_plan_set_taylor")

    def set_taylor_target(self, u):
        _check(load().mg_plan_set_taylor_target(self.h, float(u)), "mg_plan_set_taylor_target")

    def set_magnus_order(self, order):
        _check(load().mg_plan_set_magnus_order(self.h, int(order)), "mg_plan_set_magnus_order")

    def set_controls(self, N, P, t0, dt, w, samples):
        import torch
        lib = load()
        w = torch.as_tensor(w, dtype=torch.float64).contiguous().cpu()
        samples = torch.as_tensor(samples, dtype=torch.float64).contiguous()
        host = not samples.is_cuda
        self._w = w
        self._samples = samples
        _check(lib.mg_set_controls(self.h, N, P, float(t0), float(dt), _ptr(w), _ptr(samples),
                                   MG_FLAG_HOST_PTRS if host else 0), "mg_set_controls")

    def evolve(self, output, inp, out, reorth_every=0, host=False, report=True):
        lib = load()
        rep = mg_report()
        _check(lib.mg_evolve(self.h, output, _ptr(inp), _ptr(out), reorth_every,
                             MG_FLAG_HOST_PTRS if host else 0, ctypes.byref(rep) if report else None),
               "mg_evolve")
        return rep.as_dict() if report else None

    def close(self):
        if self.h:
            load().mg_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """mg_server: memory-admitted continuous batching of jobs on one context."""

    def __init__(self, ctx: Context, mem_budget_bytes: int, quantum_intervals: int = 256):
        h = ctypes.c_void_p()
        _check(load().mg_server_create(ctx.h, int(mem_budget_bytes), int(quantum_intervals), ctypes.byref(h)),
               "mg_server_create")
        self.h = h
        self.ctx = ctx
        self._keep = {}

    def submit(self, H0, Hk, N, P, t0, dt, w, samples, output, inp, out, precision=MG_PREC_SPLIT, slices=6,
               host=False, action=False, tolerance=0.0):
        """Returns the job id, or None when the job is not admissible now (MG_EAGAIN).
        action=True runs a state job on the action-based path (MG_FLAG_STATE_ACTION)."""
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float64)
        j = mg_job(int(H0.shape[0]), int(Hk.shape[0]) if Hk is not None else 0, H0.data_ptr(),
                   Hk.data_ptr() if Hk is not None else None, int(N), int(P), float(t0), float(dt),
                   w.ctypes.data_as(ctypes.c_void_p), samples.data_ptr() if samples is not None else None,
                   int(output), inp.data_ptr() if inp is not None else None, out.data_ptr(), int(precision),
                   int(slices), (MG_FLAG_HOST_PTRS if host else 0) | (MG_FLAG_STATE_ACTION if action else 0),
                   float(tolerance))
        jid = ctypes.c_uint64()
        r = load().mg_submit(self.h, ctypes.byref(j), ctypes.byref(jid))
        if r == MG_EAGAIN:
            return None
        _check(r, "mg_submit")
        self._keep[jid.value] = (out, w)
        return jid.value

    def wait(self, job_id, timeout_s=-1.0):
        rep = mg_job_report()
        r = load().mg_wait(self.h, ctypes.c_uint64(job_id), float(timeout_s), ctypes.byref(rep))
        if r == MG_ETIMEOUT:
            return None
        self._keep.pop(job_id, None)
        _check(r, "mg_wait")
        return {k: getattr(rep, k) for k, _ in rep._fields_}

    def stats(self):
        p50, p99, ips = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(load().mg_server_stats(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(ips),
                                      ctypes.byref(n)), "mg_server_stats")
        return dict(p50_ms=p50.value, p99_ms=p99.value, intervals_per_s=ips.value, completed=n.value)

    def close(self):
        if self.h:
            load().mg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# functional entry points (same names as the C ABI)
# ----------------------------------------------------------------------------
def mg_evolve_batch(ctx, plans, outputs, inputs, outs, reorth_every=0, host=False):
    """Evolve many plans together; returns the per-job status list."""
    n = len(plans)
    PA = ctypes.c_void_p * n
    IA = ctypes.c_int * n
    hp = PA(*[p.h.value for p in plans])
    oa = IA(*outputs)
    ia = PA(*[(t.data_ptr() if t is not None else None) for t in inputs])
    oa2 = PA(*[t.data_ptr() for t in outs])
    st = IA(*([0] * n))
    _check(load().mg_evolve_batch(ctx.h, n, ctypes.cast(hp, ctypes.c_void_p), ctypes.cast(oa, ctypes.c_void_p),
                                  ctypes.cast(ia, ctypes.c_void_p), ctypes.cast(oa2, ctypes.c_void_p), reorth_every,
                                  MG_FLAG_HOST_PTRS if host else 0, ctypes.cast(st, ctypes.c_void_p)),
           "mg_evolve_batch")
    return list(st)


class BatchGraph:
    """mg_batch_graph: a batch of plans captured once in a CUDA graph and replayed."""

    def __init__(self, ctx, plans, outputs, inputs, outs, reorth_every=0):
        n = len(plans)
        PA = ctypes.c_void_p * n
        IA = ctypes.c_int * n
        self._arrays = (PA(*[p.h.value for p in plans]), IA(*outputs),
                        PA(*[(t.data_ptr() if t is not None else None) for t in inputs]),
                        PA(*[t.data_ptr() for t in outs]))
        self._keep = (list(plans), list(inputs), list(outs))
        self.n = n
        h = ctypes.c_void_p()
        hp, oa, ia, oa2 = self._arrays
        _check(load().mg_batch_graph_create(ctx.h, n, ctypes.cast(hp, ctypes.c_void_p),
                                            ctypes.cast(oa, ctypes.c_void_p), ctypes.cast(ia, ctypes.c_void_p),
                                            ctypes.cast(oa2, ctypes.c_void_p), reorth_every, ctypes.byref(h)),
               "mg_batch_graph_create")
        self.h = h

    def launch(self):
        """Replay the batch; returns the per-job status list."""
        st = (ctypes.c_int * self.n)(*([0] * self.n))
        _check(load().mg_batch_graph_launch(self.h, ctypes.cast(st, ctypes.c_void_p)), "mg_batch_graph_launch")
        return list(st)

    def stats(self):
        k, a = ctypes.c_int64(), ctypes.c_int64()
        _check(load().mg_batch_graph_stats(self.h, ctypes.byref(k), ctypes.byref(a)), "mg_batch_graph_stats")
        return dict(kernel_nodes=k.value, nodes=a.value)

    def close(self):
        if self.h:
            load().mg_batch_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _entries(entries):
    arr = (mg_tune_entry * len(entries))()
    for i, e in enumerate(entries):
        for k, _ in mg_tune_entry._fields_:
            setattr(arr[i], k, e.get(k, 0.0) if k == "taylor_target" else e[k])
    return arr


def mg_tune_select(entries, tolerance, safety=4.0):
    """Index of the fastest entry whose error x safety is within tolerance (host only)."""
    idx = ctypes.c_int()
    _check(load().mg_tune_select(len(entries), _entries(entries), float(tolerance), float(safety), ctypes.byref(idx)),
           "mg_tune_select")
    return idx.value


def mg_tune_cache_store(path, key, entries, selected):
    _check(load().mg_tune_cache_store(path.encode(), key.encode(), len(entries), _entries(entries), int(selected)),
           "mg_tune_cache_store")


def mg_tune_cache_lookup(path, key):
    """The selected entry of the latest tuning under `key` (or a key continuing it), or None."""
    e = mg_tune_entry()
    r = load().mg_tune_cache_lookup(path.encode(), key.encode(), ctypes.byref(e))
    if r == MG_EAGAIN:
        return None
    _check(r, "mg_tune_cache_lookup")
    return e.as_dict()


def mg_quadrature_nodes(P: int):
    import numpy as np
    lib = load()
    x = np.zeros(P)
    w = np.zeros(P)
    _check(lib.mg_quadrature_nodes(P, x.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)),
           "mg_quadrature_nodes")
    return x, w


def mg_csr_pattern(ops):
    """(rowptr, col, diag, val) of the action path's CSR form of `ops` (nops x d x d
    complex, H0 first; host only): val is nops x nnz complex."""
    import numpy as np
    ops = np.ascontiguousarray(ops, dtype=np.complex128)
    nops, d = ops.shape[0], ops.shape[1]
    lib = load()
    nnz = ctypes.c_int64()
    src = ops.ctypes.data_as(ctypes.c_void_p)
    _check(lib.mg_csr_pattern(d, nops, src, ctypes.byref(nnz), None, None, None, None), "mg_csr_pattern")
    n = nnz.value
    rowptr, col, diag = np.zeros(d + 1, np.int32), np.zeros(max(n, 1), np.int32), np.zeros(d, np.int32)
    val = np.zeros((nops, max(n, 1)), np.complex128)
    _check(lib.mg_csr_pattern(d, nops, src, ctypes.byref(nnz), rowptr.ctypes.data_as(ctypes.c_void_p),
                              col.ctypes.data_as(ctypes.c_void_p), diag.ctypes.data_as(ctypes.c_void_p),
                              val.ctypes.data_as(ctypes.c_void_p)), "mg_csr_pattern")
    return rowptr, col[:n], diag, val[:, :n]


def mg_second_order_weights(P: int):
    """(M, C, R): the P x P second-order weight matrix, its column and row sums (host only)."""
    import numpy as np
    out = np.zeros(P * P + 2 * P)
    _check(load().mg_second_order_weights(P, out.ctypes.data_as(ctypes.c_void_p)), "mg_second_order_weights")
    return out[:P * P].reshape(P, P), out[P * P:P * P + P], out[P * P + P:]


def mg_taylor_choice(norm1: float, precision=MG_PREC_FP64, slices=6, d=1):
    """(m, s, theta) the exponential takes for a batch of largest 1-norm norm1 (host only)."""
    m, s, th = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load().mg_taylor_choice(norm1, precision, slices, d, ctypes.byref(m), ctypes.byref(s), ctypes.byref(th)),
           "mg_taylor_choice")
    return m.value, s.value, th.value


def mg_split_digits(d: int, bits: int = 42):
    """(beta, slices): the split product's digit width at dimension d and the digit count
    that carries at least `bits` bits (host only)."""
    b, s = ctypes.c_int(), ctypes.c_int()
    _check(load().mg_split_digits(int(d), int(bits), ctypes.byref(b), ctypes.byref(s)), "mg_split_digits")
    return b.value, s.value


def mg_coefficients(ctx, N, P, K, dt, w_dev, samples, c):
    _check(load().mg_coefficients(ctx.h, N, P, K, float(dt), _ptr(w_dev), _ptr(samples), _ptr(c)),
           "mg_coefficients")


def mg_build_omega(ctx, N, d, K, dt, H0, Hk, c, Hbar, tau=None, norm1=None):
    _check(load().mg_build_omega(ctx.h, N, d, K, float(dt), _ptr(H0), _ptr(Hk), _ptr(c), _ptr(Hbar), _ptr(tau),
                                 _ptr(norm1)), "mg_build_omega")


def mg_expm(ctx, batch, d, A, U, precision=MG_PREC_FP64, slices=6, squarings=None):
    _check(load().mg_expm(ctx.h, batch, d, _ptr(A), _ptr(U), precision, slices, _ptr(squarings)), "mg_expm")


def mg_cgemm(ctx, batch, d, A, B, C, precision=MG_PREC_FP64, slices=6):
    _check(load().mg_cgemm(ctx.h, batch, d, _ptr(A), _ptr(B), _ptr(C), precision, slices), "mg_cgemm")


def mg_cgemm_split_static(device, stream, batch, d, A, B, C, slices=6):
    """Split-precision product with the library's static scratch (no device allocation)."""
    _check(load().mg_cgemm_split_static(device, _stream_ptr(stream), batch, d, _ptr(A), _ptr(B), _ptr(C), slices),
           "mg_cgemm_split_static")


def mg_propagate(ctx, N, d, U, output, inp, out, reorth_every=0, precision=MG_PREC_FP64, slices=6):
    _check(load().mg_propagate(ctx.h, N, d, _ptr(U), output, _ptr(inp), _ptr(out), reorth_every, precision,
                               slices), "mg_propagate")


def mg_kernel_launch_count() -> int:
    return int(load().mg_kernel_launch_count())


# ----------------------------------------------------------------------------
# convenience: a whole workload through the ABI
# ----------------------------------------------------------------------------
def node_samples(wl, N=None):
    """Drive samples at the library's quadrature nodes t0 + n dt + (1 + x_p) dt / 2."""
    import numpy as np
    N = wl.N if N is None else N
    x, w = mg_quadrature_nodes(wl.P)
    t = wl.t0 + wl.dt * np.arange(N)[:, None] + (1.0 + x[None, :]) * (0.5 * wl.dt)
    return np.ascontiguousarray(wl.drive(t)), w


def evolve_workload(ctx, wl, precision=MG_PREC_FP64, slices=6, N=None, reorth_every=0, device="cuda", order=1,
                    flags=0, trajectory=False, taylor_target=0.0):
    """Run a workloads.Workload through mg_plan_create / mg_set_controls / mg_evolve
    (trajectory=True: the (N + 1) x d stroboscopic states of a state workload)."""
    import torch
    N = wl.N if N is None else N
    samples, w = node_samples(wl, N)
    plan = Plan(ctx, torch.from_numpy(wl.H0).to(device), torch.from_numpy(wl.Hk).to(device), precision, slices,
                flags)
    if order != 1:
        plan.set_magnus_order(order)
    if taylor_target:
        plan.set_taylor_target(taylor_target)
    plan.set_controls(N, wl.P, wl.t0, wl.dt, w, torch.from_numpy(samples).to(device))
    if wl.psi0 is None:
        out = torch.empty((wl.d, wl.d), dtype=torch.complex128, device=device)
        rep = plan.evolve(MG_OUT_PROPAGATOR, None, out, reorth_every)
    else:
        psi0 = torch.from_numpy(wl.psi0).to(device)
        shape = (N + 1, wl.d) if trajectory else (wl.d,)
        out = torch.empty(shape, dtype=torch.complex128, device=device)
        rep = plan.evolve(MG_OUT_TRAJECTORY if trajectory else MG_OUT_STATE, psi0, out, reorth_every)
    torch.cuda.synchronize()
    plan.close()
    return out, rep
