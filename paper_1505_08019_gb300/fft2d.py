"""ctypes binding of ``libfft2d.so`` (the C ABI in ``include/fft2d.h``).

Argument marshalling only: every function below forwards to the C entry
point of the same name; all the work runs in the library's CUDA kernels.
Device buffers may be given as torch tensors (contiguous, complex64, on the
plan's device) or as raw integer device pointers.  A stream may be a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or ``None`` for the
current torch stream of the current device.

If the library has not been built, importing this module raises
``ImportError``: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfft2d.so")

FFT2D_C64 = 0
FFT2D_C32H = 1
FFT2D_R32_DCT2 = 2
FFT2D_FORWARD = -1
FFT2D_INVERSE = 1
FFT2D_PASS_ROWS = 0
FFT2D_PASS_COLS = 1
FFT2D_MAX_SIDE = 16384
FFT2D_NOALLOC_MAX_SIDE = 4096

FFT2D_OK = 0
FFT2D_ERR_ARG = 1
FFT2D_ERR_NOT_POW2 = 2
FFT2D_ERR_TOO_LARGE = 3
FFT2D_ERR_OOM = 4
FFT2D_ERR_CUDA = 5
FFT2D_ERR_TIMEOUT = 6
FFT2D_ERR_BUDGET = 7
FFT2D_ERR_UNSUPPORTED = 8

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"fft2d CUDA library not built ({LIB_PATH} missing); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` or "
        "`python paper_1505_08019_gb300/build.py`")

lib = ctypes.CDLL(LIB_PATH)

_P, _I = ctypes.c_void_p, ctypes.c_int
_sigs = {
    "fft2d_plan": ([_I, _I, _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "fft2d_destroy": ([_P], _I),
    "fft2d_sync_status": ([_P], _I),
    "fft2d_selftest_timeout": ([_P, _P], _I),
    "fft2d_selftest_withheld_load": ([_P, _P, _P, _P], _I),
    "fft2d_plan_info": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                         ctypes.POINTER(_I)], _I),
    "fft2d_exec": ([_P, _P, _P, _P], _I),
    "fft2d_exec_pass": ([_P, _I, _P, _P, _P], _I),
    "fft2d_exec_stages": ([_P, _P, _P, _I, _I, _P], _I),
    "fft2d_exec_host": ([_P, _P, _P, _P], _I),
    "fft2d_exec_batched": ([_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
                           _I),
    "fft2d_stage_table": ([_I, _I, _P], _I),
    "fft2d_exec_noalloc": ([_I, _I, _I, _P, _P, _P], _I),
    "fft2d_autotune": ([_P, _P], _I),
    "fft2d_batch_variant_count": ([_I], _I),
    "fft2d_batch_variant_name": ([_I, _I], ctypes.c_char_p),
    "fft2d_batch_get_variant": ([_I, _I], _I),
    "fft2d_batch_set_variant": ([_I, _I, _I], _I),
    "fft2d_exec_host_many": ([_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
                             _I),
    "fft2d_exec_host_many_async": (
        [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P], _I),
    "fft2d_autotune_batched": ([_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
                               _I),
    "fft2d_exec_h16": ([_P, _P, _P, _I, _P, _P, _P], _I),
    "fft2d_h16_pack": ([_I, _I, _P, _P, _P, _P], _I),
    "fft2d_h16_unpack": ([_I, _I, _P, _P, _I, _P, _P], _I),
    "fft2d_variant_count": ([_I, _I], _I),
    "fft2d_variant_name": ([_I, _I, _I], ctypes.c_char_p),
    "fft2d_plan_set_variant": ([_P, _I, _I], _I),
    "fft2d_plan_describe": ([_P, ctypes.c_char_p, _I], _I),
    "fft2d_strerror": ([_I], ctypes.c_char_p),
    "fft2d_last_error": ([], ctypes.c_char_p),
    "fft2d_version": ([], _I),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class fft2d_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("dtype", ctypes.c_int), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("in_exp", ctypes.c_void_p), ("out_exp", ctypes.c_void_p)]


class fft2d_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("batches", ctypes.c_longlong), ("peak_device_bytes", ctypes.c_longlong),
                ("mean_batch_size", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("throughput_rps", ctypes.c_double)]


FFT2D_OP_FORWARD = 0
FFT2D_OP_LOWPASS = 1
FFT2D_SERVE_SIMULATE = 1

_sigs.update({
    "fft2d_lowpass": ([_I, _I, _I, _P, ctypes.c_float, ctypes.c_float, _P], _I),
    "fft2d_serve_create": ([ctypes.c_size_t, _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "fft2d_serve_submit": ([_P, ctypes.POINTER(fft2d_request),
                            ctypes.POINTER(ctypes.c_ulonglong)], _I),
    "fft2d_serve_wait": ([_P, ctypes.c_ulonglong, _I, ctypes.POINTER(ctypes.c_double)], _I),
    "fft2d_serve_stats_get": ([_P, ctypes.POINTER(fft2d_serve_stats)], _I),
    "fft2d_serve_destroy": ([_P], _I),
})
for _name in ("fft2d_lowpass", "fft2d_serve_create", "fft2d_serve_submit", "fft2d_serve_wait",
              "fft2d_serve_stats_get", "fft2d_serve_destroy"):
    _f = getattr(lib, _name)
    _f.argtypes, _f.restype = _sigs[_name]


class FFT2DError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.fft2d_strerror(status).decode()
        detail = lib.fft2d_last_error().decode()
        super().__init__(f"{where}: {msg} (status {status})" + (f" [{detail}]" if detail else ""))


def _check(status: int, where: str) -> None:
    if status != FFT2D_OK:
        raise FFT2DError(status, where)


def _dptr(x) -> int:
    """Device pointer of a torch tensor (checked) or a raw integer."""
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _hptr(x) -> int:
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if x.is_cuda:
            raise ValueError("expected a host tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    return x.ctypes.data   # numpy array


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------- C ABI mirror
def fft2d_plan(rows: int, cols: int, dtype: int = FFT2D_C64, dir: int = FFT2D_FORWARD) -> int:
    h = ctypes.c_void_p()
    _check(lib.fft2d_plan(rows, cols, dtype, dir, ctypes.byref(h)), "fft2d_plan")
    return h.value


def fft2d_destroy(plan: int) -> None:
    _check(lib.fft2d_destroy(plan), "fft2d_destroy")


def fft2d_sync_status(plan: int) -> None:
    """Wait for the device; raise FFT2DError if a kernel's bounded wait gave up."""
    _check(lib.fft2d_sync_status(plan), "fft2d_sync_status")


def fft2d_selftest_timeout(plan: int, stream=None) -> None:
    _check(lib.fft2d_selftest_timeout(plan, _stream(stream)), "fft2d_selftest_timeout")


def fft2d_selftest_withheld_load(plan: int, inp, out, stream=None) -> None:
    _check(lib.fft2d_selftest_withheld_load(plan, _dptr(inp), _dptr(out), _stream(stream)),
           "fft2d_selftest_withheld_load")


def fft2d_plan_info(plan: int) -> tuple[int, int, int, int]:
    r, c, d, s = _I(), _I(), _I(), _I()
    _check(lib.fft2d_plan_info(plan, ctypes.byref(r), ctypes.byref(c), ctypes.byref(d),
                               ctypes.byref(s)), "fft2d_plan_info")
    return r.value, c.value, d.value, s.value


def fft2d_exec(plan: int, inp, out, stream=None) -> None:
    _check(lib.fft2d_exec(plan, _dptr(inp), _dptr(out), _stream(stream)), "fft2d_exec")


def fft2d_exec_pass(plan: int, pass_: int, inp, out, stream=None) -> None:
    _check(lib.fft2d_exec_pass(plan, pass_, _dptr(inp), _dptr(out), _stream(stream)),
           "fft2d_exec_pass")


def fft2d_exec_stages(plan: int, inp, out, row_stages: int, col_stages: int,
                      stream=None) -> None:
    _check(lib.fft2d_exec_stages(plan, _dptr(inp), _dptr(out), row_stages, col_stages,
                                 _stream(stream)), "fft2d_exec_stages")


def fft2d_exec_host(plan: int, inp_host, out_host, stream=None) -> None:
    _check(lib.fft2d_exec_host(plan, _hptr(inp_host), _hptr(out_host), _stream(stream)),
           "fft2d_exec_host")


def fft2d_exec_batched(plans, inps, outs, stream=None) -> None:
    n = len(plans)
    if len(inps) != n or len(outs) != n:
        raise ValueError("plans, inputs and outputs must have the same length")
    arr = ctypes.c_void_p * max(n, 1)
    P = arr(*plans)
    I_ = arr(*[_dptr(x) for x in inps])
    O_ = arr(*[_dptr(x) for x in outs])
    _check(lib.fft2d_exec_batched(n, P, I_, O_, _stream(stream)), "fft2d_exec_batched")


def fft2d_exec_noalloc(rows: int, cols: int, dir: int, inp, out, stream=None) -> None:
    """Plan-free transform that allocates no device memory (sides <= 4096)."""
    _check(lib.fft2d_exec_noalloc(rows, cols, dir, _dptr(inp), _dptr(out), _stream(stream)),
           "fft2d_exec_noalloc")


def fft2d_exec_h16(plan: int, inp, in_exp, in_axis: int, out, out_exp, stream=None) -> None:
    """half2 transform: inp/out are (rows, cols) half2 buffers (e.g. torch
    float16 tensors of shape (rows, cols, 2)), in_exp / out_exp int32 device
    vectors (input per row or column, output per column)."""
    _check(lib.fft2d_exec_h16(plan, _dptr(inp), _dptr(in_exp), in_axis, _dptr(out),
                              _dptr(out_exp), _stream(stream)), "fft2d_exec_h16")


def fft2d_h16_pack(rows: int, cols: int, inp, out, out_exp, stream=None) -> None:
    _check(lib.fft2d_h16_pack(rows, cols, _dptr(inp), _dptr(out), _dptr(out_exp),
                              _stream(stream)), "fft2d_h16_pack")


def fft2d_h16_unpack(rows: int, cols: int, inp, exps, axis: int, out, stream=None) -> None:
    _check(lib.fft2d_h16_unpack(rows, cols, _dptr(inp), _dptr(exps), axis, _dptr(out),
                                _stream(stream)), "fft2d_h16_unpack")


def fft2d_batch_variant_count(pass_: int) -> int:
    return lib.fft2d_batch_variant_count(pass_)


def fft2d_batch_variant_name(pass_: int, index: int) -> str:
    return lib.fft2d_batch_variant_name(pass_, index).decode()


def fft2d_batch_get_variant(pass_: int, L: int) -> int:
    return lib.fft2d_batch_get_variant(pass_, L)


def fft2d_batch_set_variant(pass_: int, L: int, variant: int) -> None:
    _check(lib.fft2d_batch_set_variant(pass_, L, variant), "fft2d_batch_set_variant")


def fft2d_exec_host_many(plans, inps, outs, stream=None) -> None:
    """Pipelined fft2d_exec_host over many host images (synchronous)."""
    n = len(plans)
    if len(inps) != n or len(outs) != n:
        raise ValueError("plans, inputs and outputs must have the same length")
    arr = ctypes.c_void_p * max(n, 1)
    _check(lib.fft2d_exec_host_many(n, arr(*plans), arr(*[_hptr(x) for x in inps]),
                                    arr(*[_hptr(x) for x in outs]), _stream(stream)),
           "fft2d_exec_host_many")


def fft2d_exec_host_many_async(plans, inps, outs, stream=None) -> None:
    """fft2d_exec_host_many without the final wait: the stream is ordered
    after every copy; keep the host buffers alive until it is synchronised."""
    n = len(plans)
    if len(inps) != n or len(outs) != n:
        raise ValueError("plans, inputs and outputs must have the same length")
    arr = ctypes.c_void_p * max(n, 1)
    _check(lib.fft2d_exec_host_many_async(n, arr(*plans), arr(*[_hptr(x) for x in inps]),
                                          arr(*[_hptr(x) for x in outs]), _stream(stream)),
           "fft2d_exec_host_many_async")


def fft2d_autotune_batched(plans, inps, outs, stream=None) -> None:
    """Tune the grouped launches of this batch (buffers are overwritten)."""
    n = len(plans)
    arr = ctypes.c_void_p * max(n, 1)
    _check(lib.fft2d_autotune_batched(n, arr(*plans), arr(*[_dptr(x) for x in inps]),
                                      arr(*[_dptr(x) for x in outs]), _stream(stream)),
           "fft2d_autotune_batched")


def fft2d_autotune(plan: int, stream=None) -> None:
    """Time the kernel variants for this plan's shape and keep the fastest."""
    _check(lib.fft2d_autotune(plan, _stream(stream)), "fft2d_autotune")


def fft2d_variant_count(pass_: int, L: int) -> int:
    return lib.fft2d_variant_count(pass_, L)


def fft2d_variant_name(pass_: int, L: int, index: int) -> str:
    return lib.fft2d_variant_name(pass_, L, index).decode()


def fft2d_plan_set_variant(plan: int, pass_: int, variant: int) -> None:
    _check(lib.fft2d_plan_set_variant(plan, pass_, variant), "fft2d_plan_set_variant")


def fft2d_plan_describe(plan: int) -> str:
    buf = ctypes.create_string_buffer(256)
    _check(lib.fft2d_plan_describe(plan, buf, 256), "fft2d_plan_describe")
    return buf.value.decode()


def fft2d_lowpass(rows: int, cols: int, dtype: int, data, sigma_rows: float,
                  sigma_cols: float, stream=None) -> None:
    _check(lib.fft2d_lowpass(rows, cols, dtype, _dptr(data), sigma_rows, sigma_cols,
                             _stream(stream)), "fft2d_lowpass")


def fft2d_serve_create(hbm_budget_bytes: int, streams: int = 4, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib.fft2d_serve_create(hbm_budget_bytes, streams, flags, ctypes.byref(h)),
           "fft2d_serve_create")
    return h.value


def fft2d_serve_submit(srv: int, op: int, rows: int, cols: int, dtype: int, inp_host,
                       out_host, in_exp=None, out_exp=None) -> int:
    """Queue a request on host buffers (torch CPU tensors, numpy arrays or raw
    pointers); returns its ticket.  Keep the buffers alive until it is done.
    FFT2D_C32H requests pass half2 data with per-row input exponents
    (``in_exp``, rows int32) and receive half2 data with per-column
    exponents (``out_exp``, cols int32)."""
    req = fft2d_request(op, rows, cols, dtype, _hptr(inp_host), _hptr(out_host),
                        None if in_exp is None else _hptr(in_exp),
                        None if out_exp is None else _hptr(out_exp))
    t = ctypes.c_ulonglong()
    _check(lib.fft2d_serve_submit(srv, ctypes.byref(req), ctypes.byref(t)), "fft2d_serve_submit")
    return t.value


def fft2d_serve_wait(srv: int, ticket: int, timeout_ms: int = -1) -> float:
    """Wait for a ticket; returns its latency in ms."""
    lat = ctypes.c_double()
    _check(lib.fft2d_serve_wait(srv, ticket, timeout_ms, ctypes.byref(lat)), "fft2d_serve_wait")
    return lat.value


def fft2d_serve_stats_get(srv: int) -> dict:
    st = fft2d_serve_stats()
    _check(lib.fft2d_serve_stats_get(srv, ctypes.byref(st)), "fft2d_serve_stats_get")
    return {name: getattr(st, name) for name, _ in fft2d_serve_stats._fields_}


def fft2d_serve_destroy(srv: int) -> None:
    _check(lib.fft2d_serve_destroy(srv), "fft2d_serve_destroy")


def fft2d_stage_table(L: int, dir: int = FFT2D_FORWARD):
    """The per-stage rotation-factor table a plan uploads (numpy complex64)."""
    import numpy as np
    n = (1 << L) - 1
    out = np.zeros(max(n, 1), dtype=np.complex64)
    _check(lib.fft2d_stage_table(L, dir, out.ctypes.data), "fft2d_stage_table")
    return out[:n]


def fft2d_strerror(status: int) -> str:
    return lib.fft2d_strerror(status).decode()


def fft2d_last_error() -> str:
    return lib.fft2d_last_error().decode()


def fft2d_version() -> int:
    return lib.fft2d_version()


# ------------------------------------------------------------ convenience
class Plan:
    """Owning wrapper of an fft2d plan handle."""

    def __init__(self, rows: int, cols: int, dir: int = FFT2D_FORWARD, dtype: int = FFT2D_C64):
        self.rows, self.cols, self.dir, self.dtype = rows, cols, dir, dtype
        self.handle = fft2d_plan(rows, cols, dtype, dir)

    def __call__(self, inp, out=None, stream=None):
        """Transform device tensor ``inp`` into ``out`` (new tensor if None)."""
        if out is None:
            import torch
            out = torch.empty_like(inp)
        fft2d_exec(self.handle, inp, out, stream)
        return out

    def close(self):
        if self.handle:
            fft2d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
