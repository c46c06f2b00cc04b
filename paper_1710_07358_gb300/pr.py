"""Python binding of libpr.so (the C ABI in include/pr.h).

Two layers, both argument marshalling only:
  * ``pr_*`` functions with the C names and signatures (raw integers for
    pointers and stream handles), returning the status code;
  * tensor helpers (``reduce``, ``segmented_reduce``, ``reduce_rows``,
    ``reduce_backward``, ``reduce_host``) that take torch tensors, pass their
    device pointers and torch's current stream, allocate outputs with torch
    and raise ``PrError`` on a non-OK status.

Every reduction runs in the library's CUDA kernels; if libpr.so is missing the
first call raises.  There is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpr.so")

DTYPES = {"f32": 0, "f16": 1, "bf16": 2, "f64": 3, "i32": 4, "u32": 5, "i64": 6}
OPS = {"sum": 0, "prod": 1, "max": 2, "min": 3, "and": 4, "or": 5, "xor": 6}
PRECISIONS = {"plain": 0, "compensated": 1, "fp64_combine": 2}
KINDS = {"reduce": 0, "segmented": 1, "backward": 2, "rows": 3, "axis": 4}
STATUS = {0: "PR_OK", 1: "PR_ERR_INVALID", 2: "PR_ERR_UNSUPPORTED", 3: "PR_ERR_CUDA",
          4: "PR_ERR_TIMEOUT", 5: "PR_ERR_NOMEM"}
ELEM_SIZE = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8, "i32": 4, "u32": 4, "i64": 8}


class pr_config(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("unroll", ctypes.c_int32), ("vec_bytes", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pr_prod_aux(ctypes.Structure):
    _fields_ = [("p_nz", ctypes.c_double), ("zero_count", ctypes.c_int64), ("first_zero", ctypes.c_int64)]


class PrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


_P, _I64, _I32, _I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
_SIGS = {
    "pr_reduce": [_P, _I64, _I, _I, _P, _P],
    "pr_reduce_ex": [_P, _I64, _I, _I, _I, _I, _P, _P],
    "pr_reduce_arg": [_P, _I64, _I, _I, _P, _P, _P],
    "pr_segmented_reduce": [_P, _P, _I64, _I, _I, _P, _P],
    "pr_segmented_reduce_aux": [_P, _P, _I64, _I, _I, _I, _P, _P, _P, _P],
    "pr_reduce_rows": [_P, _I64, _I64, _I, _I, _I, _P, _P, _P, _P],
    "pr_reduce_backward": [_I, _I, _P, _I64, _I64, _P, _P, _P, _P, _P],
    "pr_reduce_axis": [_P, _I64, _I64, _I64, _I, _I, _I, _P, _P, _P, _P],
    "pr_scan": [_P, _I64, _I, _I, ctypes.c_int32, _P, _P],
    "pr_check_bounded_wait": [ctypes.c_int32, _P],
    "pr_beckmann": [_P, _P, _P, _P, _I64, ctypes.c_float, _I32, _P, _I32, _P, _P],
    "pr_golden_iterations": [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_I32)],
    "pr_line_search": [_P, _P, _P, _P, _I64, ctypes.c_float, _I32, ctypes.c_double, ctypes.c_double, _I, _I32,
                       _I32, _P, _P],
    "pr_reduce_axis_backward": [_I, _I, _P, _I64, _I64, _I64, _P, _P, _P, _P, _P],
    "pr_reduce_host": [_P, _I64, _I, _I, _P, _P],
    "pr_reduce_noalloc": [_P, _I64, _I, _I, _P, _P],
    "pr_prepare": [_P],
    "pr_debug_inject_fault": [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_I32)],
    "pr_debug_reduce_plan": [_P, _I64, _I, _I, _I, _I32, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                             ctypes.POINTER(_I64)],
    "pr_last_device_error": [_P, ctypes.POINTER(_I32)],
    "pr_get_config": [_I, _I, _I, _I, _I64, ctypes.POINTER(pr_config)],
    "pr_set_config": [_I, _I, _I, _I, _I64, ctypes.POINTER(pr_config)],
    "pr_autotune": [_I, _P, _I64, _P, _I64, _I, _I, _I, _P, ctypes.POINTER(pr_config)],
    "pr_autotune_axis": [_P, _I64, _I64, _I64, _I, _I, _I, _P, ctypes.POINTER(pr_config)],
    "pr_tune_save": [ctypes.c_char_p],
    "pr_tune_load": [ctypes.c_char_p],
}

_lib = None


def lib():
    """The loaded libpr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpr.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes, f.restype = args, _I
        L.pr_out_dtype.argtypes, L.pr_out_dtype.restype = [_I, _I], _I
        L.pr_status_string.argtypes, L.pr_status_string.restype = [_I], ctypes.c_char_p
        L.pr_last_error_message.argtypes, L.pr_last_error_message.restype = [], ctypes.c_char_p
        L.pr_version.argtypes, L.pr_version.restype = [], ctypes.c_char_p
        _lib = L
        _load_tuning(L)
    return _lib


TUNING_PATH = os.path.join(_HERE, "tuning", "gb300.json")


def _load_tuning(L):
    """Load the shipped launch-configuration table when a GPU is present (the
    library checks that the table was made on a GPU of the same name)."""
    if os.environ.get("PR_NO_TUNING") or not os.path.exists(TUNING_PATH):
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    L.pr_tune_load(TUNING_PATH.encode())


# ---------------------------------------------------------------------------
# C names (raw arguments, status returned)
# ---------------------------------------------------------------------------

def pr_reduce(x, n, dtype, op, out, stream):
    return lib().pr_reduce(x, n, dtype, op, out, stream)


def pr_reduce_ex(x, n, dtype, op, precision, out_dtype, out, stream):
    return lib().pr_reduce_ex(x, n, dtype, op, precision, out_dtype, out, stream)


def pr_reduce_arg(x, n, dtype, op, out, idx, stream):
    return lib().pr_reduce_arg(x, n, dtype, op, out, idx, stream)


def pr_segmented_reduce(x, offsets, nseg, dtype, op, out, stream):
    return lib().pr_segmented_reduce(x, offsets, nseg, dtype, op, out, stream)


def pr_segmented_reduce_aux(x, offsets, nseg, dtype, op, precision, out, argidx, aux, stream):
    return lib().pr_segmented_reduce_aux(x, offsets, nseg, dtype, op, precision, out, argidx, aux, stream)


def pr_reduce_rows(x, rows, cols, dtype, op, precision, out, argidx, aux, stream):
    return lib().pr_reduce_rows(x, rows, cols, dtype, op, precision, out, argidx, aux, stream)


def pr_reduce_backward(op, dtype, x, rows, cols, grad_out, argidx, aux, grad_in, stream):
    return lib().pr_reduce_backward(op, dtype, x, rows, cols, grad_out, argidx, aux, grad_in, stream)


def pr_reduce_axis(x, outer, n, inner, dtype, op, precision, out, argidx, aux, stream):
    return lib().pr_reduce_axis(x, outer, n, inner, dtype, op, precision, out, argidx, aux, stream)


def pr_reduce_axis_backward(op, dtype, x, outer, n, inner, grad_out, argidx, aux, grad_in, stream):
    return lib().pr_reduce_axis_backward(op, dtype, x, outer, n, inner, grad_out, argidx, aux, grad_in, stream)


def pr_scan(x, n, dtype, op, exclusive, y, stream):
    return lib().pr_scan(x, n, dtype, op, exclusive, y, stream)


def pr_check_bounded_wait(polls, stream):
    return lib().pr_check_bounded_wait(polls, stream)


def pr_beckmann(x, d, t0, cap, n, beta, power, alphas, m, out, stream):
    return lib().pr_beckmann(x, d, t0, cap, n, beta, power, alphas, m, out, stream)


def pr_golden_iterations(lo, hi, tol, count_ref):
    return lib().pr_golden_iterations(lo, hi, tol, count_ref)


def pr_line_search(x, d, t0, cap, n, beta, power, lo, hi, method, count, depth, result, stream):
    return lib().pr_line_search(x, d, t0, cap, n, beta, power, lo, hi, method, count, depth, result, stream)


def pr_reduce_host(host_x, n, dtype, op, host_out, stream):
    return lib().pr_reduce_host(host_x, n, dtype, op, host_out, stream)


def pr_reduce_noalloc(x, n, dtype, op, out, stream):
    return lib().pr_reduce_noalloc(x, n, dtype, op, out, stream)


def pr_prepare(stream):
    return lib().pr_prepare(stream)


FAULT_SITES = {"none": 0, "alloc": 1, "launch": 2}


def pr_debug_inject_fault(site, after, pending_ref):
    return lib().pr_debug_inject_fault(site, after, pending_ref)


def inject_fault(site: str, after: int = 0) -> bool:
    """Arm (or, with "none", disarm) the library's one-shot host-side fault
    hook; returns whether a fault was still pending before this call."""
    p = ctypes.c_int32(0)
    check(pr_debug_inject_fault(FAULT_SITES[site], after, ctypes.byref(p)))
    return bool(p.value)


def pr_debug_reduce_plan(x, n, dtype, op, precision, arg, stream, grid_ref, block_ref, tail_ref):
    return lib().pr_debug_reduce_plan(x, n, dtype, op, precision, arg, stream, grid_ref, block_ref, tail_ref)


def reduce_plan(x, op: str, precision: str = "plain", arg: bool = False, stream=None) -> dict:
    """The launch reduce() (or reduce_arg(), with arg) would make for x:
    {"grid", "block", "tail_vectors"} (tail_vectors: the vectors past the
    grid-stride part that blocks claim in tiles; 0 for none)."""
    g, b, t = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    check(pr_debug_reduce_plan(_ptr(x), x.numel(), DTYPES[dtype_name(x)], OPS[op], PRECISIONS[precision],
                               1 if arg else 0, _stream(x, stream), ctypes.byref(g), ctypes.byref(b),
                               ctypes.byref(t)))
    return {"grid": g.value, "block": b.value, "tail_vectors": t.value}


def pr_last_device_error(stream, code_ref):
    return lib().pr_last_device_error(stream, code_ref)


def pr_out_dtype(dtype, op):
    return lib().pr_out_dtype(dtype, op)


def pr_status_string(status):
    return lib().pr_status_string(status).decode()


def pr_last_error_message():
    return lib().pr_last_error_message().decode()


def pr_version():
    return lib().pr_version().decode()


def pr_get_config(kind, dtype, op, precision, n, cfg_ref):
    return lib().pr_get_config(kind, dtype, op, precision, n, cfg_ref)


def pr_set_config(kind, dtype, op, precision, n, cfg_ref):
    return lib().pr_set_config(kind, dtype, op, precision, n, cfg_ref)


def pr_autotune(kind, x, n, offsets, nseg, dtype, op, precision, stream, best_ref):
    return lib().pr_autotune(kind, x, n, offsets, nseg, dtype, op, precision, stream, best_ref)


def pr_autotune_axis(x, outer, n, inner, dtype, op, precision, stream, best_ref):
    return lib().pr_autotune_axis(x, outer, n, inner, dtype, op, precision, stream, best_ref)


def pr_tune_save(path):
    return lib().pr_tune_save(path.encode() if isinstance(path, str) else path)


def pr_tune_load(path):
    return lib().pr_tune_load(path.encode() if isinstance(path, str) else path)


def check(status):
    if status != 0:
        raise PrError(status, pr_last_error_message())


# ---------------------------------------------------------------------------
# Tensor helpers
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def dtype_name(t) -> str:
    torch = _torch()
    m = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16", torch.float64: "f64",
         torch.int32: "i32", torch.int64: "i64"}
    if hasattr(torch, "uint32"):
        m[torch.uint32] = "u32"
    if t.dtype not in m:
        raise TypeError("unsupported tensor dtype %s" % t.dtype)
    return m[t.dtype]


def torch_dtype(name: str):
    torch = _torch()
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16, "f64": torch.float64,
            "i32": torch.int32, "i64": torch.int64, "u32": getattr(torch, "uint32", None)}[name]


def out_dtype_name(dtype: str, op: str) -> str:
    if dtype in ("f16", "bf16"):
        return dtype if op in ("max", "min") else "f32"
    if dtype == "i32" and op == "sum":
        return "i64"
    return dtype


def _stream(t, stream=None):
    torch = _torch()
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return torch.cuda.current_stream(t.device).cuda_stream


def _ptr(t):
    return t.data_ptr() if t is not None else None


def reduce(x, op: str, precision: str = "plain", out_dtype: str | None = None, out=None, stream=None):
    """0-d tensor holding the reduction of every element of the CUDA tensor x."""
    torch = _torch()
    if not x.is_cuda:
        raise ValueError("reduce() needs a CUDA tensor; use reduce_host() for host memory")
    if not x.is_contiguous():
        raise ValueError("x must be contiguous")
    d = dtype_name(x)
    od = out_dtype or out_dtype_name(d, op)
    if out is None:
        out = torch.empty((), dtype=torch_dtype(od), device=x.device)
    check(pr_reduce_ex(_ptr(x), x.numel(), DTYPES[d], OPS[op], PRECISIONS[precision], DTYPES[od],
                       _ptr(out), _stream(x, stream)))
    return out


def reduce_arg(x, op: str, out=None, idx=None, stream=None):
    """(0-d value tensor, 0-d int64 index tensor): max or min of x and the index
    of its first occurrence (written into out / idx when given)."""
    torch = _torch()
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("reduce_arg() needs a contiguous CUDA tensor")
    d = dtype_name(x)
    if out is None:
        out = torch.empty((), dtype=torch_dtype(out_dtype_name(d, op)), device=x.device)
    if idx is None:
        idx = torch.empty((), dtype=torch.int64, device=x.device)
    check(pr_reduce_arg(_ptr(x), x.numel(), DTYPES[d], OPS[op], _ptr(out), _ptr(idx), _stream(x, stream)))
    return out, idx


def _outputs(count, dtype_out, device, argidx, aux, out, argidx_out, aux_out):
    """Output tensors of a reduction with `count` results: the caller's when
    given, else new ones (argidx / aux only when requested)."""
    torch = _torch()
    if out is None:
        out = torch.empty(count, dtype=dtype_out, device=device)
    ai = (argidx_out if argidx_out is not None else torch.empty(count, dtype=torch.int64, device=device)) \
        if argidx else None
    ax = (aux_out if aux_out is not None else torch.empty(count * 24, dtype=torch.int8, device=device)) \
        if aux else None
    return out, ai, ax


def segmented_reduce(x, offsets, op: str, precision: str = "plain", argidx: bool = False,
                     aux: bool = False, stream=None, out=None, argidx_out=None, aux_out=None):
    """Per-segment reductions of x[offsets[s]:offsets[s+1]] (offsets: int64 CUDA tensor).

    Returns out, or (out, argidx) / (out, aux) when requested; aux is an
    int8 tensor of nseg * 24 bytes (pr_prod_aux records), see prod_aux_fields().
    out / argidx_out / aux_out: caller-owned output tensors to write instead."""
    torch = _torch()
    d = dtype_name(x)
    nseg = offsets.numel() - 1
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous int64 CUDA tensor")
    out, ai, ax = _outputs(max(nseg, 0), torch_dtype(out_dtype_name(d, op)), x.device, argidx, aux, out,
                           argidx_out, aux_out)
    check(pr_segmented_reduce_aux(_ptr(x), _ptr(offsets), nseg, DTYPES[d], OPS[op], PRECISIONS[precision],
                                  _ptr(out), _ptr(ai), _ptr(ax), _stream(x, stream)))
    if argidx:
        return out, ai
    if aux:
        return out, ax
    return out


def reduce_rows(x, op: str, precision: str = "plain", argidx: bool = False, aux: bool = False, stream=None,
                out=None, argidx_out=None, aux_out=None):
    """Reduce a contiguous [rows, cols] CUDA tensor along its last dimension
    (outputs as in segmented_reduce)."""
    if x.dim() != 2 or not x.is_contiguous():
        raise ValueError("reduce_rows needs a contiguous 2-D tensor")
    d = dtype_name(x)
    rows, cols = x.shape
    out, ai, ax = _outputs(rows, torch_dtype(out_dtype_name(d, op)), x.device, argidx, aux, out, argidx_out,
                           aux_out)
    check(pr_reduce_rows(_ptr(x), rows, cols, DTYPES[d], OPS[op], PRECISIONS[precision], _ptr(out), _ptr(ai),
                         _ptr(ax), _stream(x, stream)))
    if argidx:
        return out, ai
    if aux:
        return out, ax
    return out


def scan(x, op: str, exclusive: bool = False, out=None, stream=None):
    """Prefix scan of a contiguous CUDA tensor (flattened) under op; same
    number of elements, in the output type of the reduction (pr_out_dtype)."""
    torch = _torch()
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("scan needs a contiguous CUDA tensor")
    d = dtype_name(x)
    y = out if out is not None else torch.empty(x.shape, dtype=torch_dtype(out_dtype_name(d, op)), device=x.device)
    check(pr_scan(_ptr(x), x.numel(), DTYPES[d], OPS[op], 1 if exclusive else 0, _ptr(y), _stream(x, stream)))
    return y


SEARCH = {"golden": 0, "fibonacci": 1}


def _links(x, d, t0, cap):
    torch = _torch()
    for t in (x, d, t0, cap):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != x.numel():
            raise ValueError("x, d, t0, cap: contiguous float32 CUDA tensors of one length")


def beckmann(x, d, t0, cap, alphas, beta: float = 0.15, power: int = 4, stream=None, out=None):
    """phi(alpha) of the Beckmann objective at each alpha (at most 16), one
    pass over the links; a float64 CUDA tensor (out, when given)."""
    torch = _torch()
    _links(x, d, t0, cap)
    al = torch.as_tensor(alphas, dtype=torch.float64).reshape(-1).to(x.device)
    if out is None:
        out = torch.empty(al.numel(), dtype=torch.float64, device=x.device)
    check(pr_beckmann(_ptr(x), _ptr(d), _ptr(t0), _ptr(cap), x.numel(), beta, power, _ptr(al), al.numel(),
                      _ptr(out), _stream(x, stream)))
    return out


def golden_iterations(lo: float, hi: float, tol: float) -> int:
    """Golden-section iterations until the bracket is at most tol wide
    (pr_golden_iterations)."""
    k = ctypes.c_int32(0)
    check(pr_golden_iterations(lo, hi, tol, ctypes.byref(k)))
    return k.value


def line_search(x, d, t0, cap, lo: float = 0.0, hi: float = 1.0, beta: float = 0.15, power: int = 4,
                method: str = "golden", tol: float | None = None, count: int | None = None, depth: int = 2,
                result=None, stream=None):
    """Minimise the Beckmann objective on [lo, hi] by golden-section (count
    iterations, or enough for a bracket of width tol) or Fibonacci search
    (count evaluations).  Returns a float64 CUDA tensor: final a, b, the
    better of the last two points, its phi."""
    torch = _torch()
    _links(x, d, t0, cap)
    if count is None:
        if method != "golden" or tol is None:
            raise ValueError("give count, or tol for golden-section search")
        count = golden_iterations(lo, hi, tol)
    res = result if result is not None else torch.empty(4, dtype=torch.float64, device=x.device)
    check(pr_line_search(_ptr(x), _ptr(d), _ptr(t0), _ptr(cap), x.numel(), beta, power, lo, hi, SEARCH[method],
                         count, depth, _ptr(res), _stream(x, stream)))
    return res


def axis_shape(shape, dim):
    """(outer, n, inner) of a reduction of `dim` over a contiguous tensor of `shape`."""
    dim = dim % len(shape)
    outer = 1
    for v in shape[:dim]:
        outer *= v
    inner = 1
    for v in shape[dim + 1:]:
        inner *= v
    return outer, shape[dim], inner


def reduce_axis(x, op: str, dim: int, precision: str = "plain", argidx: bool = False, aux: bool = False,
                stream=None, out=None, argidx_out=None, aux_out=None):
    """Reduce a contiguous CUDA tensor along `dim` (the other dimensions kept).

    Returns out, or (out, argidx) / (out, aux) when requested, shaped like x
    without `dim`; aux is an int8 tensor of 24-byte pr_prod_aux records.
    out / argidx_out / aux_out: caller-owned output tensors to write instead."""
    torch = _torch()
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("reduce_axis needs a contiguous CUDA tensor")
    d = dtype_name(x)
    outer, n, inner = axis_shape(tuple(x.shape), dim)
    oshape = tuple(v for i, v in enumerate(x.shape) if i != dim % x.dim())
    if out is None:
        out = torch.empty(oshape, dtype=torch_dtype(out_dtype_name(d, op)), device=x.device)
    ai = (argidx_out if argidx_out is not None else torch.empty(oshape, dtype=torch.int64, device=x.device)) \
        if argidx else None
    ax = (aux_out if aux_out is not None else torch.empty(outer * inner * 24, dtype=torch.int8, device=x.device)) \
        if aux else None
    check(pr_reduce_axis(_ptr(x), outer, n, inner, DTYPES[d], OPS[op], PRECISIONS[precision], _ptr(out), _ptr(ai),
                         _ptr(ax), _stream(x, stream)))
    if argidx:
        return out, ai
    if aux:
        return out, ax
    return out


def reduce_axis_backward(op: str, x, dim: int, grad_out, argidx=None, aux=None, out=None, stream=None):
    """grad_in (x's shape) for reduce_axis(x, op, dim); x is read only for prod
    (anything with .shape and .data_ptr() serves otherwise)."""
    torch = _torch()
    d = dtype_name(grad_out)
    shape = tuple(x.shape)
    outer, n, inner = axis_shape(shape, dim)
    gi = out if out is not None else torch.empty(shape, dtype=grad_out.dtype, device=grad_out.device)
    xp = _ptr(x) if op == "prod" else None
    check(pr_reduce_axis_backward(OPS[op], DTYPES[d], xp, outer, n, inner, _ptr(grad_out.contiguous()),
                                  _ptr(argidx), _ptr(aux), _ptr(gi), _stream(grad_out, stream)))
    return gi


def prod_aux_fields(aux):
    """(p_nz float64, zero_count int64, first_zero int64) tensors from an aux byte tensor."""
    torch = _torch()
    rec = aux.view(torch.int64).view(-1, 3)
    return rec[:, 0].view(torch.float64), rec[:, 1], rec[:, 2]


def reduce_backward(op: str, x, grad_out, argidx=None, aux=None, out=None, stream=None):
    """grad_in [rows, cols] for a row reduction of x (see pr_reduce_backward)."""
    torch = _torch()
    d = dtype_name(grad_out)
    rows, cols = x.shape
    gi = out if out is not None else torch.empty((rows, cols), dtype=grad_out.dtype, device=grad_out.device)
    xp = _ptr(x) if op == "prod" else None
    check(pr_reduce_backward(OPS[op], DTYPES[d], xp, rows, cols, _ptr(grad_out.contiguous()), _ptr(argidx),
                             _ptr(aux), _ptr(gi), _stream(grad_out, stream)))
    return gi


def reduce_host(x, op: str, stream=None):
    """Reduce a host tensor (pinned for full speed) on the current GPU; returns a Python number."""
    torch = _torch()
    if x.is_cuda or not x.is_contiguous():
        raise ValueError("reduce_host needs a contiguous host tensor")
    import numpy as np
    d = dtype_name(x)
    od = out_dtype_name(d, op)
    res = np.zeros(1, dtype={"f32": np.float32, "f64": np.float64, "i32": np.int32, "u32": np.uint32,
                             "i64": np.int64, "f16": np.uint16, "bf16": np.uint16}[od])
    st = torch.cuda.current_stream().cuda_stream if stream is None else _stream(x, stream)
    check(pr_reduce_host(_ptr(x), x.numel(), DTYPES[d], OPS[op], res.ctypes.data, st))
    if od == "f16":
        return float(res.view(np.float16)[0])
    if od == "bf16":
        return float((res.astype(np.uint32) << 16).view(np.float32)[0])
    return res[0].item()


def prepare(stream=None):
    torch = _torch()
    st = torch.cuda.current_stream().cuda_stream if stream is None else _stream(None, stream)
    check(pr_prepare(st))


def last_device_error(stream=None) -> int:
    torch = _torch()
    st = torch.cuda.current_stream().cuda_stream if stream is None else _stream(None, stream)
    code = ctypes.c_int32(0)
    check(pr_last_device_error(st, ctypes.byref(code)))
    return code.value


def get_config(kind: str, dtype: str, op: str, precision: str = "plain", n: int = 1) -> dict:
    c = pr_config()
    check(pr_get_config(KINDS[kind], DTYPES[dtype], OPS[op], PRECISIONS[precision], n, ctypes.byref(c)))
    return c.as_dict()


def set_config(kind: str, dtype: str, op: str, precision: str, n: int, cfg: dict):
    c = pr_config(**cfg)
    check(pr_set_config(KINDS[kind], DTYPES[dtype], OPS[op], PRECISIONS[precision], n, ctypes.byref(c)))


def autotune(kind: str, x, op: str, precision: str = "plain", offsets=None, stream=None, dim: int = -1) -> dict:
    """Tune (and keep) the configuration for x's size bucket: kind "reduce"
    (x 1-D), "segmented" (x 1-D plus offsets), "rows" (x a contiguous
    [rows, cols] tensor, timed with the differentiation forward's outputs) or
    "axis" (x contiguous, reduced along `dim`, with the same outputs)."""
    d = dtype_name(x)
    c = pr_config()
    nseg = offsets.numel() - 1 if offsets is not None else 0
    inner = 0
    if kind == "rows":
        if x.dim() != 2 or not x.is_contiguous():
            raise ValueError("autotune('rows') needs a contiguous 2-D tensor")
        nseg = x.shape[0]
    if kind == "axis":
        if not x.is_contiguous():
            raise ValueError("autotune('axis') needs a contiguous tensor")
        outer, n, inner = axis_shape(tuple(x.shape), dim)
        nseg = outer
        check(pr_autotune_axis(_ptr(x), outer, n, inner, DTYPES[d], OPS[op], PRECISIONS[precision],
                               _stream(x, stream), ctypes.byref(c)))
        return c.as_dict()
    check(pr_autotune(KINDS[kind], _ptr(x), x.numel(), _ptr(offsets), nseg, DTYPES[d], OPS[op],
                      PRECISIONS[precision], _stream(x, stream), ctypes.byref(c)))
    return c.as_dict()
