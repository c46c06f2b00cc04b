"""CPU oracle for the parallel reduction (Section 1.1, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The product path never imports this package and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain sequential loops, exact or
extended-precision accumulation); this module only marshals numpy arrays.
The line search built on the reduction (golden-section and Fibonacci search
of the Beckmann objective) is plain float64 Python in ``linesearch.py``.

Dtype names: f32 f16 bf16 f64 i32 u32 i64.  bf16 and f16 arrays are passed as
their 16-bit patterns (``uint16``; an ``np.float16`` array is viewed as such).
Combiner names: sum prod max min and or xor.

Output types (the reduction's result type for each input type):
  f32 -> f32;  f16/bf16: sum,prod -> f32, max,min -> same type;  f64 -> f64;
  i32: sum -> i64, others -> i32;  u32 -> u32 (sum/prod wrap mod 2^32);
  i64 -> i64 (sum/prod wrap mod 2^64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPES = {"f32": 0, "f16": 1, "bf16": 2, "f64": 3, "i32": 4, "u32": 5, "i64": 6}
OPS = {"sum": 0, "prod": 1, "max": 2, "min": 3, "and": 4, "or": 5, "xor": 6}
FLOAT_DTYPES = ("f32", "f16", "bf16", "f64")
INT_DTYPES = ("i32", "u32", "i64")
_NP_STORAGE = {"f32": np.float32, "f16": np.uint16, "bf16": np.uint16, "f64": np.float64,
               "i32": np.int32, "u32": np.uint32, "i64": np.int64}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, ISO C, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC) or _foreign(_LIB):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _foreign(path):
    """True if path is an ELF shared object for another CPU architecture."""
    import platform
    want = {"x86_64": 62, "aarch64": 183}.get(platform.machine())
    with open(path, "rb") as f:
        head = f.read(20)
    return want is not None and head[:4] == b"\x7fELF" and int.from_bytes(head[18:20], "little") != want


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        PD, PI64 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        sig = {
            "orc_exact_sum": (D, [P, I64, I]),
            "orc_exact_abs_sum": (D, [P, I64, I]),
            "orc_exact_sum_minus": (D, [P, I64, I, D]),
            "orc_sum_f64_loop": (D, [P, I64, I]),
            "orc_sum_f64_chunked": (D, [P, I64, I, I]),
            "orc_reduce_int": (I, [P, I64, I, I, P]),
            "orc_argext": (I, [P, I64, I, I, PD, PI64]),
            "orc_argext_int": (I, [P, I64, I, I, PI64]),
            "orc_maxmin": (D, [P, I64, I, I]),
            "orc_prod": (D, [P, I64, I]),
            "orc_prod_scaled": (I, [P, I64, I, PD, PI64]),
            "orc_prod_aux": (I, [P, I64, I, PD, PI64, PI64]),
            "orc_prod_except": (D, [P, I64, I, I64]),
            "orc_scan": (I, [P, I64, I, I, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
    return _lib


def _arr(x, dtype):
    """Contiguous array in this dtype's storage type (bf16/f16 as uint16 bit patterns)."""
    if dtype not in DTYPES:
        raise ValueError("unknown dtype %r" % (dtype,))
    a = np.asarray(x)
    if dtype == "f16" and a.dtype == np.float16:
        a = a.view(np.uint16)
    want = _NP_STORAGE[dtype]
    if a.dtype != want:
        raise TypeError("dtype %s expects numpy %s storage, got %s" % (dtype, np.dtype(want), a.dtype))
    return np.ascontiguousarray(a.reshape(-1))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def out_dtype(dtype: str, op: str) -> str:
    if dtype in ("f16", "bf16"):
        return dtype if op in ("max", "min") else "f32"
    if dtype == "i32" and op == "sum":
        return "i64"
    return dtype


def supported(dtype: str, op: str) -> bool:
    return not (dtype in FLOAT_DTYPES and op in ("and", "or", "xor"))


def identity(dtype: str, op: str):
    """The combiner's neutral element in the output type (value an empty reduction yields)."""
    od = out_dtype(dtype, op)
    if op == "sum":
        return 0.0 if od in FLOAT_DTYPES else 0
    if op == "prod":
        return 1.0 if od in FLOAT_DTYPES else 1
    if op in ("or", "xor"):
        return 0
    if op == "and":
        return {"i32": -1, "u32": 0xFFFFFFFF, "i64": -1}[od]
    big = {"i32": (-(2 ** 31), 2 ** 31 - 1), "u32": (0, 2 ** 32 - 1), "i64": (-(2 ** 63), 2 ** 63 - 1)}
    if od in FLOAT_DTYPES:
        return float("-inf") if op == "max" else float("inf")
    lo, hi = big[od]
    return lo if op == "max" else hi


# ---------------------------------------------------------------------------
# Reductions (Section 1.1: x_0 (x) x_1 (x) ... (x) x_{n-1}; Algorithm 1's loop)
# ---------------------------------------------------------------------------

def reduce(x, dtype: str, op: str):
    """The reduction's defined value.

    integer / bitwise: exact, as a Python int of the output type;
    float max/min:     exact (an input element), as a Python float;
    float sum:         the exact sum rounded once to double;
    float prod:        the product in double-double with a separate exponent,
                       rounded once to double.
    """
    if not supported(dtype, op):
        raise ValueError("combiner %s is not defined on %s" % (op, dtype))
    a = _arr(x, dtype)
    n, d = a.size, DTYPES[dtype]
    L = _L()
    if dtype in INT_DTYPES:
        od = out_dtype(dtype, op)
        buf = (ctypes.c_uint8 * 8)()
        if L.orc_reduce_int(_ptr(a), n, d, OPS[op], ctypes.cast(buf, ctypes.c_void_p)) != 0:
            raise ValueError("bad combiner")
        raw = bytes(buf)
        if od == "i64":
            return int.from_bytes(raw[:8], "little", signed=True)
        if od == "i32":
            return int.from_bytes(raw[:4], "little", signed=True)
        return int.from_bytes(raw[:4], "little", signed=False)
    if op == "sum":
        return L.orc_exact_sum(_ptr(a), n, d)
    if op == "prod":
        return L.orc_prod(_ptr(a), n, d)
    return L.orc_maxmin(_ptr(a), n, d, OPS[op])


def sum_f64_loop(x, dtype: str) -> float:
    """Algorithm 1 verbatim: a double accumulator, elements added in index order."""
    a = _arr(x, dtype)
    return _L().orc_sum_f64_loop(_ptr(a), a.size, DTYPES[dtype])


def sum_f64_chunked(x, dtype: str, threads: int) -> float:
    """Algorithm 1 per contiguous chunk on `threads` host threads (double
    accumulators), the chunk sums added in chunk order: the multi-core CPU
    baseline.  The C loops run with the GIL released."""
    a = _arr(x, dtype)
    return _L().orc_sum_f64_chunked(_ptr(a), a.size, DTYPES[dtype], int(threads))


def exact_sum(x, dtype: str) -> float:
    a = _arr(x, dtype)
    return _L().orc_exact_sum(_ptr(a), a.size, DTYPES[dtype])


def abs_sum(x, dtype: str) -> float:
    """sum_i |x_i|, exact then rounded once (the scale of every sum tolerance)."""
    a = _arr(x, dtype)
    return _L().orc_exact_abs_sum(_ptr(a), a.size, DTYPES[dtype])


def sum_error(x, dtype: str, r: float) -> float:
    """|sum_i x_i - r|, computed exactly and rounded once."""
    a = _arr(x, dtype)
    return abs(_L().orc_exact_sum_minus(_ptr(a), a.size, DTYPES[dtype], float(r)))


def argext(x, dtype: str, op: str):
    """(extremum, index of its first occurrence); NaN is the extremum of both
    max and min, -0 < +0.  Empty input gives (identity, -1)."""
    assert op in ("max", "min")
    a = _arr(x, dtype)
    L = _L()
    idx = ctypes.c_int64(-1)
    if dtype in INT_DTYPES:
        L.orc_argext_int(_ptr(a), a.size, DTYPES[dtype], OPS[op], ctypes.byref(idx))
        return (reduce(a, dtype, op), idx.value)
    v = ctypes.c_double(0.0)
    L.orc_argext(_ptr(a), a.size, DTYPES[dtype], OPS[op], ctypes.byref(v), ctypes.byref(idx))
    return (v.value, idx.value)


def prod_scaled(x, dtype: str):
    """Product as (significand in +-[0.5,1), exponent); finite non-zero inputs only."""
    a = _arr(x, dtype)
    m, e = ctypes.c_double(0), ctypes.c_int64(0)
    if _L().orc_prod_scaled(_ptr(a), a.size, DTYPES[dtype], ctypes.byref(m), ctypes.byref(e)) != 0:
        raise ValueError("prod_scaled needs finite non-zero inputs")
    return m.value, e.value


def prod_aux(x, dtype: str):
    """(product of the non-zero elements, number of zeros, index of the first zero or -1)."""
    a = _arr(x, dtype)
    p, zc, zi = ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _L().orc_prod_aux(_ptr(a), a.size, DTYPES[dtype], ctypes.byref(p), ctypes.byref(zc), ctypes.byref(zi))
    return p.value, zc.value, zi.value


def prod_except(x, dtype: str, i: int) -> float:
    """prod_{j != i} x_j (the derivative of the product with respect to x_i)."""
    a = _arr(x, dtype)
    return _L().orc_prod_except(_ptr(a), a.size, DTYPES[dtype], int(i))


# ---------------------------------------------------------------------------
# Segmented form: the same reduction over each x[off[s]:off[s+1]]
# ---------------------------------------------------------------------------

def segmented(x, offsets, dtype: str, op: str):
    """List of per-segment results (reduce() of each slice; identity if empty)."""
    a = _arr(x, dtype)
    off = np.asarray(offsets, dtype=np.int64)
    out = []
    for s in range(off.size - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        out.append(reduce(a[lo:hi], dtype, op) if hi > lo else identity(dtype, op))
    return out


def segmented_argext(x, offsets, dtype: str, op: str):
    """Per segment (extremum, first index within the segment)."""
    a = _arr(x, dtype)
    off = np.asarray(offsets, dtype=np.int64)
    return [argext(a[int(off[s]):int(off[s + 1])], dtype, op) for s in range(off.size - 1)]


# ---------------------------------------------------------------------------
# Prefix scan
# ---------------------------------------------------------------------------

def scan(x, dtype: str, op: str, exclusive: bool = False):
    """Prefix combinations of x in index order: y[i] = x[0] op ... op x[i]
    (inclusive) or x[0] op ... op x[i-1] (exclusive, y[0] = identity).
    Integer and bitwise combiners (y in the output type: int64 for an int32
    sum) and float max / min (y as float64 values)."""
    a = _arr(x, dtype)
    n = a.size
    if dtype in INT_DTYPES:
        od = out_dtype(dtype, op)
        y = np.zeros(n, dtype={"i64": np.int64, "i32": np.int32, "u32": np.uint32}[od])
    else:
        if op not in ("max", "min"):
            raise ValueError("the float scan is defined for max and min")
        y = np.zeros(n, dtype=np.float64)
    if n and _L().orc_scan(_ptr(a), n, DTYPES[dtype], OPS[op], int(bool(exclusive)), _ptr(y)) != 0:
        raise ValueError("bad combiner")
    return y


# ---------------------------------------------------------------------------
# Reduction along one axis of a contiguous [outer, n, inner] array
# ---------------------------------------------------------------------------

def axis_slices(x, dtype: str, outer: int, n: int, inner: int):
    """The outer*inner columns x[p, :, q] as contiguous arrays, output order (p, q)."""
    a = _arr(x, dtype).reshape(outer, n, inner)
    for p in range(outer):
        for q in range(inner):
            yield np.ascontiguousarray(a[p, :, q])


def axis(x, dtype: str, op: str, outer: int, n: int, inner: int):
    """out[p*inner + q] = reduce(x[p, :, q]) (the identity when n == 0)."""
    return [reduce(c, dtype, op) if n else identity(dtype, op) for c in axis_slices(x, dtype, outer, n, inner)]


def axis_argext(x, dtype: str, op: str, outer: int, n: int, inner: int):
    """Per output (extremum, first index i along the axis)."""
    return [argext(c, dtype, op) for c in axis_slices(x, dtype, outer, n, inner)]


# ---------------------------------------------------------------------------
# Gradients of a reduction along the last dimension of a [rows, cols] array
# ---------------------------------------------------------------------------

def grad(x, dtype: str, op: str, g):
    """d(reduce(x[r,:]))/dx[r,c] * g[r] for every element, in float64.

    sum:     g[r]
    max/min: g[r] at the first index of the extremum, 0 elsewhere
    prod:    g[r] * prod_{j != c} x[r,j]
    """
    a = np.asarray(x)
    if a.ndim == 1:
        a = a.reshape(1, -1)
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    rows, cols = a.shape
    out = np.zeros((rows, cols), dtype=np.float64)
    for r in range(rows):
        row = np.ascontiguousarray(a[r])
        if op == "sum":
            out[r, :] = g[r]
        elif op in ("max", "min"):
            _, i = argext(row, dtype, op)
            if i >= 0:
                out[r, i] = g[r]
        elif op == "prod":
            for c in range(cols):
                out[r, c] = g[r] * prod_except(row, dtype, c)
        else:
            raise ValueError("no gradient for %s" % op)
    return out
