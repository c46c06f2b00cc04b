"""Helpers for the GPU parity tests: move seeded numpy inputs to the device
(optionally misaligned by a few elements), read outputs back bit-exactly and
state the tolerances every float comparison uses."""
import math

import numpy as np

import oracle

NP_STORAGE = {"f32": np.float32, "f16": np.uint16, "bf16": np.uint16, "f64": np.float64,
              "i32": np.int32, "u32": np.uint32, "i64": np.int64}
TORCH_VIEW = {"f32": "float32", "f64": "float64", "i32": "int32", "u32": "int32", "i64": "int64",
              "f16": "int16", "bf16": "int16"}


def to_device(x, dtype, offset=0, device="cuda"):
    """CUDA tensor holding x, starting `offset` elements past a 256-byte boundary."""
    import torch
    from paper_1710_07358_gb300 import pr
    a = np.ascontiguousarray(x)
    if dtype == "f16" and a.dtype == np.float16:
        a = a.view(np.uint16)
    a = a.astype(NP_STORAGE[dtype], copy=False)
    buf = np.zeros(a.size + offset, dtype=a.dtype)
    buf[offset:] = a
    raw = torch.from_numpy(buf.view(np.uint8)).to(device)
    es = a.dtype.itemsize
    t = raw[offset * es:]
    tdt = pr.torch_dtype(dtype)
    return t.view(tdt) if a.size else torch.empty(0, dtype=tdt, device=device)


def bits_of(t, dtype):
    """numpy array with the output's storage bits (host)."""
    import torch
    v = t.reshape(-1).view(getattr(torch, TORCH_VIEW[dtype])).cpu().numpy()
    return v.view(NP_STORAGE[dtype])


def values_of(t, dtype):
    """Python values: ints for integer types, exact floats for float types."""
    b = bits_of(t, dtype)
    if dtype == "bf16":
        return [float(v) for v in (b.astype(np.uint32) << 16).view(np.float32)]
    if dtype == "f16":
        return [float(v) for v in b.view(np.float16)]
    if dtype in ("f32", "f64"):
        return [float(v) for v in b]
    return [int(v) for v in b]


def same_float(a, b):
    """Equal as values, NaN equal to NaN, and the sign of zero must agree."""
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return a == b and math.copysign(1.0, a) == math.copysign(1.0, b)


def sum_bound(x, dtype, precision="plain"):
    """|computed - exact| allowed for a float sum of x.

    fp32/fp16/bf16, plain or fp64-combine: 1e-6 * sum|x| (fp32 accumulation);
    compensated: 2^-24 * sum|x| (one final rounding to fp32 dominates);
    fp64 input: (n-1) * 2^-53 * sum|x|, the worst case of any order."""
    a = oracle.abs_sum(x, dtype)
    n = np.asarray(x).size
    if dtype == "f64":
        return max(n - 1, 1) * 2.0 ** -53 * a
    if precision == "compensated":
        return 2.0 ** -24 * a
    return 1e-6 * a


def prod_rel_bound(n, dtype):
    """Relative error allowed for a product of n values: (n-1) units in the last
    place of the accumulation type (the worst case of any evaluation order);
    fp64 products also round once converting their 64-bit significand to
    double, covered by max(n - 1, 2)."""
    if dtype == "f64":
        return max(n - 1, 2) * 2.0 ** -53
    return max(n - 1, 1) * 2.0 ** -24


# ---------------------------------------------------------------------------
# Canaries: device output buffers with guard bytes before and after them
# ---------------------------------------------------------------------------

GUARD = 256          # bytes on each side; keeps the buffer 256-byte aligned
CANARY = 0xA5


class Guarded:
    """A device output tensor of `shape` / torch `dtype` inside a larger byte
    buffer whose GUARD bytes before and after it hold CANARY.  check() fails
    if a kernel wrote outside the tensor (the compute-sanitizer substitute
    for writes past out, y, grad_in, argidx and aux)."""

    def __init__(self, shape, dtype, device="cuda", fill=None):
        import torch
        shape = tuple(shape) if isinstance(shape, (tuple, list)) else (int(shape),)
        numel = 1
        for v in shape:
            numel *= v
        self.nbytes = numel * torch.empty((), dtype=dtype).element_size()
        self.raw = torch.full((GUARD + self.nbytes + GUARD,), CANARY, dtype=torch.uint8, device=device)
        self.tensor = self.raw[GUARD:GUARD + self.nbytes].view(dtype).view(shape)
        if fill is not None:
            self.tensor.fill_(fill)

    def check(self):
        import torch
        torch.cuda.synchronize()
        head = self.raw[:GUARD]
        tail = self.raw[GUARD + self.nbytes:]
        assert bool(torch.all(head == CANARY)), "write before the output buffer"
        assert bool(torch.all(tail == CANARY)), "write past the end of the output buffer"
        return self.tensor


def guarded_like(shape, name):
    """Guarded output for one of the library's dtype names (f32, i64, ...)."""
    from paper_1710_07358_gb300 import pr
    import torch
    dt = pr.torch_dtype(name) if name != "aux" else torch.int8
    return Guarded(shape, dt)
