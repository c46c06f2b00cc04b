"""pr_reduce_noalloc: the plain reduction for callers that cannot allocate
device memory (memory pools or arenas that own every allocation,
allocation-free real-time paths).  Its scratch is a static device array shared
by every call, so this file checks two calls in a row against pr_reduce on the
same data, through the C ABI.  It is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, same_float, sum_bound

pytestmark = pytest.mark.gpu

CASES = [("f32", "sum", synth.uniform_f32), ("f32", "max", synth.uniform_f32), ("bf16", "sum", None),
         ("f64", "prod", synth.uniform_f64), ("i32", "sum", synth.uniform_i32), ("u32", "xor", synth.random_u32),
         ("i64", "min", synth.random_i64)]


def _data(dtype, gen, n, seed):
    if dtype == "bf16":
        return synth.f32_to_bf16_bits(synth.normal_f32(n, seed))
    return gen(n, seed)


def _via(fn, t, dtype, op):
    import torch
    od = pr.out_dtype_name(dtype, op)
    out = torch.empty((), dtype=pr.torch_dtype(od), device=t.device)
    st = torch.cuda.current_stream().cuda_stream
    pr.check(fn(t.data_ptr(), t.numel(), pr.DTYPES[dtype], pr.OPS[op], out.data_ptr(), st))
    torch.cuda.synchronize()
    return values_of(out, od)[0]


@pytest.mark.parametrize("dtype,op,gen", CASES)
@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (4097, 1), ((1 << 22) + 5, 3), (1 << 26, 0)])
def test_noalloc_matches_pr_reduce_twice(dtype, op, gen, n, offset):
    x = _data(dtype, gen, n, 1000 + n)
    t = to_device(x, dtype, offset)
    ref = _via(pr.pr_reduce, t, dtype, op)
    for _ in range(2):                                   # the shared scratch is reused
        got = _via(pr.pr_reduce_noalloc, t, dtype, op)
        if dtype in ("i32", "u32", "i64") or op in ("max", "min"):
            assert (got == ref) if isinstance(ref, int) else same_float(got, ref)
        elif op == "sum":
            bound = sum_bound(x, dtype) if n else 0.0
            assert abs(got - ref) <= bound and oracle.sum_error(x, dtype, got) <= bound
        else:
            assert abs(got - ref) <= max(n - 1, 1) * 2.0 ** -53 * abs(ref)


def test_noalloc_rejects_bad_arguments():
    assert pr.pr_reduce_noalloc(None, 5, 0, 0, 0x10000, None) == 1
    assert pr.pr_reduce_noalloc(0x10000, 5, 0, pr.OPS["xor"], 0x10000, None) == 2
