"""Parity at the sizes the measurements are quoted on.

Every workload the benchmark times is run here at its full size, through the
same entry points and with the same launch shapes (the shipped tuning table,
or the autotuner where the benchmark runs it), and every result is compared
with the oracle:

  plain sweep   n = 2^28: fp32 sum / max / min (U[-1,1)), int32 sum / max /
                min (U[-2^20, 2^20)), uint32 and / or / xor (random bits, and
                all-ones / all-zeros inputs with planted bits at the head, the
                middle and the tail), fp64 product (U[0.999, 1.001)); the
                paper's own length n = 5 533 214; n = 2^30 + 5 (64-bit
                element offsets: 4 GiB of fp32 / int32)
  precision     bf16 and fp16 N(0,1) sums at n = 2^28 in all three precision
                modes; the ill-conditioned fp32 set (condition ~1e10) at 2^26
  batching      4096 log-uniform segments (about 3.15e8 fp32 values), sum and
                max, every segment, with the table's launch shape and after
                the autotuner, replayed from a CUDA graph
  prefix scan   n = 2^28: uint32 exclusive sum, int32 sum widening to int64,
                fp32 running max, every element
  any axis      the middle axis of [16, 4096, 4096] (sum; max with its index;
                the sum's gradient) and the first axis of [16384, 16384] (sum),
                1 GiB each, on sampled outputs

Integer, bitwise and max / min results are compared bit for bit; float sums
by their exact error against the bounds stated in include/pr.h (1e-6 sum|x|
plain, 2^-24 sum|x| compensated); the fp64 product by its relative error
against max(n - 1, 2) 2^-53.  The differentiation workload ([64, 2^20]) is checked
at full size in test_gpu_autograd.py.
"""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import values_of, same_float, sum_bound, prod_rel_bound

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 1 << 28


def dev(x):
    import torch
    a = np.ascontiguousarray(x)
    if a.dtype == np.float16:
        a = a.view(np.uint16)
    t = torch.from_numpy(a).cuda()
    return t


def run(t, dtype, op, precision="plain", out_dtype=None):
    import torch
    tt = t.view(pr.torch_dtype(dtype)) if t.dtype != pr.torch_dtype(dtype) else t
    out = pr.reduce(tt, op, precision=precision, out_dtype=out_dtype)
    torch.cuda.synchronize()
    return values_of(out, out_dtype or pr.out_dtype_name(dtype, op))[0]


def table_config_in_use(kind, dtype, op, precision, n):
    """The tuned configuration the benchmark's launch of this size uses (the
    binding loads the shipped table for this GPU), or None off that GPU."""
    import json
    import torch
    with open(pr.TUNING_PATH) as f:
        table = json.load(f)
    if table["gpu"] != torch.cuda.get_device_name():
        return None
    bucket = n.bit_length() - 1
    for e in table["entries"]:
        if (e["kind"], e["dtype"], e["op"], e["precision"], e["bucket"]) == \
                (pr.KINDS[kind], pr.DTYPES[dtype], pr.OPS[op], pr.PRECISIONS[precision], bucket):
            return {k: e[k] for k in ("block", "blocks_per_sm", "unroll", "vec_bytes")}
    return None


def assert_table_shape(kind, dtype, op, precision, n):
    want = table_config_in_use(kind, dtype, op, precision, n)
    if want is not None:
        assert pr.get_config(kind, dtype, op, precision, n) == want, (kind, dtype, op, precision)


# ---------------------------------------------------------------------------
# plain sweep at n = 2^28
# ---------------------------------------------------------------------------

def test_f32_sum_max_min_2e28():
    x = synth.uniform_f32(N, synth.config_seed(1))
    t = dev(x)
    for op in ("sum", "max", "min"):
        assert_table_shape("reduce", "f32", op, "plain", N)
    got = run(t, "f32", "sum")
    assert oracle.sum_error(x, "f32", got) <= sum_bound(x, "f32")
    for op in ("max", "min"):
        assert same_float(run(t, "f32", op), oracle.reduce(x, "f32", op)), op
    # planted extrema at the last element and the first
    t[N - 1] = 3.5
    t[0] = -3.5
    x[N - 1], x[0] = 3.5, -3.5
    assert run(t, "f32", "max") == oracle.reduce(x, "f32", "max") == 3.5
    assert run(t, "f32", "min") == oracle.reduce(x, "f32", "min") == -3.5


def test_i32_sum_max_min_2e28():
    x = synth.uniform_i32(N, synth.config_seed(1) + 100)
    t = dev(x)
    for op in ("sum", "max", "min"):
        assert_table_shape("reduce", "i32", op, "plain", N)
        assert run(t, "i32", op) == oracle.reduce(x, "i32", op), op
    k = N - 3                                             # planted in the ragged tail region
    t[k] = 2 ** 31 - 1
    x[k] = 2 ** 31 - 1
    assert run(t, "i32", "max") == oracle.reduce(x, "i32", "max") == 2 ** 31 - 1
    assert run(t, "i32", "sum") == oracle.reduce(x, "i32", "sum")


def test_u32_bitwise_2e28_random_and_planted():
    import torch
    x = synth.random_u32(N, synth.config_seed(1) + 200)
    t = dev(x.view(np.int32))
    for op in ("and", "or", "xor"):
        assert_table_shape("reduce", "u32", op, "plain", N)
        assert run(t, "u32", op) == oracle.reduce(x, "u32", op), op
    del t, x
    # random words give AND = 0 and OR = all ones with near certainty: plant
    # single bits at the head, the middle and the tail instead
    where = {0: 1 << 3, N // 2 + 1: 1 << 17, N - 1: 1 << 31}
    ones = np.full(N, 0xFFFFFFFF, dtype=np.uint32)
    for i, b in where.items():
        ones[i] ^= b
    t = dev(ones.view(np.int32))
    want = 0xFFFFFFFF ^ sum(where.values())
    assert run(t, "u32", "and") == oracle.reduce(ones, "u32", "and") == want
    assert run(t, "u32", "xor") == oracle.reduce(ones, "u32", "xor")
    del t, ones
    zeros = np.zeros(N, dtype=np.uint32)
    for i, b in where.items():
        zeros[i] = b
    t = dev(zeros.view(np.int32))
    assert run(t, "u32", "or") == oracle.reduce(zeros, "u32", "or") == sum(where.values())
    assert run(t, "u32", "xor") == oracle.reduce(zeros, "u32", "xor") == sum(where.values())
    torch.cuda.synchronize()


def test_f64_product_2e28():
    x = synth.uniform_f64(N, synth.config_seed(1) + 300)
    t = dev(x)
    assert_table_shape("reduce", "f64", "prod", "plain", N)
    got = run(t, "f64", "prod")
    want = oracle.reduce(x, "f64", "prod")
    assert want != 0.0 and abs(got - want) <= prod_rel_bound(N, "f64") * abs(want), (got, want)


def test_paper_length_5533214():
    n = synth.PAPER_N
    xi = synth.uniform_i32(n, 5533)
    xf = synth.uniform_f32(n, 5534)
    ti, tf = dev(xi), dev(xf)
    for op in ("sum", "max", "min"):
        assert run(ti, "i32", op) == oracle.reduce(xi, "i32", op)
    assert oracle.sum_error(xf, "f32", run(tf, "f32", "sum")) <= sum_bound(xf, "f32")
    for op in ("max", "min"):
        assert same_float(run(tf, "f32", op), oracle.reduce(xf, "f32", op))


def test_beyond_2e30_elements():
    """4 GiB inputs: element offsets above 2^31 bytes and 2^30 elements."""
    import torch
    n = (1 << 30) + 5
    iota = np.arange(n, dtype=np.int64)
    xi = (iota % (1 << 20)).astype(np.int32)
    t = dev(xi)
    assert run(t, "i32", "sum") == oracle.reduce(xi, "i32", "sum")
    t[n - 1] = 2 ** 31 - 1
    xi[n - 1] = 2 ** 31 - 1
    assert run(t, "i32", "max") == oracle.reduce(xi, "i32", "max") == 2 ** 31 - 1
    del t, xi
    xu = iota.astype(np.uint32)                          # i mod 2^32 = i here
    t = dev(xu.view(np.int32))
    assert run(t, "u32", "xor") == oracle.reduce(xu, "u32", "xor") == [n - 1, 1, n, 0][(n - 1) % 4]
    del t, xu, iota
    xf = synth.uniform_f32(n, 3030)
    t = dev(xf)
    assert oracle.sum_error(xf, "f32", run(t, "f32", "sum")) <= sum_bound(xf, "f32")
    t[n - 2] = 7.25
    xf[n - 2] = 7.25
    assert run(t, "f32", "max") == 7.25 == oracle.reduce(xf, "f32", "max")
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# precision forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_half_precision_sums_2e28(dtype):
    x = synth.normal_bf16(N, synth.config_seed(2)) if dtype == "bf16" else synth.normal_f16(N, synth.config_seed(2))
    t = dev(x)
    for precision in ("plain", "fp64_combine", "compensated"):
        assert_table_shape("reduce", dtype, "sum", precision, N)
        got = run(t, dtype, "sum", precision)
        assert oracle.sum_error(x, dtype, got) <= sum_bound(x, dtype, precision), (precision, got)
    # the fp64 value before the final rounding
    r64 = run(t, dtype, "sum", "compensated", out_dtype="f64")
    assert oracle.sum_error(x, dtype, r64) <= sum_bound(x, dtype, "compensated")


def test_ill_conditioned_2e26_all_precisions():
    x, n_big, exact = synth.ill_conditioned_f32(1 << 26, synth.config_seed(2))
    t = dev(x)
    a = oracle.abs_sum(x, "f32")
    assert oracle.exact_sum(x, "f32") == exact and 5e9 <= a / exact <= 2e10
    errs = {}
    for precision in ("plain", "fp64_combine", "compensated"):
        got = run(t, "f32", "sum", precision)
        errs[precision] = oracle.sum_error(x, "f32", got)
        assert errs[precision] <= sum_bound(x, "f32", precision), (precision, got)
    assert errs["compensated"] <= errs["fp64_combine"] <= errs["plain"]
    r64 = run(t, "f32", "sum", "compensated", out_dtype="f64")
    assert oracle.sum_error(x, "f32", r64) <= 2.0 ** -24 * a


# ---------------------------------------------------------------------------
# batching: the 4096-segment workload, every segment
# ---------------------------------------------------------------------------

def check_all_segments(x, off, op, got, argidx=None):
    for s in range(len(off) - 1):
        seg = x[off[s]:off[s + 1]]
        if op == "sum":
            assert oracle.sum_error(seg, "f32", got[s]) <= sum_bound(seg, "f32"), s
        else:
            v, i = oracle.argext(seg, "f32", op)
            assert same_float(got[s], v), s
            if argidx is not None:
                assert argidx[s] == i, s


def test_segmented_4096_log_uniform_every_segment():
    import torch
    vals, off = synth.segmented_workload(4096, synth.config_seed(3))
    assert 2.9e8 < vals.size < 3.4e8
    xv, ov = dev(vals), dev(off)
    for op in ("sum", "max"):
        old = pr.get_config("segmented", "f32", op, "plain", 4096)
        assert_table_shape("segmented", "f32", op, "plain", 4096)
        try:
            # the table's launch shape, called directly
            if op == "max":
                out, ai = pr.segmented_reduce(xv, ov, op, argidx=True)
                check_all_segments(vals, off, op, values_of(out, "f32"), ai.cpu().numpy())
            else:
                out = pr.segmented_reduce(xv, ov, op)
                check_all_segments(vals, off, op, values_of(out, "f32"))
            # what the benchmark times: the autotuner's choice, replayed from a graph
            cfg = pr.autotune("segmented", xv, op, offsets=ov)
            assert pr.get_config("segmented", "f32", op, "plain", 4096) == cfg
            res = torch.empty(4096, dtype=torch.float32, device="cuda")
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                pr.prepare(s)
                pr.check(pr.pr_segmented_reduce(xv.data_ptr(), ov.data_ptr(), 4096, 0, pr.OPS[op], res.data_ptr(),
                                                s.cuda_stream))
            s.synchronize()
            direct = res.clone()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                pr.check(pr.pr_segmented_reduce(xv.data_ptr(), ov.data_ptr(), 4096, 0, pr.OPS[op], res.data_ptr(),
                                                s.cuda_stream))
            res.fill_(float("nan"))
            for _ in range(2):
                g.replay()
            torch.cuda.synchronize()
            assert torch.equal(res.view(torch.int32), direct.view(torch.int32))
            check_all_segments(vals, off, op, values_of(res, "f32"))
            assert pr.last_device_error() == 0
        finally:
            pr.set_config("segmented", "f32", op, "plain", 4096, old)


# ---------------------------------------------------------------------------
# the next rows at their benchmark sizes: prefix scans of 2^28 elements and
# the 1 GiB axis reductions
# ---------------------------------------------------------------------------

def test_scans_2e28_every_element():
    import torch
    xi = synth.uniform_i32(N, synth.config_seed(6), 0, 1 << 8)     # counting-sort offsets
    t = dev(xi)
    y = pr.scan(t.view(torch.uint32), "sum", exclusive=True)
    got = y.view(torch.int32).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.scan(xi.view(np.uint32), "u32", "sum", True))
    del y, got
    y64 = pr.scan(t, "sum")
    assert np.array_equal(y64.cpu().numpy(), oracle.scan(xi, "i32", "sum", False))
    del y64, t
    xf = synth.normal_f32(N, synth.config_seed(6) + 1)
    yf = pr.scan(dev(xf), "max").cpu().numpy()
    assert np.array_equal(yf.astype(np.float64), oracle.scan(xf, "f32", "max", False))


def test_axis_1gib_shapes_sampled_outputs():
    import torch
    shape = (16, 4096, 4096)
    x = synth.normal_f32(16 * 4096 * 4096, synth.config_seed(5))
    t = dev(x).view(*shape)
    s = pr.reduce_axis(t, "sum", 1).cpu().numpy()
    m, ai = pr.reduce_axis(t, "max", 1, argidx=True)
    m, ai = m.cpu().numpy(), ai.cpu().numpy()
    xs = x.reshape(shape)
    rng = np.random.default_rng(5)
    picks = [(0, 0), (15, 4095), (7, 2048)] + [tuple(v) for v in zip(rng.integers(0, 16, 61), rng.integers(0, 4096, 61))]
    for p, q in picks:
        col = np.ascontiguousarray(xs[p, :, q])
        assert oracle.sum_error(col, "f32", float(s[p, q])) <= sum_bound(col, "f32"), (p, q)
        assert oracle.argext(col, "f32", "max") == (float(m[p, q]), int(ai[p, q])), (p, q)
    g = torch.from_numpy(synth.normal_f32(16 * 4096, 55).reshape(16, 4096)).cuda()
    gi = pr.reduce_axis_backward("sum", t, 1, g)
    assert torch.equal(gi, g[:, None, :].expand(shape))
    del t, gi
    c = synth.normal_f32(16384 * 16384, synth.config_seed(5) + 1)
    tc = dev(c).view(16384, 16384)
    cs = pr.reduce_axis(tc, "sum", 0).cpu().numpy()
    cm = c.reshape(16384, 16384)
    for q in [0, 1, 8191, 16383] + list(rng.integers(0, 16384, 28)):
        col = np.ascontiguousarray(cm[:, q])
        assert oracle.sum_error(col, "f32", float(cs[q])) <= sum_bound(col, "f32"), q
