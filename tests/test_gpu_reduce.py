"""Parity of the plain reduction (pr_reduce / pr_reduce_ex) with the oracle.

Integer, bitwise and max/min results must be bit-exact; float sums must lie
within the stated bound of the exact sum; products within (n-1) ulps."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, same_float, sum_bound, prod_rel_bound, guarded_like

pytestmark = pytest.mark.gpu

PAIRS = [(d, o) for d in ("f32", "f16", "bf16", "f64", "i32", "u32", "i64")
         for o in ("sum", "prod", "max", "min", "and", "or", "xor") if oracle.supported(d, o)]
SIZES = [0, 1, 2, 7, 31, 32, 33, 255, 4095, 65537, (1 << 20) + 3]


def gen(dtype, op, n, seed):
    """Inputs shaped like the sweep workloads.  Product inputs lie in 1 +- 2^-7
    (fp64: [0.999, 1.001]) so that for n <= 2^20 no partial product in any
    order leaves the normal range of the accumulation type."""
    near1 = (1.0 - 2.0 ** -7, 1.0 + 2.0 ** -7)
    if dtype == "f32":
        return synth.uniform_f32(n, seed, *near1) if op == "prod" else synth.uniform_f32(n, seed)
    if dtype == "f64":
        return synth.uniform_f64(n, seed) if op == "prod" else synth.uniform_f64(n, seed, -1.0, 1.0)
    if dtype == "bf16":
        v = synth.uniform_f32(n, seed, *near1) if op == "prod" else synth.normal_f32(n, seed)
        return synth.f32_to_bf16_bits(v)
    if dtype == "f16":
        v = synth.uniform_f32(n, seed, *near1) if op == "prod" else synth.normal_f32(n, seed)
        return v.astype(np.float16)
    if dtype == "i32":
        return synth.uniform_i32(n, seed)
    if dtype == "u32":
        return synth.random_u32(n, seed)
    return synth.random_i64(n, seed)


def check(x, dtype, op, got, precision="plain"):
    if dtype in oracle.INT_DTYPES:
        assert got == oracle.reduce(x, dtype, op)
    elif op in ("max", "min"):
        assert same_float(got, oracle.reduce(x, dtype, op))
    elif op == "sum":
        err = oracle.sum_error(x, dtype, got)
        assert err <= sum_bound(x, dtype, precision), (err, sum_bound(x, dtype, precision))
    else:
        want = oracle.reduce(x, dtype, op)
        n = np.asarray(x).size
        if dtype in ("f16", "bf16"):
            dtype = "f32"
        assert abs(got - want) <= prod_rel_bound(n, dtype) * abs(want), (got, want)


def run(x, dtype, op, offset=0, precision="plain", out_dtype=None):
    """The reduction of x, written into a canary-guarded output."""
    t = to_device(x, dtype, offset)
    od = out_dtype or pr.out_dtype_name(dtype, op)
    g = guarded_like((), od)
    pr.reduce(t, op, precision=precision, out_dtype=out_dtype, out=g.tensor)
    return values_of(g.check(), od)[0]


@pytest.mark.parametrize("dtype,op", PAIRS)
def test_sizes(dtype, op):
    for k, n in enumerate(SIZES):
        x = gen(dtype, op, n, 100 + k)
        check(x, dtype, op, run(x, dtype, op))


@pytest.mark.parametrize("dtype,op", PAIRS)
@pytest.mark.parametrize("offset", [1, 3])
def test_misaligned_base(dtype, op, offset):
    for n in (5, 4097, 100003):
        x = gen(dtype, op, n, 7 * n + offset)
        check(x, dtype, op, run(x, dtype, op, offset=offset))


def test_identities_on_empty_input():
    for dtype, op in PAIRS:
        got = run(gen(dtype, op, 0, 1), dtype, op)
        want = oracle.identity(dtype, op)
        if isinstance(want, float):
            assert same_float(got, want), (dtype, op, got)
        else:
            od = oracle.out_dtype(dtype, op)
            mask = (1 << (64 if od == "i64" else 32)) - 1
            assert got & mask == want & mask, (dtype, op, got)


def test_integer_closed_forms():
    n = 5_533_214                                     # the paper's vector length
    iota = np.arange(n, dtype=np.int64)
    assert run(iota.astype(np.int32), "i32", "sum") == n * (n - 1) // 2
    assert run(iota.astype(np.uint32), "u32", "xor") == [n - 1, 1, n, 0][(n - 1) % 4]
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    assert run(perm, "i32", "min") == 0 and run(perm, "i32", "max") == n - 1
    c = np.full(n, 3, dtype=np.uint32)
    assert run(c, "u32", "prod") == pow(3, n, 2 ** 32)
    assert run(c, "u32", "xor") == (3 if n % 2 else 0)
    f = np.full(1 << 20, 0.25, dtype=np.float32)      # exact in any order
    assert run(f, "f32", "sum") == 0.25 * (1 << 20)


@pytest.mark.parametrize("where", [0, 1, 4095, 65535, -2, -1])
def test_planted_bits_and_extrema(where):
    n = (1 << 20) + 3
    ones = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    zeros = np.zeros(n, dtype=np.uint32)
    bit = 1 << (abs(where) % 32)
    assert run(synth.plant(ones, where, 0xFFFFFFFF ^ bit), "u32", "and") == 0xFFFFFFFF ^ bit
    assert run(synth.plant(zeros, where, bit), "u32", "or") == bit
    assert run(synth.plant(zeros, where, bit), "u32", "xor") == bit
    x = synth.uniform_f32(n, 5)
    assert run(synth.plant(x, where, 3.5), "f32", "max") == 3.5
    assert run(synth.plant(x, where, -3.5), "f32", "min") == -3.5
    xi = synth.uniform_i32(n, 6)
    assert run(synth.plant(xi, where, 2 ** 31 - 1), "i32", "max") == 2 ** 31 - 1
    assert run(synth.plant(xi, where, -2 ** 31), "i32", "min") == -2 ** 31


def test_float_special_values():
    n = 100003
    x = synth.uniform_f32(n, 9)
    for op in ("sum", "max", "min", "prod"):
        got = run(synth.plant(x, 777, np.nan), "f32", op)
        assert math.isnan(got), op
    assert run(synth.plant(x, 5, np.inf), "f32", "sum") == math.inf
    assert run(synth.plant(x, 5, np.inf), "f32", "max") == math.inf
    assert math.isnan(run(synth.plant(synth.plant(x, 5, np.inf), 9, -np.inf), "f32", "sum"))
    z = np.zeros(n, dtype=np.float32)
    z[::2] = -0.0
    assert same_float(run(z, "f32", "max"), 0.0)
    assert same_float(run(z, "f32", "min"), -0.0)
    assert same_float(run(np.full(n, -0.0, np.float32), "f32", "max"), -0.0)
    d = synth.uniform_f64(n, 3)
    assert math.isnan(run(synth.plant(d, 11, np.nan), "f64", "max"))
    assert same_float(run(synth.plant(d, 11, -0.0), "f64", "prod"), -0.0)
    assert run(synth.plant(d, 11, -np.inf), "f64", "prod") == -math.inf
    assert math.isnan(run(synth.plant(synth.plant(d, 11, np.inf), 12, 0.0), "f64", "prod"))
    h = synth.normal_f32(n, 4).astype(np.float16)
    assert math.isnan(run(synth.plant(h, 3, np.float16(np.nan)), "f16", "max"))


def test_f64_product_extended_range_and_subnormals():
    # 2^1000 * 2^1000 * 2^-1000 * 2^-1000 ... : no intermediate overflow
    x = np.array([2.0 ** 1000, 2.0 ** 1000, 2.0 ** -1000, 2.0 ** -999] * 1000, dtype=np.float64)
    assert run(x, "f64", "prod") == oracle.reduce(x, "f64", "prod") == 2.0 ** 1000
    s = np.array([5e-324, 2.0 ** 1000, 2.0 ** 74, 3.0] * 3, dtype=np.float64)   # 2^-1074 is subnormal
    assert run(s, "f64", "prod") == oracle.reduce(s, "f64", "prod") == 27.0
    r = synth.uniform_f64(1 << 20, 12)
    got, want = run(r, "f64", "prod"), oracle.reduce(r, "f64", "prod")
    # half the factors multiply on the fp64 pipe (each within 2^-53), half on
    # the integer pipes (each within 2^-61): inside (n - 1) * 2^-53
    assert abs(got - want) <= prod_rel_bound(r.size, "f64") * abs(want)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("precision", ["plain", "fp64_combine", "compensated"])
def test_precision_modes(dtype, precision):
    n = (1 << 20) + 5
    x = gen(dtype, "sum", n, 21)
    check(x, dtype, "sum", run(x, dtype, "sum", precision=precision), precision)
    if precision != "plain":
        r64 = run(x, dtype, "sum", precision=precision, out_dtype="f64")
        assert oracle.sum_error(x, dtype, r64) <= sum_bound(x, dtype, precision)


def test_ill_conditioned_compensated_vs_plain():
    x, n_big, exact = synth.ill_conditioned_f32(1 << 22, 22)
    a = oracle.abs_sum(x, "f32")
    errs = {}
    for precision in ("plain", "fp64_combine", "compensated"):
        r = run(x, "f32", "sum", precision=precision, out_dtype="f64" if precision != "plain" else None)
        errs[precision] = oracle.sum_error(x, "f32", r)
    assert errs["plain"] <= 1e-6 * a
    assert errs["compensated"] <= 2.0 ** -24 * a
    assert errs["compensated"] <= errs["plain"]


def test_deterministic_repeats():
    x = to_device(synth.uniform_f32((1 << 22) + 1, 31), "f32")
    import torch
    first = pr.reduce(x, "sum").cpu().view(torch.int32).item()
    for _ in range(20):
        assert pr.reduce(x, "sum").cpu().view(torch.int32).item() == first
    c = to_device(synth.normal_f32(1 << 21, 32), "f32")
    a = [pr.reduce(c, "sum", precision="compensated", out_dtype="f64").item() for _ in range(5)]
    assert len(set(a)) == 1


def test_every_config_variant_agrees_with_oracle():
    x = synth.uniform_f32((1 << 20) + 7, 41)
    t = to_device(x, "f32", offset=1)
    old = pr.get_config("reduce", "f32", "sum", "plain", t.numel())
    try:
        for block in (128, 256, 1024):
            for bps in (1, 2):
                for unroll in (2, 4):
                    for vb in (16, 32):
                        pr.set_config("reduce", "f32", "sum", "plain", t.numel(),
                                      dict(block=block, blocks_per_sm=bps, unroll=unroll, vec_bytes=vb))
                        got = values_of(pr.reduce(t, "sum"), "f32")[0]
                        check(x, "f32", "sum", got)
    finally:
        pr.set_config("reduce", "f32", "sum", "plain", t.numel(), old)


def test_graph_capture_replays_plain_reduce():
    import torch
    x = to_device(synth.uniform_f32(1 << 20, 51), "f32")
    out = torch.empty((), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pr.prepare(s)
        pr.reduce(x, "max", out=out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pr.reduce(x, "max", out=out, stream=s)
    x.fill_(0.0)
    x[123] = 7.0
    g.replay()
    torch.cuda.synchronize()
    assert out.item() == 7.0


NP = {"f32": np.float32, "i32": np.int32, "u32": np.uint32, "f64": np.float64}


def test_host_memory_path():
    import torch
    for dtype, op in (("f32", "sum"), ("i32", "sum"), ("u32", "xor"), ("f64", "prod")):
        n = (100 << 20) // np.dtype(NP[dtype]).itemsize + 3     # two 64 MiB chunks
        x = gen(dtype, op, n, 61)
        t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        got = pr.reduce_host(t, op)
        if dtype == "f32":
            assert oracle.sum_error(x, "f32", got) <= sum_bound(x, "f32")
        elif dtype == "f64":
            want = oracle.reduce(x, "f64", "prod")
            assert abs(got - want) <= prod_rel_bound(n, "f64") * abs(want)
        else:
            od = oracle.out_dtype(dtype, op)
            want = oracle.reduce(x, dtype, op)
            mask = (1 << (64 if od == "i64" else 32)) - 1
            assert got & mask == want & mask
    big = synth.uniform_i32((200 << 20) // 4 + 11, 62)       # four chunks
    assert pr.reduce_host(torch.from_numpy(big).pin_memory(), "sum") == oracle.reduce(big, "i32", "sum")


ARG_DTYPES = ["f32", "f16", "bf16", "f64", "i32", "u32", "i64"]


@pytest.mark.parametrize("dtype", ARG_DTYPES)
@pytest.mark.parametrize("op", ["max", "min"])
def test_reduce_arg_first_index(dtype, op):
    """Whole-array arg-extremum: the extremum and its first index, with ties."""
    for k, (n, offset) in enumerate([(0, 0), (1, 0), (37, 1), (4097, 3), ((1 << 20) + 3, 0), (5_533_214, 1)]):
        if dtype in ("i32", "u32", "i64"):
            x = {"i32": synth.uniform_i32(n, k, -50, 50), "u32": synth.uniform_i32(n, k, 0, 100).astype(np.uint32),
                 "i64": synth.uniform_i32(n, k, -50, 50).astype(np.int64)}[dtype]
        else:
            x = gen(dtype, "max", n, k)
        if n > 10:                       # plant a tie for the extremum: two positions, first must win
            v = oracle.argext(x, dtype, op)[0]
            x = np.array(x, copy=True)
            x.reshape(-1)[n // 3] = x.reshape(-1)[oracle.argext(x, dtype, op)[1]]
        t = to_device(x, dtype, offset)
        gv, gi = guarded_like((), pr.out_dtype_name(dtype, op)), guarded_like((), "i64")
        val, idx = pr.reduce_arg(t, op, out=gv.tensor, idx=gi.tensor)
        gv.check(), gi.check()
        wv, wi = oracle.argext(x, dtype, op)
        got = values_of(val, pr.out_dtype_name(dtype, op))[0]
        assert int(idx.item()) == wi, (n, int(idx.item()), wi)
        if isinstance(got, int):
            assert got == int(wv)
        else:
            assert same_float(got, wv)


def test_reduce_arg_nan_and_signed_zero():
    x = synth.uniform_f32(100003, 3)
    x[[50000, 77]] = np.nan
    v, i = pr.reduce_arg(to_device(x, "f32"), "max")
    assert math.isnan(v.item()) and i.item() == 77
    z = np.zeros(10001, np.float32)
    z[:5000] = -0.0
    v, i = pr.reduce_arg(to_device(z, "f32"), "max")
    assert same_float(v.item(), 0.0) and i.item() == 5000
    v, i = pr.reduce_arg(to_device(z, "f32"), "min")
    assert same_float(v.item(), -0.0) and i.item() == 0


@pytest.mark.parametrize("dtype,op,precision", [("f32", "sum", "plain"), ("f32", "sum", "compensated"),
                                                ("f32", "max", "plain"), ("bf16", "sum", "compensated"),
                                                ("i32", "sum", "plain"), ("u32", "xor", "plain"),
                                                ("f64", "prod", "plain")])
@pytest.mark.parametrize("nbytes", [4, 4096, 65536])
def test_small_inputs_run_as_one_block(dtype, op, precision, nbytes):
    """Inputs of at most 64 KiB: one block, which finishes without the
    ticket; results as the oracle's, misaligned too, and the same bits on a
    repeat.  (One byte more is a multi-block launch.)"""
    import torch
    es = {"f32": 4, "bf16": 2, "i32": 4, "u32": 4, "f64": 8}[dtype]
    n = nbytes // es
    gen = {"f32": lambda m, s: synth.uniform_f32(m, s), "bf16": synth.normal_bf16, "i32": synth.uniform_i32,
           "u32": synth.random_u32, "f64": synth.uniform_f64}[dtype]
    x = gen(n, 60 + n % 7)
    for offset in (0, 1):
        t = to_device(x, dtype, offset)
        assert pr.reduce_plan(t, op, precision=precision)["grid"] == 1
        od = "f32" if (dtype == "bf16" and op == "sum") else pr.out_dtype_name(dtype, op)
        got = values_of(pr.reduce(t, op, precision=precision), od)[0]
        assert values_of(pr.reduce(t, op, precision=precision), od)[0] == got
        if op == "sum" and dtype in ("f32", "bf16"):
            assert oracle.sum_error(x, dtype, got) <= sum_bound(x, dtype, precision)
        elif op == "prod":
            want = oracle.reduce(x, dtype, op)
            assert abs(got - want) <= prod_rel_bound(n, dtype) * abs(want)
        elif dtype == "f32":
            assert same_float(got, oracle.reduce(x, dtype, op))
        else:
            assert got == oracle.reduce(x, dtype, op)
    if dtype == "f32" and op == "max":
        v, i = pr.reduce_arg(to_device(x, dtype), "max")
        assert pr.reduce_plan(to_device(x, dtype), "max", arg=True)["grid"] == 1
        wv, wi = oracle.argext(x, "f32", "max")
        assert float(v.item()) == wv and int(i.item()) == wi
    big = to_device(gen(n + 64 // es + 1, 61), dtype)
    assert pr.reduce_plan(big, op, precision=precision)["grid"] > 1 or nbytes < 65536
