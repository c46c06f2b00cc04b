"""Parity of the one-pass prefix scan with the oracle, element by element."""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, bits_of, guarded_like

pytestmark = pytest.mark.gpu


def gen(dtype, size, seed):
    if dtype == "f32":
        return synth.normal_f32(size, seed)
    if dtype == "f64":
        return synth.uniform_f64(size, seed, -1, 1)
    if dtype == "bf16":
        return synth.f32_to_bf16_bits(synth.normal_f32(size, seed))
    if dtype == "f16":
        return synth.normal_f32(size, seed).astype(np.float16)
    if dtype == "i32":
        return synth.uniform_i32(size, seed)
    if dtype == "u32":
        return synth.random_u32(size, seed)
    return synth.random_i64(size, seed)


def got_values(y, dtype, op):
    """The scan output as numpy: integers in the output type, floats as float64."""
    od = pr.out_dtype_name(dtype, op)
    b = bits_of(y, od)
    if od == "bf16":
        return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if od == "f16":
        return b.view(np.float16).astype(np.float64)
    if od in ("f32", "f64"):
        return b.astype(np.float64)
    return b


def assert_same(got, want, dtype):
    if dtype in oracle.INT_DTYPES:
        assert np.array_equal(got, want)
        return
    nan_g, nan_w = np.isnan(got), np.isnan(want)
    assert np.array_equal(nan_g, nan_w)
    ok = ~nan_w
    assert np.array_equal(got[ok], want[ok])
    assert np.array_equal(np.signbit(got[ok]), np.signbit(want[ok]))     # -0 vs +0


def run(x, dtype, op, exclusive, offset=0):
    """The scan of x, written into a canary-guarded output."""
    t = to_device(x, dtype, offset)
    g = guarded_like(t.numel(), pr.out_dtype_name(dtype, op))
    y = pr.scan(t, op, exclusive=exclusive, out=g.tensor)
    g.check()
    return got_values(y, dtype, op)


# around the 32 KB tile (8192 4-byte elements; 4096 8-byte, 16384 2-byte)
SIZES = [1, 5, 4095, 4096, 4097, 8191, 8192, 8193, 3 * 8192, 100000, (1 << 20) + 3]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("exclusive", [False, True])
def test_scan_int32_sum_and_max(n, exclusive):
    x = gen("i32", n, n)
    for op in ("sum", "max"):
        assert_same(run(x, "i32", op, exclusive), oracle.scan(x, "i32", op, exclusive), "i32")


PAIRS = [("u32", "sum"), ("i64", "sum"), ("i32", "min"), ("u32", "xor"), ("u32", "and"), ("u32", "or"),
         ("i64", "prod"), ("i64", "max"), ("f32", "max"), ("f32", "min"), ("f64", "max"), ("bf16", "max"),
         ("f16", "min")]


@pytest.mark.parametrize("dtype,op", PAIRS)
@pytest.mark.parametrize("offset", [0, 1])
def test_scan_dtypes(dtype, op, offset):
    n = 70001
    x = gen(dtype, n, 3 + offset)
    for exclusive in (False, True):
        assert_same(run(x, dtype, op, exclusive, offset), oracle.scan(x, dtype, op, exclusive), dtype)


@pytest.mark.parametrize("dtype,op", [("i64", "sum"), ("f64", "max"), ("bf16", "max"), ("u32", "or")])
@pytest.mark.parametrize("tiles", [1, 2, 7, 300])
def test_scan_whole_tiles(dtype, op, tiles):
    """n an exact number of 32 KB tiles and one element either side: every
    tile staged, then a one-element ragged tail, then one element short."""
    es = {"i64": 8, "f64": 8, "bf16": 2, "u32": 4}[dtype]
    base = tiles * (32768 // es)
    for n in (base - 1, base, base + 1):
        x = gen(dtype, n, tiles + n)
        for exclusive in (False, True):
            assert_same(run(x, dtype, op, exclusive), oracle.scan(x, dtype, op, exclusive), dtype)


@pytest.mark.parametrize("dtype,op", [("u32", "sum"), ("i32", "sum"), ("f32", "min")])
def test_scan_unaligned_output(dtype, op):
    """x aligned but y one element past a 16-byte boundary: every tile is read
    and written element-wise, with the same result."""
    import torch
    n = 5 * 8192 + 77
    x = gen(dtype, n, 9)
    t = to_device(x, dtype)
    od = pr.out_dtype_name(dtype, op)
    buf = torch.zeros(n + 1, dtype=pr.torch_dtype(od), device="cuda")
    y = buf[1:]
    assert y.data_ptr() % 16 != 0
    for exclusive in (False, True):
        pr.scan(t, op, exclusive=exclusive, out=y)
        assert_same(got_values(y, dtype, op), oracle.scan(x, dtype, op, exclusive), dtype)
    assert buf[0].item() == 0


def test_scan_float_nan_and_signed_zeros():
    n = 50000
    x = synth.normal_f32(n, 5)
    x[10000:10010] = 0.0
    x[12000] = -0.0
    x[30000] = np.nan
    for op in ("max", "min"):
        for exclusive in (False, True):
            assert_same(run(x, "f32", op, exclusive), oracle.scan(x, "f32", op, exclusive), "f32")
    z = np.array([0.0, -0.0] * 3000, dtype=np.float32)
    assert_same(run(z, "f32", "min", False), oracle.scan(z, "f32", "min"), "f32")
    assert_same(run(z, "f32", "max", False), oracle.scan(z, "f32", "max"), "f32")


def test_scan_large_int_sum_and_no_device_error():
    n = (1 << 26) + 12345
    x = synth.uniform_i32(n, 6)
    got = run(x, "i32", "sum", False)
    assert_same(got, oracle.scan(x, "i32", "sum"), "i32")
    assert pr.last_device_error() == 0


def test_scan_empty_and_closed_forms():
    import torch
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    assert pr.scan(e, "sum").numel() == 0
    ones = torch.ones(1 << 21, dtype=torch.int64, device="cuda")
    y = pr.scan(ones, "sum").cpu().numpy()
    assert np.array_equal(y, np.arange(1, (1 << 21) + 1))
    ye = pr.scan(ones, "sum", exclusive=True).cpu().numpy()
    assert np.array_equal(ye, np.arange(0, 1 << 21))


def test_scan_deterministic_and_graph_replay():
    import torch
    n = 3 * (1 << 20) + 7
    x = to_device(gen("u32", n, 7), "u32")
    want = oracle.scan(gen("u32", n, 7), "u32", "xor")
    s = torch.cuda.Stream()
    y = torch.empty(n, dtype=torch.int32, device="cuda")      # u32 bits
    with torch.cuda.stream(s):
        pr.scan(x, "xor", out=y, stream=s)         # grows the tile state outside capture
    s.synchronize()
    assert np.array_equal(bits_of(y, "u32"), want)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pr.check(pr.pr_scan(x.data_ptr(), n, pr.DTYPES["u32"], pr.OPS["xor"], 0, y.data_ptr(), s.cuda_stream))
    for _ in range(4):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(bits_of(y, "u32"), want)      # fresh flags on every replay


def test_scan_rejects():
    import torch
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(pr.PrError):
        pr.scan(x, "sum")


def test_bounded_wait_runs_out_and_reports_timeout():
    """The look-back's bounded wait, on a tile state nothing publishes: it must
    give up, leave PR_ERR_TIMEOUT in the error word, and leave the context
    usable (a scan right after is correct)."""
    import torch
    assert pr.last_device_error() == 0
    pr.check(pr.pr_check_bounded_wait(2000, torch.cuda.current_stream().cuda_stream))
    assert pr.last_device_error() == 4                       # PR_ERR_TIMEOUT
    assert pr.last_device_error() == 0                       # read and cleared
    x = gen("i32", 100000, 8)
    assert_same(run(x, "i32", "sum", False), oracle.scan(x, "i32", "sum"), "i32")
