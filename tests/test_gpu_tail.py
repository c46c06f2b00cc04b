"""The plain reduction's claimed tail: inputs of 768 MiB and more leave the
vectors past a multiple of the grid's stride (about the last tenth) to tiles
that blocks claim from a counter.  Checked here: the launch plan takes the
tail where it should; every op gives the oracle's result (bit for bit where
the result is exact, within the stated bound for float sums and products)
with aligned and misaligned inputs; arg-extremum indices planted in claimed
tiles and across the grid-stride / claimed boundary come out
first-occurrence; repeats and CUDA-graph replays give the same bits (the
claim counter is re-armed by every launch); and a segmented reduction that
claims chunks from the same counter right after still gives the oracle's
results."""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, same_float, sum_bound, prod_rel_bound, Guarded

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = (1 << 28) + 1237          # 1 GiB of 32-bit values plus a ragged end
PAD = 3                       # misaligned views start this many elements in
ONE_PER_SM = dict(block=1024, blocks_per_sm=1, unroll=2, vec_bytes=32)


def plan(t, op, **kw):
    return pr.reduce_plan(t, op, **kw)


@pytest.fixture
def shape():
    """Set a launch shape for (dtype, op) at N for one test, then restore
    the table's."""
    saved = []

    def use(dtype, op, cfg, precision="plain", n=N):
        saved.append((dtype, op, precision, n, pr.get_config("reduce", dtype, op, precision, n)))
        pr.set_config("reduce", dtype, op, precision, n, cfg)
    yield use
    for dtype, op, precision, n, c in saved:
        pr.set_config("reduce", dtype, op, precision, n, c)


@pytest.fixture(scope="module")
def inputs():
    """Per dtype: host values of N + PAD elements and their device copy
    (views at offset 0 and PAD share them)."""
    import torch
    cache = {}

    def get(dtype):
        if dtype not in cache:
            if dtype == "f32":
                x = synth.uniform_f32(N + PAD, 800)
            elif dtype == "i32":
                x = synth.uniform_i32(N + PAD, 801)
            else:
                x = synth.random_u32(N + PAD, 802)
            cache[dtype] = (x, to_device(x, dtype))
        return cache[dtype]
    yield get
    cache.clear()
    torch.cuda.empty_cache()


def test_plan_takes_the_tail_from_768_mib(shape):
    import torch
    head = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
    p = plan(head, "sum")                             # the measured fp32 sum, table shape
    assert p["tail_vectors"] > 0 and p["block"] == 1024, p
    nvec = (1 << 28) * 4 // 32                        # about a tenth of the vectors
    assert nvec // 20 < p["tail_vectors"] < nvec // 5, p
    assert plan(head[: 1 << 27], "sum")["tail_vectors"] == 0      # 512 MiB: grid-stride only
    # with one block of 1024 threads per SM every plain trait's tail kernel
    # fits beside the grid-stride one
    i32 = head.view(torch.int32)
    u32 = head.view(pr.torch_dtype("u32"))
    for t, dtype, ops in ((head, "f32", ("sum", "max", "min")), (i32, "i32", ("sum", "max")),
                          (u32, "u32", ("xor", "and", "or"))):
        for op in ops:
            shape(dtype, op, ONE_PER_SM, n=1 << 28)
            p = plan(t, op)
            assert p["tail_vectors"] > 0 and p["block"] == 1024, (dtype, op, p)


CASES = [("f32", "sum"), ("f32", "max"), ("f32", "min"), ("i32", "sum"), ("i32", "max"), ("u32", "xor"),
         ("u32", "and"), ("u32", "or")]


@pytest.mark.parametrize("launch", ["table", "1024x1"])
@pytest.mark.parametrize("offset", [0, PAD])
@pytest.mark.parametrize("dtype,op", CASES)
def test_tail_matches_oracle_and_repeats(dtype, op, offset, launch, shape, inputs):
    """With the table's launch shape (the tail where its kernel fits) and
    with one 1024-thread block per SM (the tail always)."""
    import torch
    xall, dall = inputs(dtype)
    x, t = xall[offset:offset + N], dall[offset:offset + N]
    if op == "and":
        # keep some bits set through 2^28 ANDs, and clear one late in the tail
        x = x | np.uint32(0xFFFF0000)
        x[N - 17] &= np.uint32(0xFFFEFFFF)
        t = to_device(x, dtype, offset)
    if launch == "1024x1":
        shape(dtype, op, ONE_PER_SM)
        assert plan(t, op)["tail_vectors"] > 0
    od = pr.out_dtype_name(dtype, op)
    g = Guarded((), pr.torch_dtype(od))
    pr.reduce(t, op, out=g.tensor)
    first = values_of(g.check(), od)[0]
    if dtype == "f32" and op == "sum":
        assert oracle.sum_error(x, dtype, first) <= sum_bound(x, dtype)
    elif dtype == "f32":
        assert same_float(first, oracle.reduce(x, dtype, op))
    else:
        assert first == oracle.reduce(x, dtype, op)
    for _ in range(3):
        assert values_of(pr.reduce(t, op), od)[0] == first
    # graph replay: every replay claims tiles from a re-armed counter
    s = torch.cuda.Stream()
    pr.pr_prepare(s.cuda_stream)
    out = torch.empty((), dtype=pr.torch_dtype(od), device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        pr.reduce(t, op, out=out, stream=s)
    for _ in range(3):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert values_of(out, od)[0] == first


def tail_start(t, op, arg=False):
    """First element index of the claimed part (vectors of 32 bytes)."""
    p = plan(t, op, arg=arg)
    assert p["tail_vectors"] > 0
    es = t.element_size()
    ve = 32 // es
    head = (-(t.data_ptr() // es)) % ve
    nvec = (t.numel() - head) // ve
    return head + (nvec - p["tail_vectors"]) * ve


@pytest.mark.parametrize("op", ["max", "min"])
def test_argext_planted_in_claimed_tiles(op, inputs):
    """int32 (its arg-extremum tail kernel fits beside the grid-stride one at
    the default shape; values in [-2^20, 2^20), planted +-2^30)."""
    xall, dall = inputs("i32")
    x, t = xall[:N], dall[:N]
    ts = tail_start(t, op, arg=True)
    big = (1 << 30) if op == "max" else -(1 << 30)
    planted = []

    def plant(i):
        planted.append((i, int(t[i].item())))
        t[i] = big

    try:
        # ties inside the claimed part: the first wins
        plant(ts + 1000003)
        plant(N - 5)
        v, i = pr.reduce_arg(t, op)
        assert int(v.item()) == big and int(i.item()) == ts + 1000003
        # ties across the boundary: the grid-stride part's occurrence first
        plant(ts - 1)
        v, i = pr.reduce_arg(t, op)
        assert int(i.item()) == ts - 1
    finally:
        for i, old in reversed(planted):
            t[i] = old
    # the extremum on the first claimed element, and on the last element
    for at in (ts, N - 1):
        old = int(t[at].item())
        t[at] = big
        try:
            v, i = pr.reduce_arg(t, op)
            assert int(v.item()) == big and int(i.item()) == at
        finally:
            t[at] = old
    v, i = pr.reduce_arg(t, op)
    wv, wi = oracle.argext(x, "i32", op)
    assert int(v.item()) == wv and int(i.item()) == wi


def test_compensated_and_product_forms_with_the_tail(shape, inputs):
    """Traits whose tiles leave partials of their own kind: the compensated
    fp32 pair and the fp64 product's split state (2 GiB), each with one
    1024-thread block per SM and a vector width whose tail kernel fits."""
    xall, dall = inputs("f32")
    x, t = xall[:N], dall[:N]
    shape("f32", "sum", ONE_PER_SM, precision="compensated")
    assert plan(t, "sum", precision="compensated")["tail_vectors"] > 0
    got = values_of(pr.reduce(t, "sum", precision="compensated"), "f32")[0]
    assert oracle.sum_error(x, "f32", got) <= sum_bound(x, "f32", "compensated")
    r64 = values_of(pr.reduce(t, "sum", precision="compensated", out_dtype="f64"), "f64")[0]
    assert oracle.sum_error(x, "f32", r64) <= sum_bound(x, "f32", "compensated")
    # fp32 accumulators with the fp64 combine: the tiles' partials are fp64 too
    shape("f32", "sum", ONE_PER_SM, precision="fp64_combine")
    assert plan(t, "sum", precision="fp64_combine")["tail_vectors"] > 0
    got = values_of(pr.reduce(t, "sum", precision="fp64_combine"), "f32")[0]
    assert oracle.sum_error(x, "f32", got) <= sum_bound(x, "f32", "fp64_combine")
    n64 = (1 << 28) + 9
    xp = synth.uniform_f64(n64, 813)
    tp = to_device(xp, "f64")
    shape("f64", "prod", dict(block=1024, blocks_per_sm=1, unroll=2, vec_bytes=16), n=n64)
    assert plan(tp, "prod")["tail_vectors"] > 0
    got = values_of(pr.reduce(tp, "prod"), "f64")[0]
    want = oracle.reduce(xp, "f64", "prod")
    assert want != 0.0 and abs(got - want) <= prod_rel_bound(n64, "f64") * abs(want)


def test_segmented_after_a_tail_reduction_on_the_same_stream(inputs):
    import torch
    xall, dall = inputs("f32")
    x, t = xall[:N], dall[:N]
    assert plan(t, "sum")["tail_vectors"] > 0
    pr.reduce(t, "sum")
    off = synth.offsets_from_lengths(synth.segment_lengths(3000, 815, 20000))
    xs = synth.normal_f32(int(off[-1]), 816)
    got = values_of(pr.segmented_reduce(to_device(xs, "f32"), torch.from_numpy(off).cuda(), "max"), "f32")
    want = oracle.segmented(xs, off, "f32", "max")
    assert all(same_float(a, float(b)) for a, b in zip(got, want))
    again = values_of(pr.reduce(t, "sum"), "f32")[0]
    assert oracle.sum_error(x, "f32", again) <= sum_bound(x, "f32")


@pytest.mark.parametrize("launch", ["table", "1024x1"])
def test_float_product_with_planted_factors_is_exact(launch, shape):
    """fp32 product of 2^28 + 1237 factors, all 1 except 64 twos and 60
    halves spread over the grid-stride part and the claimed tiles: every
    partial product is a power of two within range, so any association gives
    exactly 16; a zero in the last tile then gives +0."""
    import torch
    x = torch.ones(N, dtype=torch.float32, device="cuda")
    if launch == "1024x1":
        shape("f32", "prod", ONE_PER_SM)
        assert plan(x, "prod")["tail_vectors"] > 0
    ts = tail_start(x, "prod") if plan(x, "prod")["tail_vectors"] > 0 else N - N // 10
    rng = np.random.default_rng(817)
    twos = np.concatenate([rng.integers(0, ts, 32), rng.integers(ts, N, 32)])
    halves = np.concatenate([rng.integers(0, ts, 30), rng.integers(ts, N, 30)])
    twos = np.unique(twos)
    halves = np.setdiff1d(np.unique(halves), twos)
    x[torch.from_numpy(twos).cuda()] = 2.0
    x[torch.from_numpy(halves).cuda()] = 0.5
    want = 2.0 ** (len(twos) - len(halves))
    g = Guarded((), torch.float32)
    pr.reduce(x, "prod", out=g.tensor)
    assert values_of(g.check(), "f32")[0] == want
    x[N - 2] = 0.0
    assert same_float(values_of(pr.reduce(x, "prod"), "f32")[0], 0.0)
