"""Parity of the segmented and row reductions with the oracle, segment by segment."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, same_float, sum_bound, prod_rel_bound, guarded_like

pytestmark = pytest.mark.gpu


def dev_off(off):
    import torch
    return torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda()


def check_segments(x, off, dtype, op, out_vals, argidx=None, precision="plain"):
    off = np.asarray(off)
    for s in range(len(off) - 1):
        seg = x[off[s]:off[s + 1]]
        got = out_vals[s]
        if dtype in oracle.INT_DTYPES:
            want = oracle.reduce(seg, dtype, op) if seg.size else oracle.identity(dtype, op)
            assert got == want, (s, got, want)
        elif op in ("max", "min"):
            v, i = oracle.argext(seg, dtype, op)
            assert same_float(got, v), (s, got, v)
            if argidx is not None:
                assert argidx[s] == i, (s, argidx[s], i)
        elif op == "sum":
            if seg.size:
                assert oracle.sum_error(seg, dtype, got) <= sum_bound(seg, dtype, precision), s
            else:
                assert same_float(got, 0.0)
        else:
            want = oracle.reduce(seg, dtype, "prod") if seg.size else 1.0
            d = "f64" if dtype == "f64" else "f32"
            assert abs(got - want) <= prod_rel_bound(max(seg.size, 1), d) * abs(want) + 0.0, (s, got, want)


def run_seg(x, off, dtype, op, offset=0, argidx=False, aux=False, precision="plain"):
    """Segment results (and argidx / aux), written into canary-guarded outputs."""
    t = to_device(x, dtype, offset)
    nseg = len(off) - 1
    od = pr.out_dtype_name(dtype, op)
    go, ga, gx = guarded_like(nseg, od), guarded_like(nseg, "i64"), guarded_like(nseg * 24, "aux")
    res = pr.segmented_reduce(t, dev_off(off), op, precision=precision, argidx=argidx, aux=aux, out=go.tensor,
                              argidx_out=ga.tensor, aux_out=gx.tensor)
    for g in (go, ga, gx):
        g.check()
    if argidx:
        return values_of(res[0], od), res[1].cpu().numpy()
    if aux:
        return values_of(res[0], od), res[1]
    return values_of(res, od), None


def gen_vals(dtype, op, n, seed):
    # product inputs near 1: no partial product leaves the normal range
    if dtype == "f32":
        return synth.uniform_f32(n, seed, 1 - 2.0 ** -7, 1 + 2.0 ** -7) if op == "prod" else synth.normal_f32(n, seed)
    if dtype == "f64":
        return synth.uniform_f64(n, seed) if op == "prod" else synth.uniform_f64(n, seed, -1, 1)
    if dtype == "bf16":
        return synth.f32_to_bf16_bits(synth.normal_f32(n, seed))
    if dtype == "f16":
        return synth.normal_f32(n, seed).astype(np.float16)
    if dtype == "i32":
        return synth.uniform_i32(n, seed)
    if dtype == "u32":
        return synth.random_u32(n, seed)
    return synth.random_i64(n, seed)


SEG_PAIRS = [("f32", "sum"), ("f32", "max"), ("f32", "min"), ("f32", "prod"), ("bf16", "sum"), ("f16", "max"),
             ("f64", "sum"), ("f64", "prod"), ("f64", "min"), ("i32", "sum"), ("i32", "max"), ("u32", "xor"),
             ("u32", "and"), ("i64", "sum"), ("i64", "min")]


@pytest.mark.parametrize("dtype,op", SEG_PAIRS)
@pytest.mark.parametrize("nseg,max_len", [(1, 1), (3, 40000), (17, 5000), (300, 70000), (2000, 300)])
def test_log_uniform_segments(dtype, op, nseg, max_len):
    off = synth.offsets_from_lengths(synth.segment_lengths(nseg, nseg + max_len, max_len))
    x = gen_vals(dtype, op, int(off[-1]), nseg)
    vals, _ = run_seg(x, off, dtype, op)
    check_segments(x, off, dtype, op, vals)


@pytest.mark.parametrize("dtype,op", [("f32", "sum"), ("f32", "max"), ("i32", "sum"), ("u32", "or")])
def test_empty_and_tiny_segments(dtype, op):
    rng = np.random.default_rng(3)
    lens = rng.integers(0, 4, size=50000)
    lens[:7] = 0                      # leading empties
    lens[-5:] = 0                     # trailing empties
    lens[1000] = 300000               # one long segment among tiny ones
    off = synth.offsets_from_lengths(lens)
    x = gen_vals(dtype, op, int(off[-1]), 4)
    vals, _ = run_seg(x, off, dtype, op)
    check_segments(x, off, dtype, op, vals)


def test_one_segment_spanning_every_block_and_subrange():
    n = (1 << 22) + 13
    x = synth.normal_f32(n, 5)
    for off in ([0, n], [17, n - 3], [5, 5, 1 << 21, n, n]):
        for op in ("sum", "max"):
            vals, _ = run_seg(x, off, "f32", op, offset=1)
            check_segments(x, off, "f32", op, vals)


@pytest.mark.parametrize("offset", [0, 1, 3])
@pytest.mark.parametrize("op", ["max", "min"])
def test_argidx_first_extremum(op, offset):
    off = synth.offsets_from_lengths(synth.segment_lengths(200, 9, 30000))
    x = synth.normal_f32(int(off[-1]), 10)
    # plant ties: the extremum twice in some segments, at its start and end
    for s in range(0, 200, 7):
        lo, hi = off[s], off[s + 1]
        v = 9.0 if op == "max" else -9.0
        x[hi - 1] = v
        x[lo] = v
    vals, ai = run_seg(x, off, "f32", op, offset=offset, argidx=True)
    check_segments(x, off, "f32", op, vals, argidx=ai)
    xi = synth.uniform_i32(int(off[-1]), 11, -5, 5)            # many ties
    vals, ai = run_seg(xi, off, "i32", op, offset=offset, argidx=True)
    for s in range(200):
        assert ai[s] == oracle.argext(xi[off[s]:off[s + 1]], "i32", op)[1]


def test_product_aux():
    import torch
    off = synth.offsets_from_lengths(synth.segment_lengths(300, 12, 3000))
    x = synth.uniform_f32(int(off[-1]), 13, 1 - 2.0 ** -7, 1 + 2.0 ** -7)
    rng = np.random.default_rng(14)
    for s in range(0, 300, 3):              # 0, 1 or 2 zeros in a third of the segments
        lo, hi = off[s], off[s + 1]
        for _ in range(s % 3):
            x[rng.integers(lo, hi)] = 0.0 if s % 2 else -0.0
    vals, ax = run_seg(x, off, "f32", "prod", aux=True)
    p_nz, zc, zi = (t.cpu().numpy() for t in pr.prod_aux_fields(ax))
    for s in range(300):
        seg = x[off[s]:off[s + 1]]
        wp, wz, wi = oracle.prod_aux(seg, "f32")
        assert zc[s] == wz and zi[s] == wi, s
        assert abs(p_nz[s] - wp) <= prod_rel_bound(seg.size, "f32") * abs(wp), s
        want = oracle.reduce(seg, "f32", "prod")
        assert (vals[s] == want == 0.0 and math.copysign(1, vals[s]) == math.copysign(1, want)) or \
            abs(vals[s] - want) <= prod_rel_bound(seg.size, "f32") * abs(want), s


@pytest.mark.parametrize("precision", ["fp64_combine", "compensated"])
def test_segmented_precision_modes(precision):
    off = synth.offsets_from_lengths(synth.segment_lengths(100, 15, 100000))
    x, _, _ = synth.ill_conditioned_f32(int(off[-1]), 16)
    vals, _ = run_seg(x, off, "f32", "sum", precision=precision)
    check_segments(x, off, "f32", "sum", vals, precision=precision)


def test_rows_api_matches_segments():
    import torch
    rows, cols = 37, 12345
    x = synth.rows_normal(rows, cols, 17)
    t = to_device(x.reshape(-1), "f32", 1).view(rows, cols)
    for op in ("sum", "max", "min", "prod"):
        if op == "prod":
            xx = synth.uniform_f32(rows * cols, 18, 0.9, 1.1).reshape(rows, cols)
            tt = to_device(xx.reshape(-1), "f32", 1).view(rows, cols)
        else:
            xx, tt = x, t
        off = np.arange(rows + 1) * cols
        if op in ("max", "min"):
            out, ai = pr.reduce_rows(tt, op, argidx=True)
            check_segments(xx.reshape(-1), off, "f32", op, values_of(out, "f32"), argidx=ai.cpu().numpy())
        else:
            out = pr.reduce_rows(tt, op)
            check_segments(xx.reshape(-1), off, "f32", op, values_of(out, "f32"))
    z = torch.empty((5, 0), dtype=torch.float32, device="cuda")
    assert values_of(pr.reduce_rows(z, "sum"), "f32") == [0.0] * 5
    assert values_of(pr.reduce_rows(z, "max"), "f32") == [-math.inf] * 5


def test_segmented_deterministic_and_graph_replay():
    import torch
    off = synth.offsets_from_lengths(synth.segment_lengths(512, 19, 200000))
    x = to_device(synth.normal_f32(int(off[-1]), 20), "f32")
    o = dev_off(off)
    ref = pr.segmented_reduce(x, o, "sum").clone()
    for _ in range(5):
        assert torch.equal(pr.segmented_reduce(x, o, "sum").view(torch.int32), ref.view(torch.int32))
    s = torch.cuda.Stream()
    out = torch.empty(512, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        pr.prepare(s)
        pr.check(pr.pr_segmented_reduce(x.data_ptr(), o.data_ptr(), 512, 0, 0, out.data_ptr(), s.cuda_stream))
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pr.check(pr.pr_segmented_reduce(x.data_ptr(), o.data_ptr(), 512, 0, 0, out.data_ptr(), s.cuda_stream))
    out.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_every_config_variant():
    off = synth.offsets_from_lengths(synth.segment_lengths(300, 21, 100000))
    x = synth.normal_f32(int(off[-1]), 22)
    t = to_device(x, "f32", 3)
    o = dev_off(off)
    old = pr.get_config("segmented", "f32", "max", "plain", 300)
    try:
        for block in (128, 256, 512):
            for unroll in (2, 4):
                for vb in (16, 32):
                    pr.set_config("segmented", "f32", "max", "plain", 300,
                                  dict(block=block, blocks_per_sm=2, unroll=unroll, vec_bytes=vb))
                    out, ai = pr.segmented_reduce(t, o, "max", argidx=True)
                    check_segments(x, off, "f32", "max", values_of(out, "f32"), argidx=ai.cpu().numpy())
    finally:
        pr.set_config("segmented", "f32", "max", "plain", 300, old)


def test_malformed_offsets_raise_device_error_and_recover():
    x = to_device(synth.normal_f32(64, 23), "f32")
    bad = dev_off([0, 10, 5, 20])          # non-monotone, all within [0, 20]
    pr.segmented_reduce(x, bad, "sum")
    assert pr.last_device_error() == 1
    assert pr.last_device_error() == 0     # cleared
    good = [0, 10, 20, 64]
    vals, _ = run_seg(synth.normal_f32(64, 23), good, "f32", "sum")
    check_segments(synth.normal_f32(64, 23), good, "f32", "sum", vals)


@pytest.mark.parametrize("rows,cols,offset", [(10000, 37, 1), (3, (1 << 21) + 5, 3), (1, 1 << 22, 0),
                                              (64, 4096, 2), (700, 1000, 0), (1, 8, 0), (5, 24, 0),
                                              (64, 1 << 16, 0), (3000, 64, 0), (333, 4104, 0), (2, 1 << 22, 0)])
def test_row_kernel_shapes(rows, cols, offset):
    """Many short rows (many per block) and few long rows split across blocks
    and combined through per-row tickets.  Aligned rows that are a whole
    number of vectors take the row kernel, the others the segmented kernel."""
    x = synth.normal_f32(rows * cols, rows + cols)
    t = to_device(x, "f32", offset).view(rows, cols)
    off = np.arange(rows + 1, dtype=np.int64) * cols
    for op in ("sum", "max", "min"):
        go, ga = guarded_like(rows, "f32"), guarded_like(rows, "i64")
        if op == "sum":
            out = pr.reduce_rows(t, op, out=go.tensor)
            check_segments(x, off, "f32", op, values_of(go.check(), "f32"))
        else:
            out, ai = pr.reduce_rows(t, op, argidx=True, out=go.tensor, argidx_out=ga.tensor)
            check_segments(x, off, "f32", op, values_of(go.check(), "f32"), argidx=ga.check().cpu().numpy())
    xp = synth.uniform_f32(rows * cols, 7, 1 - 2.0 ** -7, 1 + 2.0 ** -7)
    xp[::997] = 0.0
    tp = to_device(xp, "f32", offset).view(rows, cols)
    go, gx = guarded_like(rows, "f32"), guarded_like(rows * 24, "aux")
    out, ax = pr.reduce_rows(tp, "prod", aux=True, out=go.tensor, aux_out=gx.tensor)
    go.check(), gx.check()
    p_nz, zc, zi = (v.cpu().numpy() for v in pr.prod_aux_fields(ax))
    vals = values_of(out, "f32")
    for r in list(range(min(rows, 20))) + [rows - 1]:
        seg = xp[r * cols:(r + 1) * cols]
        wp, wz, wi = oracle.prod_aux(seg, "f32")
        assert zc[r] == wz and zi[r] == wi
        assert abs(p_nz[r] - wp) <= prod_rel_bound(cols, "f32") * abs(wp)
        want = oracle.reduce(seg, "f32", "prod")
        assert abs(vals[r] - want) <= prod_rel_bound(cols, "f32") * abs(want)


ROW_PAIRS = [("bf16", "sum"), ("f16", "max"), ("f64", "sum"), ("f64", "prod"), ("f64", "min"), ("i32", "sum"),
             ("i32", "max"), ("u32", "xor"), ("i64", "sum"), ("i64", "min")]


@pytest.mark.parametrize("dtype,op", ROW_PAIRS)
def test_row_kernel_dtypes(dtype, op):
    rows, cols = 37, 3 * 4096
    x = gen_vals(dtype, op, rows * cols, 31)
    t = to_device(x, dtype).view(rows, cols)
    off = np.arange(rows + 1, dtype=np.int64) * cols
    od = pr.out_dtype_name(dtype, op)
    if op in ("max", "min"):
        out, ai = pr.reduce_rows(t, op, argidx=True)
        check_segments(x, off, dtype, op, values_of(out, od), argidx=ai.cpu().numpy())
    else:
        check_segments(x, off, dtype, op, values_of(pr.reduce_rows(t, op), od))


@pytest.mark.parametrize("precision", ["fp64_combine", "compensated"])
def test_row_kernel_precision_modes(precision):
    rows, cols = 9, 1 << 18
    x, _, _ = synth.ill_conditioned_f32(rows * cols, 32)
    t = to_device(x, "f32").view(rows, cols)
    off = np.arange(rows + 1, dtype=np.int64) * cols
    check_segments(x, off, "f32", "sum", values_of(pr.reduce_rows(t, "sum", precision=precision), "f32"),
                   precision=precision)


def test_row_kernel_every_config_variant():
    import torch
    rows, cols = 7, 40000
    x = synth.normal_f32(rows * cols, 33)
    xp = synth.uniform_f32(rows * cols, 34, 1 - 2.0 ** -7, 1 + 2.0 ** -7)
    xp[5 * cols + 123] = 0.0
    t = to_device(x, "f32").view(rows, cols)
    tp = to_device(xp, "f32").view(rows, cols)
    off = np.arange(rows + 1, dtype=np.int64) * cols
    n = rows * cols
    old = {op: pr.get_config("rows", "f32", op, "plain", n) for op in ("sum", "max", "prod")}
    ref = None
    try:
        for block in (128, 256, 512, 1024):
            for unroll in (2, 4):
                for vb in (16, 32):
                    cfg = dict(block=block, blocks_per_sm=2, unroll=unroll, vec_bytes=vb)
                    for op in old:
                        pr.set_config("rows", "f32", op, "plain", n, cfg)
                    out, ai = pr.reduce_rows(t, "max", argidx=True)
                    check_segments(x, off, "f32", "max", values_of(out, "f32"), argidx=ai.cpu().numpy())
                    s1 = pr.reduce_rows(t, "sum")
                    check_segments(x, off, "f32", "sum", values_of(s1, "f32"))
                    assert torch.equal(pr.reduce_rows(t, "sum").view(torch.int32), s1.view(torch.int32))
                    out, ax = pr.reduce_rows(tp, "prod", aux=True)
                    p_nz, zc, zi = (v.cpu().numpy() for v in pr.prod_aux_fields(ax))
                    for r in range(rows):
                        seg = xp[r * cols:(r + 1) * cols]
                        wp, wz, wi = oracle.prod_aux(seg, "f32")
                        assert zc[r] == wz and zi[r] == wi
                        assert abs(p_nz[r] - wp) <= prod_rel_bound(cols, "f32") * abs(wp)
    finally:
        for op, c in old.items():
            pr.set_config("rows", "f32", op, "plain", n, c)
