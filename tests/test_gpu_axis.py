"""Parity of the axis reduction (middle axis of [outer, n, inner]) and its
backward with the oracle, output by output."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from paper_1710_07358_gb300.autograd import reduce as ad_reduce
from gpu_helpers import to_device, values_of, same_float, sum_bound, prod_rel_bound, guarded_like

pytestmark = pytest.mark.gpu


def gen(dtype, op, size, seed):
    if dtype == "f32":
        return synth.uniform_f32(size, seed, 1 - 2.0 ** -7, 1 + 2.0 ** -7) if op == "prod" else synth.normal_f32(size, seed)
    if dtype == "f64":
        return synth.uniform_f64(size, seed) if op == "prod" else synth.uniform_f64(size, seed, -1, 1)
    if dtype == "bf16":
        return synth.f32_to_bf16_bits(synth.normal_f32(size, seed))
    if dtype == "f16":
        return synth.normal_f32(size, seed).astype(np.float16)
    if dtype == "i32":
        return synth.uniform_i32(size, seed)
    if dtype == "u32":
        return synth.random_u32(size, seed)
    return synth.random_i64(size, seed)


def check_axis(x, dtype, op, shape, got, argidx=None, precision="plain"):
    outer, n, inner = shape
    for o, col in enumerate(oracle.axis_slices(x, dtype, outer, n, inner)):
        g = got[o]
        if dtype in oracle.INT_DTYPES:
            want = oracle.reduce(col, dtype, op) if n else oracle.identity(dtype, op)
            assert g == want, (o, g, want)
        elif op in ("max", "min"):
            v, i = oracle.argext(col, dtype, op)
            assert same_float(g, v), (o, g, v)
            if argidx is not None:
                assert argidx[o] == i, (o, argidx[o], i)
        elif op == "sum":
            if n:
                assert oracle.sum_error(col, dtype, g) <= sum_bound(col, dtype, precision), o
            else:
                assert same_float(g, 0.0)
        else:
            want = oracle.reduce(col, dtype, "prod") if n else 1.0
            d = "f64" if dtype == "f64" else "f32"
            assert abs(g - want) <= prod_rel_bound(max(n, 1), d) * abs(want), (o, g, want)


def run_axis(x, dtype, op, shape, offset=0, argidx=False, precision="plain"):
    """Outputs of the middle-axis reduction, written into canary-guarded buffers."""
    t = to_device(x, dtype, offset).view(*shape)
    od = pr.out_dtype_name(dtype, op)
    oshape = (shape[0], shape[2])
    go, ga = guarded_like(oshape, od), guarded_like(oshape, "i64")
    res = pr.reduce_axis(t, op, 1, precision=precision, argidx=argidx, out=go.tensor, argidx_out=ga.tensor)
    go.check(), ga.check()
    if argidx:
        return values_of(res[0], od), res[1].reshape(-1).cpu().numpy()
    return values_of(res, od), None


# shapes: columns of one vector or less per row, many vectors per row, rows
# split across many warps (long axis, few outputs), a single row, an empty axis
SHAPES = [(3, 17, 5), (2, 1000, 64), (1, 4096, 40), (4, 3, 4096), (1, 1, 8), (5, 0, 7), (2, 20000, 8),
          (16, 64, 1024), (1, 50000, 1), (3, 300, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("offset", [0, 1])
def test_axis_f32_sum_max(shape, offset):
    size = shape[0] * shape[1] * shape[2]
    x = synth.normal_f32(size, sum(shape) + offset)
    for op in ("sum", "max", "min"):
        vals, ai = run_axis(x, "f32", op, shape, offset, argidx=op != "sum")
        check_axis(x, "f32", op, shape, vals, argidx=ai)


PAIRS = [("f32", "prod"), ("bf16", "sum"), ("f16", "max"), ("f64", "sum"), ("f64", "prod"), ("f64", "min"),
         ("i32", "sum"), ("i32", "max"), ("u32", "xor"), ("u32", "and"), ("i64", "sum"), ("i64", "min")]


@pytest.mark.parametrize("dtype,op", PAIRS)
@pytest.mark.parametrize("shape", [(3, 300, 48), (2, 5000, 16), (4, 7, 1000)])
def test_axis_dtypes(dtype, op, shape):
    size = shape[0] * shape[1] * shape[2]
    x = gen(dtype, op, size, 40 + shape[2])
    vals, ai = run_axis(x, dtype, op, shape, argidx=op in ("max", "min") and dtype not in ("u32",))
    check_axis(x, dtype, op, shape, vals, argidx=ai)


def test_axis_planted_extremes_nan_and_zeros():
    import torch
    outer, n, inner = 2, 500, 24
    x = synth.normal_f32(outer * n * inner, 41).reshape(outer, n, inner)
    x[0, 7, 3] = 50.0
    x[0, 9, 3] = 50.0            # tie: the first index wins
    x[1, 0, 5] = -60.0
    x[1, 499, 6] = np.nan        # NaN is the extremum of max and min
    x[0, :, 10] = -0.0
    x[0, 250, 10] = 0.0          # -0 < +0
    flat = x.reshape(-1)
    for op in ("max", "min"):
        vals, ai = run_axis(flat, "f32", op, (outer, n, inner), argidx=True)
        check_axis(flat, "f32", op, (outer, n, inner), vals, argidx=ai)
    t = torch.from_numpy(flat).cuda().view(outer, n, inner)
    _, ai = pr.reduce_axis(t, "max", 1, argidx=True)
    assert ai[0, 3].item() == 7 and ai[0, 10].item() == 250 and ai[1, 6].item() == 499


@pytest.mark.parametrize("precision", ["fp64_combine", "compensated"])
def test_axis_precision_modes(precision):
    outer, n, inner = 2, 1 << 15, 16
    x, _, _ = synth.ill_conditioned_f32(outer * n * inner, 42)
    vals, _ = run_axis(x, "f32", "sum", (outer, n, inner), precision=precision)
    check_axis(x, "f32", "sum", (outer, n, inner), vals, precision=precision)


def test_axis_product_aux():
    outer, n, inner = 3, 400, 16
    x = synth.uniform_f32(outer * n * inner, 43, 1 - 2.0 ** -7, 1 + 2.0 ** -7).reshape(outer, n, inner)
    x[0, 5, 2] = 0.0
    x[1, 7, 9] = 0.0
    x[1, 300, 9] = -0.0
    flat = x.reshape(-1)
    import torch
    t = torch.from_numpy(flat).cuda().view(outer, n, inner)
    out, ax = pr.reduce_axis(t, "prod", 1, aux=True)
    p_nz, zc, zi = (v.cpu().numpy() for v in pr.prod_aux_fields(ax))
    vals = values_of(out, "f32")
    for o, col in enumerate(oracle.axis_slices(flat, "f32", outer, n, inner)):
        wp, wz, wi = oracle.prod_aux(col, "f32")
        assert zc[o] == wz and zi[o] == wi
        assert abs(p_nz[o] - wp) <= prod_rel_bound(n, "f32") * abs(wp)
        want = oracle.reduce(col, "f32", "prod")
        assert same_float(vals[o], want) if want == 0 else abs(vals[o] - want) <= prod_rel_bound(n, "f32") * abs(want)


def test_axis_deterministic_and_every_config():
    import torch
    outer, n, inner = 2, 3000, 200
    x = synth.normal_f32(outer * n * inner, 44)
    t = torch.from_numpy(x).cuda().view(outer, n, inner)
    nkey = outer * n * inner
    old = pr.get_config("axis", "f32", "sum", "plain", nkey)
    oldm = pr.get_config("axis", "f32", "max", "plain", nkey)
    try:
        for block in (64, 256, 1024):
            for unroll in (2, 4):
                for vb in (16, 32):
                    cfg = dict(block=block, blocks_per_sm=2, unroll=unroll, vec_bytes=vb)
                    pr.set_config("axis", "f32", "sum", "plain", nkey, cfg)
                    pr.set_config("axis", "f32", "max", "plain", nkey, cfg)
                    s1 = pr.reduce_axis(t, "sum", 1)
                    check_axis(x, "f32", "sum", (outer, n, inner), values_of(s1, "f32"))
                    assert torch.equal(pr.reduce_axis(t, "sum", 1).view(torch.int32), s1.view(torch.int32))
                    m, ai = pr.reduce_axis(t, "max", 1, argidx=True)
                    check_axis(x, "f32", "max", (outer, n, inner), values_of(m, "f32"), argidx=ai.reshape(-1).cpu().numpy())
    finally:
        pr.set_config("axis", "f32", "sum", "plain", nkey, old)
        pr.set_config("axis", "f32", "max", "plain", nkey, oldm)


def axis_grad_oracle(x3, dtype, op, g2):
    """oracle.grad applied to every column x3[p, :, q] with grad_out g2[p, q]."""
    outer, n, inner = x3.shape
    want = np.zeros((outer, n, inner))
    for p in range(outer):
        cols = np.ascontiguousarray(x3[p].T)                  # [inner, n]
        want[p] = oracle.grad(cols, dtype, op, g2[p]).T
    return want


@pytest.mark.parametrize("op", ["sum", "max", "min", "prod"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(3, 200, 40), (2, 50, 7), (4, 64, 256)])
def test_axis_backward_matches_oracle(op, dtype, shape):
    import torch
    outer, n, inner = shape
    if op == "prod":
        x = synth.uniform_f32(outer * n * inner, 45, 0.5, 1.5).reshape(shape)
        x[0, 3, 1] = 0.0                     # one zero in column (0, 1)
        x[1, 4, 2] = 0.0
        x[1, 9, 2] = 0.0                     # two zeros in column (1, 2)
    else:
        x = synth.normal_f32(outer * n * inner, 46).reshape(shape)
    if dtype == "f64":
        x = x.astype(np.float64)
    t = torch.from_numpy(x).cuda().requires_grad_(True)
    g = torch.from_numpy(synth.normal_f32(outer * inner, 47).reshape(outer, inner)).cuda().to(t.dtype)
    y = ad_reduce(t, op, dim=1)
    y.backward(g)
    got = t.grad.double().cpu().numpy()
    want = axis_grad_oracle(x, dtype, op, g.double().cpu().numpy())
    if op in ("sum", "max", "min"):
        assert np.array_equal(got, want)
    else:
        tol = (n + 2) * (2.0 ** -24 if dtype == "f32" else 2.0 ** -53)
        assert np.allclose(got, want, rtol=tol, atol=tol * np.abs(want).max())
        assert np.count_nonzero(got[1, :, 2]) == 0 and np.count_nonzero(got[0, :, 1]) == 1


def test_autograd_every_dim_matches_torch():
    import torch
    gen = torch.Generator(device="cuda").manual_seed(48)
    x = torch.randn(5, 6, 7, 8, dtype=torch.float64, device="cuda", generator=gen, requires_grad=True)
    for dim in range(4):
        for op, ref in (("sum", lambda v: v.sum(dim=dim)), ("max", lambda v: v.amax(dim=dim)),
                        ("prod", lambda v: v.prod(dim=dim))):
            y = ad_reduce(x, op, dim=dim)
            yr = ref(x)
            n = x.shape[dim]
            # two float64 evaluations in different orders: each within
            # (n - 1) 2^-53 of the exact value (sum: of sum |x|; prod: relative)
            with torch.no_grad():
                if op == "max":
                    assert torch.equal(y, yr)
                elif op == "sum":
                    assert bool(torch.all((y - yr).abs() <= 2 * (n - 1) * 2.0 ** -53 * x.abs().sum(dim=dim)))
                else:
                    assert bool(torch.all((y - yr).abs() <= 2 * (n - 1) * 2.0 ** -53 * yr.abs()))
            g = torch.randn(y.shape, dtype=y.dtype, device=y.device, generator=gen)
            (gi,) = torch.autograd.grad(y, x, g)
            (gr,) = torch.autograd.grad(yr, x, g)
            assert torch.allclose(gi, gr, rtol=1e-10, atol=1e-12), (op, dim)
