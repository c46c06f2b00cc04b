"""Backward kernels and the autograd wrapper, against the oracle's gradient
(which is pinned by finite differences on the CPU) and fp64 finite differences
of the GPU forward."""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from paper_1710_07358_gb300.autograd import reduce as ad_reduce
from gpu_helpers import to_device, Guarded

pytestmark = pytest.mark.gpu


def slice_inputs(op, seed, rows=3, cols=1000):
    """1000-element rows; prod rows carry 0, 1 and 2 planted zeros."""
    if op == "prod":
        x = synth.uniform_f32(rows * cols, seed, 0.5, 1.5).reshape(rows, cols)
        if rows > 2:
            x[1, 17] = 0.0
            x[2, 3] = 0.0
            x[2, 999] = 0.0
        return x
    return synth.rows_normal(rows, cols, seed)


@pytest.mark.parametrize("op", ["sum", "max", "min", "prod"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_autograd_matches_oracle_gradient(op, dtype):
    import torch
    x = slice_inputs(op, 30)
    if dtype == "f64":
        x = x.astype(np.float64)
    t = torch.from_numpy(x).cuda().requires_grad_(True)
    y = ad_reduce(t, op)
    g = torch.tensor([1.5, -0.25, 2.0], dtype=t.dtype, device="cuda")
    y.backward(g)
    got = t.grad.double().cpu().numpy()
    want = oracle.grad(x, dtype, op, g.double().cpu().numpy())
    if op in ("sum", "max", "min"):
        assert np.array_equal(got, want)
    else:
        # (cols - 1) roundings in the forward product, two in the backward
        tol = (x.shape[1] + 2) * (2.0 ** -24 if dtype == "f32" else 2.0 ** -53)
        assert np.allclose(got, want, rtol=tol, atol=tol * np.abs(want).max())
        assert np.count_nonzero(got[2]) == 0 and np.count_nonzero(got[1]) == 1


@pytest.mark.parametrize("op", ["sum", "max", "prod"])
def test_finite_differences_of_gpu_forward(op):
    """Central differences in fp64 of the GPU forward itself (fp64 path)."""
    import torch
    x = slice_inputs(op, 31, rows=1).astype(np.float64)
    t = torch.from_numpy(x).cuda()
    tg = t.clone().requires_grad_(True)
    ad_reduce(tg, op).sum().backward()
    grad = tg.grad.cpu().numpy()[0]
    srt = np.sort(x[0])
    h = 1e-3 if op != "max" else min(1e-3, (srt[-1] - srt[-2]) / 4)
    rng = np.random.default_rng(0)
    idx = list(rng.choice(1000, 40, replace=False)) + [int(np.argmax(x[0]))]
    for i in idx:
        xp, xm = t.clone(), t.clone()
        xp[0, i] += h
        xm[0, i] -= h
        fd = (pr.reduce_rows(xp, op).item() - pr.reduce_rows(xm, op).item()) / (2 * h)
        scale = np.abs(grad).max()
        assert abs(fd - grad[i]) <= 1e-6 * abs(grad[i]) + 1e-9 * scale, (op, i, fd, grad[i])


def test_reduce_over_other_dims():
    import torch
    x = torch.randn(6, 7, 8, dtype=torch.float64, device="cuda", requires_grad=True)
    for dim in (0, 1, 2):
        y = ad_reduce(x, "max", dim=dim)
        assert torch.equal(y, x.amax(dim=dim))
        (g,) = torch.autograd.grad(y.sum(), x)
        assert g.sum().item() == y.numel()


def test_backward_unaligned_rows():
    import torch
    rows, cols = 5, 1001                      # rows start at every alignment
    x = synth.rows_normal(rows, cols, 33)
    t = to_device(x.reshape(-1), "f32", 1).view(rows, cols)
    g = torch.arange(1, rows + 1, dtype=torch.float32, device="cuda")
    for op in ("sum", "max"):
        gd = Guarded((rows, cols), torch.float32)
        if op == "max":
            _, ai = pr.reduce_rows(t, "max", argidx=True)
            gi = pr.reduce_backward("max", t, g, argidx=ai, out=gd.tensor)
        else:
            gi = pr.reduce_backward("sum", t, g, out=gd.tensor)
        gd.check()
        want = oracle.grad(x, "f32", op, g.cpu().numpy())
        assert np.array_equal(gi.double().cpu().numpy(), want)


@pytest.mark.slow
def test_full_size_forward_backward_properties():
    """[64, 2^20] fp32: the differentiation workload, checked on sampled rows
    against the oracle and by properties that hold at any size."""
    import torch
    rows, cols = 64, 1 << 20
    x = synth.rows_normal(rows, cols, synth.config_seed(4))
    t = torch.from_numpy(x).cuda()
    g = torch.linspace(-1, 1, rows, device="cuda")
    s = pr.reduce_rows(t, "sum")
    for r in (0, 31, 63):
        assert oracle.sum_error(x[r], "f32", s[r].item()) <= 1e-6 * oracle.abs_sum(x[r], "f32")
    gi = pr.reduce_backward("sum", t, g)
    assert torch.equal(gi, g[:, None].expand(rows, cols))
    m, ai = pr.reduce_rows(t, "max", argidx=True)
    for r in (0, 17, 63):
        v, i = oracle.argext(x[r], "f32", "max")
        assert m[r].item() == v and ai[r].item() == i
    gi = pr.reduce_backward("max", t, g, argidx=ai)
    assert torch.equal(gi.sum(dim=1), g) and torch.count_nonzero(gi).item() == torch.count_nonzero(g).item()
    xp = synth.prod_rows(rows, cols, synth.config_seed(4))
    tp = torch.from_numpy(xp).cuda()
    p, ax = pr.reduce_rows(tp, "prod", aux=True)
    _, zc, zi = pr.prod_aux_fields(ax)
    for r in (0, 40):
        pnz, wz, wi = oracle.prod_aux(xp[r], "f32")
        assert zc[r].item() == wz and zi[r].item() == wi
    assert torch.all(p == 0)
    gi = pr.reduce_backward("prod", tp, g, aux=ax)
    assert torch.count_nonzero(gi).item() == 0          # every row has >= 2 zeros
