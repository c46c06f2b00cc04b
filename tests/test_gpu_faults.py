"""Failure handling with faults injected on the host (no GPU is faulted):
the library's one-shot hook makes its next device allocation or kernel
launch fail.  Each entry point must return the documented status, enqueue
nothing after the failing step (outputs keep their sentinel), leave no
completion ticket armed and no half-made state behind: the next call on the
same stream is exact."""
import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, sum_bound, same_float

pytestmark = pytest.mark.gpu

CUDA, NOMEM = 3, 5


@pytest.fixture(autouse=True)
def disarmed():
    pr.inject_fault("none")
    yield
    assert pr.inject_fault("none") is False, "an armed fault was never consumed"


def expect_failure(status, code):
    assert status == code, (status, pr.pr_last_error_message())
    assert "injected" in pr.pr_last_error_message()


def stream_ptr():
    import torch
    return torch.cuda.current_stream().cuda_stream


def test_plain_reduce_launch_failure():
    import torch
    x = synth.uniform_f32((1 << 22) + 3, 80)
    t = to_device(x, "f32", 1)
    out = torch.full((), 12345.0, device="cuda")
    pr.inject_fault("launch")
    expect_failure(pr.pr_reduce(t.data_ptr(), t.numel(), 0, 0, out.data_ptr(), stream_ptr()), CUDA)
    torch.cuda.synchronize()
    assert out.item() == 12345.0                          # nothing was enqueued
    pr.reduce(t, "sum", out=out)                          # the ticket was never armed
    assert oracle.sum_error(x, "f32", out.item()) <= sum_bound(x, "f32")
    v, i = pr.reduce_arg(t, "max")
    assert (float(v), int(i)) == oracle.argext(x, "f32", "max")


def test_segmented_rows_backward_launch_failures():
    import torch
    off = synth.offsets_from_lengths(synth.segment_lengths(500, 81, 20000))
    x = synth.normal_f32(int(off[-1]), 82)
    t, o = to_device(x, "f32"), torch.from_numpy(off).cuda()
    out = torch.full((500,), 7.0, device="cuda")
    pr.inject_fault("launch")
    expect_failure(pr.pr_segmented_reduce(t.data_ptr(), o.data_ptr(), 500, 0, 2, out.data_ptr(), stream_ptr()), CUDA)
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))
    got = values_of(pr.segmented_reduce(t, o, "max"), "f32")
    for s in range(500):
        assert same_float(got[s], oracle.reduce(x[off[s]:off[s + 1]], "f32", "max"))
    rows, cols = 16, 1 << 16
    xr = synth.rows_normal(rows, cols, 83)
    tr = torch.from_numpy(xr).cuda()
    out = torch.full((rows,), 7.0, device="cuda")
    pr.inject_fault("launch")
    with pytest.raises(pr.PrError):
        pr.reduce_rows(tr, "sum", out=out)
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))
    s = pr.reduce_rows(tr, "sum")
    for r in (0, 15):
        assert oracle.sum_error(xr[r], "f32", s[r].item()) <= sum_bound(xr[r], "f32")
    g = torch.ones(rows, device="cuda")
    gi = torch.full((rows, cols), 7.0, device="cuda")
    pr.inject_fault("launch")
    with pytest.raises(pr.PrError):
        pr.reduce_backward("sum", tr, g, out=gi)
    torch.cuda.synchronize()
    assert bool(torch.all(gi == 7.0))
    pr.reduce_backward("sum", tr, g, out=gi)
    assert bool(torch.all(gi == 1.0))


def test_axis_failure_between_its_two_launches():
    import torch
    shape = (2, 20000, 8)                                 # row splits: a partials pass, then a finishing pass
    x = synth.normal_f32(shape[0] * shape[1] * shape[2], 84)
    t = torch.from_numpy(x).cuda().view(*shape)
    out = torch.full((2, 8), 7.0, device="cuda")
    pr.inject_fault("launch", after=1)                    # the first launch passes, the finishing one fails
    with pytest.raises(pr.PrError):
        pr.reduce_axis(t, "sum", 1, out=out)
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))
    pr.reduce_axis(t, "sum", 1, out=out)
    got = out.reshape(-1).cpu().numpy()
    for o, col in enumerate(oracle.axis_slices(x, "f32", *shape)):
        assert oracle.sum_error(col, "f32", float(got[o])) <= sum_bound(col, "f32")


def test_scan_and_line_search_launch_failures():
    import torch
    n = 3 * 8192 + 5
    xs = synth.random_u32(n, 85)
    t = torch.from_numpy(xs.view(np.int32)).cuda().view(torch.uint32)
    y = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    pr.inject_fault("launch")
    with pytest.raises(pr.PrError):
        pr.scan(t, "sum", out=y.view(torch.uint32))
    torch.cuda.synchronize()
    assert bool(torch.all(y == 7))
    pr.scan(t, "sum", out=y.view(torch.uint32))
    assert np.array_equal(y.cpu().numpy().view(np.uint32), oracle.scan(xs, "u32", "sum"))
    links = synth.network_links(20011, 86)
    lt = [torch.from_numpy(a).cuda() for a in links]
    want = pr.line_search(*lt, count=12).cpu().numpy()
    res = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    pr.inject_fault("launch", after=2)                    # init and the first pass run, the second fails
    with pytest.raises(pr.PrError):
        pr.line_search(*lt, count=12, result=res)
    torch.cuda.synchronize()
    assert bool(torch.all(res == 7.0))                    # the result is written by the last pass only
    assert np.array_equal(pr.line_search(*lt, count=12, result=res).cpu().numpy(), want)
    assert pr.last_device_error() == 0


def test_host_path_launch_failure_waits_for_its_copies():
    import torch
    n = (100 << 20) // 4 + 3                              # two 64 MiB chunks
    x = synth.uniform_i32(n, 87)
    h = torch.from_numpy(x).pin_memory()
    pr.inject_fault("launch", after=1)                    # the second chunk's reduction fails
    with pytest.raises(pr.PrError):
        pr.reduce_host(h, "sum")
    h.zero_()                                             # the caller may reuse its buffer at once
    h.copy_(torch.from_numpy(x))
    assert pr.reduce_host(h, "sum") == oracle.reduce(x, "i32", "sum")


def test_allocation_failures_keep_no_partial_state():
    import torch
    x = synth.uniform_f32((1 << 20) + 7, 88)
    t = to_device(x, "f32")
    s = torch.cuda.Stream()                               # a new stream: its workspace is made on first use
    pr.inject_fault("alloc")
    assert pr.pr_prepare(s.cuda_stream) == NOMEM and "injected" in pr.pr_last_error_message()
    out = pr.reduce(t, "sum", stream=s)                   # allocates afresh
    s.synchronize()
    assert oracle.sum_error(x, "f32", out.item()) <= sum_bound(x, "f32")
    # per-stream growth buffers: the workspace allocation passes, the next one fails
    for what in ("scan", "search", "axis"):
        s2 = torch.cuda.Stream()
        pr.inject_fault("alloc", after=1)
        with pytest.raises(pr.PrError) as e:
            if what == "scan":
                xs = synth.random_u32(1 << 20, 89)
                ts = torch.from_numpy(xs.view(np.int32)).cuda().view(torch.uint32)
                pr.scan(ts, "xor", stream=s2)
            elif what == "search":
                links = [torch.from_numpy(a).cuda() for a in synth.network_links(4001, 90)]
                pr.line_search(*links, count=5, stream=s2)
            else:
                xa = torch.from_numpy(synth.normal_f32(2 * 20000 * 8, 91)).cuda().view(2, 20000, 8)
                pr.reduce_axis(xa, "sum", 1, stream=s2)
        assert e.value.status == NOMEM, what
        s2.synchronize()
        if what == "scan":
            y = pr.scan(ts, "xor", stream=s2)
            s2.synchronize()
            assert np.array_equal(y.view(torch.int32).cpu().numpy().view(np.uint32), oracle.scan(xs, "u32", "xor"))
        elif what == "search":
            r = pr.line_search(*links, count=5, stream=s2)
            s2.synchronize()
            assert r[1].item() - r[0].item() == pytest.approx(0.6180339887498949 ** 5, rel=1e-9)
        else:
            o = pr.reduce_axis(xa, "sum", 1, stream=s2)
            s2.synchronize()
            xa_h = xa.reshape(-1).cpu().numpy()
            for k, col in enumerate(oracle.axis_slices(xa_h, "f32", 2, 20000, 8)):
                assert oracle.sum_error(col, "f32", float(o.reshape(-1)[k])) <= sum_bound(col, "f32")
