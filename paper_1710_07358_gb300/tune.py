"""Build the launch-configuration table for this GPU with the library's autotuner.

For every (dtype, combiner, precision) of the plain reduction and a range of
size buckets, and for the segmented reduction on log-uniform segments, this
calls pr_autotune on synthetic data (timing every block size / blocks-per-SM /
unroll / vector-width candidate with CUDA events) and saves the winners with
pr_tune_save.  The binding loads the table for the current GPU on first use.

    python -m paper_1710_07358_gb300.tune [--out PATH] [--sizes 20,24,28] [--quick]
"""
from __future__ import annotations

import argparse
import os

from . import pr

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.json")

PLAIN = [("f32", "sum"), ("f32", "prod"), ("f32", "max"), ("f32", "min"),
         ("f16", "sum"), ("f16", "prod"), ("f16", "max"), ("f16", "min"),
         ("bf16", "sum"), ("bf16", "prod"), ("bf16", "max"), ("bf16", "min"),
         ("f64", "sum"), ("f64", "prod"), ("f64", "max"), ("f64", "min")] + \
        [(d, o) for d in ("i32", "u32", "i64") for o in ("sum", "prod", "max", "min", "and", "or", "xor")]
PRECISE = [("f32", "compensated"), ("f32", "fp64_combine"), ("f16", "compensated"), ("f16", "fp64_combine"),
           ("bf16", "compensated"), ("bf16", "fp64_combine")]


def _data(torch, dtype, op, n, g):
    dev = "cuda"
    if dtype in ("f32", "f16", "bf16"):
        if op == "prod":
            x = 1.0 + (torch.rand(n, generator=g, device=dev) - 0.5) * 2 ** -6
        else:
            x = torch.rand(n, generator=g, device=dev) * 2 - 1
        return x.to(pr.torch_dtype(dtype))
    if dtype == "f64":
        return torch.rand(n, generator=g, device=dev, dtype=torch.float64) * 0.002 + 0.999
    if dtype == "i32":
        return torch.randint(-(1 << 20), 1 << 20, (n,), generator=g, device=dev, dtype=torch.int32)
    if dtype == "u32":
        return torch.randint(-(1 << 31), (1 << 31) - 1, (n,), generator=g, device=dev,
                             dtype=torch.int32).view(torch.uint32)
    return torch.randint(-(1 << 62), 1 << 62, (n,), generator=g, device=dev, dtype=torch.int64)


def tune_backward(torch, rows=64, cols=1 << 20, reps=5):
    """Pick the backward kernel's launch shape by timing pr_reduce_backward (SUM)
    with CUDA events over the candidate space; the winner is set for every
    differentiable op of the dtype at this size bucket."""
    best = {}
    for dtype in ("f32", "f64"):
        tdt = pr.torch_dtype(dtype)
        x = torch.zeros(rows, cols, dtype=tdt, device="cuda")
        g = torch.ones(rows, dtype=tdt, device="cuda")
        gi = torch.empty_like(x)
        n = rows * cols
        results = []
        for block in (256, 512, 1024):
            for bps in (1, 2, 4, 8):
                if block * bps > 2048:
                    continue
                for unroll in (2, 4):
                    for vb in (16, 32):
                        cfg = dict(block=block, blocks_per_sm=bps, unroll=unroll, vec_bytes=vb)
                        pr.set_config("backward", dtype, "sum", "plain", n, cfg)
                        for _ in range(2):
                            pr.reduce_backward("sum", x, g, out=gi)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        ts = []
                        for _ in range(reps):
                            e0.record()
                            pr.reduce_backward("sum", x, g, out=gi)
                            e1.record()
                            e1.synchronize()
                            ts.append(e0.elapsed_time(e1))
                        results.append((min(ts), cfg))
        t, cfg = min(results, key=lambda r: r[0])
        for op in ("sum", "max", "min", "prod"):
            pr.set_config("backward", dtype, op, "plain", n, cfg)
        best[dtype] = (t, cfg)
        print("backward %dx%d %s: %.1f us %s" % (rows, cols, dtype, t * 1e3, cfg), flush=True)
        del x, gi
    return best


def tune_rows(torch, rows=64, cols=1 << 20):
    """Row reductions as autograd runs them (argidx for max/min, product aux for
    prod), tuned by the library's autotuner for the rows*cols bucket."""
    g = torch.Generator(device="cuda")
    g.manual_seed(2)
    x = torch.randn(rows, cols, generator=g, device="cuda")
    for op in ("sum", "max", "min", "prod"):
        cfg = pr.autotune("rows", x, op)
        print("rows %dx%d f32 %s: %s" % (rows, cols, op, cfg), flush=True)
    del x


def tune_axis(torch):
    """Axis reductions of the bench's 1 GiB shapes (middle axis of [16, 4096,
    4096], first axis of [16384, 16384]), with the library's autotuner."""
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    x = torch.randn(16, 4096, 4096, generator=g, device="cuda")
    for op in ("sum", "max", "min", "prod"):
        cfg = pr.autotune("axis", x, op, dim=1)
        print("axis [16,4096,4096] dim 1 f32 %s: %s" % (op, cfg), flush=True)
    del x


def main():
    import torch
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--sizes", default="20,22,24,26,28,30")
    ap.add_argument("--quick", action="store_true", help="only 2^28 and the segmented workload")
    ap.add_argument("--only", default="reduce,segmented,rows,backward,axis",
                    help="comma list of the parts to re-tune; the other entries of the shipped table are kept")
    args = ap.parse_args()
    parts = set(args.only.split(","))
    sizes = [28] if args.quick else [int(s) for s in args.sizes.split(",")]
    if "reduce" not in parts:
        sizes = []
    torch.cuda.set_device(0)
    pr.lib()                      # loads the shipped table, which the new entries refine
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    for k in sizes:
        n = 1 << k
        for dtype, op in PLAIN:
            if k >= 30 and dtype in ("f64", "i64"):
                continue
            x = _data(torch, dtype, op, n, g)
            cfg = pr.autotune("reduce", x, op)
            print("reduce 2^%d %s %s: %s" % (k, dtype, op, cfg), flush=True)
            del x
        for dtype, prec in PRECISE:
            x = _data(torch, dtype, "sum", n, g)
            cfg = pr.autotune("reduce", x, "sum", precision=prec)
            print("reduce 2^%d %s sum %s: %s" % (k, dtype, prec, cfg), flush=True)
            del x
        torch.cuda.empty_cache()
    if "segmented" in parts:
        vals, off = synth.segmented_workload(4096, synth.config_seed(3))
        xv = torch.from_numpy(vals).cuda()
        ov = torch.from_numpy(off).cuda()
        for op in ("sum", "max", "min", "prod"):
            cfg = pr.autotune("segmented", xv, op, offsets=ov)
            print("segmented 4096 f32 %s: %s" % (op, cfg), flush=True)
        for prec in ("compensated", "fp64_combine"):
            cfg = pr.autotune("segmented", xv, "sum", precision=prec, offsets=ov)
            print("segmented 4096 f32 sum %s: %s" % (prec, cfg), flush=True)
        del xv, ov
    # row reductions and gradients of the differentiation workload (64 rows of 2^20)
    if "rows" in parts:
        tune_rows(torch)
    if "backward" in parts:
        tune_backward(torch)
    if "axis" in parts:
        tune_axis(torch)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    pr.check(pr.pr_tune_save(args.out))
    print("saved", args.out)


if __name__ == "__main__":
    main()
