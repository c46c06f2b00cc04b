"""Benchmark of the parallel reduction on GB300.

Headline (one JSON line on stdout): reduce GB/s and fraction of the HBM roofline
for the plain fp32 sum over n = 2^28 elements (1 GiB, uniform [-1,1)), inputs
resident in HBM.  A step is one pr_reduce call (one kernel launch); the input is
8x larger than L2, so no flush is needed between steps.

Also reported in the same line:
  e2e          the same metric through pr_reduce_host (pinned host buffer, chunked
               host->device copies, result read back) per step;
  roofline     achieved / measured HBM peak of the dominant kernel, per launch;
  cpu_baseline the CPU oracle (exact fixed-point sum, one host core) on the same data,
               and beside it the chunked multi-core loop over every core the process
               may use (cpu_baseline_multicore), both with the CPU model;
  forms        every op / dtype of the sweep at 2^28, the precision modes, the
               segmented form (4096 log-uniform segments, autotuned, replayed from a
               CUDA graph), forward+backward of [64, 2^20] row reductions, and
               reductions of a non-last axis (1 GiB: middle axis of [16, 4096,
               4096] with its gradient, first axis of [16384, 16384]), one-pass
               prefix scans of 2^28 elements, golden-section / Fibonacci line
               searches of the Beckmann objective over 2^24 links, and the n sweep
               of the fp32 sum (2^10 .. 2^30 and the paper's 5 533 214);
               each form's results are checked against the oracle ("check":
               errors against their bounds, or exactness) in the CPU-baseline leg.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-forms]

With N > 1 (launched by torch.distributed.run) every rank reduces its own copy
of the workload on its own GPU (replicas: the path has no exchange step); the
time is the maximum over ranks and value counts all ranks' bytes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_HEAD = 1 << 28
METRIC = "reduce GB/s & % of HBM peak, n=2^28 fp32 sum; segmented/fwd+bwd vs plain"
WORKLOAD = "plain fp32 sum, n=2^28 uniform[-1,1) (1 GiB), one scalar out"
L2_NOTE = "input 1 GiB > 129 MB L2; no flush needed"
KERNEL_SOURCES = ["common.cuh", "traits.cuh", "kernels.cuh", "inst_f32.cu"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text):
    """C++ source without its comments and blank space: what the compiler
    reads, so that an edit of comments alone keeps a profile's hash."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":                     # string / character literal
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_hash():
    """Hash of the headline kernel's sources (code only, comments stripped)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1710_07358_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_for(key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(key)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def time_launches(fn, steps, warmup, stream):
    """Run fn() warmup + steps times; per-launch CUDA events on `stream`.
    Returns (total ms of the timed region, mean ms per launch)."""
    import torch
    for _ in range(warmup):
        fn()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(steps):
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return t0.elapsed_time(t1), sum(per) / len(per)


def gbs(nbytes, ms):
    from paper_1710_07358_gb300.metrics import gbs as _g
    return _g(nbytes, ms * 1e-3)


def cpu_oracle_sum(x):
    """The oracle's fp32 sum (exact fixed-point accumulation), one host core."""
    import oracle
    t = time.perf_counter()
    oracle.exact_sum(x, "f32")
    return time.perf_counter() - t


def cpu_model():
    """The host CPU's model name as lscpu reports it (else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_chunked_baseline(x, reps=5):
    """The multi-core CPU baseline: Algorithm 1 with a double accumulator per
    contiguous chunk, one chunk per core this process may run on, chunk sums
    added in order.  Returns (GB/s, cores)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.sum_f64_chunked(x, "f32", cores)
    best = None
    for _ in range(reps):
        t = time.perf_counter()
        oracle.sum_f64_chunked(x, "f32", cores)
        dt = time.perf_counter() - t
        best = dt if best is None or dt < best else best
    return gbs(x.size * 4, best * 1e3), cores


class Checker:
    """The oracle leg's checks of every form's results (run after the form's
    timed region, on host copies of its inputs): exact results are compared
    bit for bit, float sums by their exact error against the bounds of
    include/pr.h, products by relative error.  Independent oracle calls run
    on a thread pool (the oracle's C loops release the GIL)."""

    def __init__(self):
        import concurrent.futures
        import oracle
        self.oracle = oracle
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(os.sched_getaffinity(0))))

    @staticmethod
    def host(t):
        """numpy copy of a CUDA tensor in the oracle's storage type."""
        import numpy as np
        import torch
        if t.dtype in (torch.bfloat16, torch.float16):
            a = t.view(torch.int16).cpu().numpy().view(np.uint16)
            return a.view(np.float16) if t.dtype == torch.float16 else a
        if hasattr(torch, "uint32") and t.dtype == torch.uint32:
            return t.view(torch.int32).cpu().numpy().view(np.uint32)
        return t.cpu().numpy()

    @staticmethod
    def value(t):
        """Python value of a 0-d CUDA result tensor."""
        import torch
        if hasattr(torch, "uint32") and t.dtype == torch.uint32:
            return int(t.view(torch.int32).item()) & 0xFFFFFFFF
        if t.dtype in (torch.bfloat16, torch.float16):
            return float(t.float().item())
        return t.item()

    def sum(self, x, dtype, got, precision="plain"):
        o = self.oracle
        fa = self.pool.submit(o.abs_sum, x, dtype)
        fe = self.pool.submit(o.sum_error, x, dtype, float(got))
        a, err = fa.result(), fe.result()
        bound = 2.0 ** -24 * a if precision == "compensated" else 1e-6 * a
        return {"abs_err": err, "bound": bound, "rel_to_sum_abs": err / a if a else 0.0, "ok": err <= bound}

    def exact(self, x, dtype, op, got):
        want = self.oracle.reduce(x, dtype, op)
        ok = (got == want) if not isinstance(want, float) else (got == want or (got != got and want != want))
        return {"exact": bool(ok)}

    def prod(self, x, dtype, got):
        want = self.oracle.reduce(x, dtype, "prod")
        rel = abs(got - want) / abs(want) if want else abs(got)
        bound = max(x.size - 1, 1) * (2.0 ** -53 if dtype == "f64" else 2.0 ** -24)
        return {"rel_err": rel, "bound": bound, "ok": rel <= bound}

    def segments(self, x, off, op, got):
        """Every segment: sums by exact error, max by equality."""
        o = self.oracle
        nseg = len(off) - 1

        def one(k):
            seg = x[off[k]:off[k + 1]]
            if op == "sum":
                a = o.abs_sum(seg, "f32")
                e = o.sum_error(seg, "f32", float(got[k]))
                return e, 1e-6 * a
            v = o.reduce(seg, "f32", op)
            return (0.0 if v == float(got[k]) else float("inf")), 0.0
        errs = list(self.pool.map(one, range(nseg)))
        worst = max(e / b if b else (0.0 if e == 0 else float("inf")) for e, b in errs)
        return {"segments": nseg, "worst_err_over_bound" if op == "sum" else "mismatches":
                worst if op == "sum" else sum(1 for e, _ in errs if e), "ok": worst <= 1.0}

    def close(self):
        self.pool.shutdown()


# --------------------------------------------------------------------------
# Secondary forms (all on the same GPU, same run)
# --------------------------------------------------------------------------

FORM_GROUPS = ("plain", "precision", "illcond", "segmented", "fwdbwd", "axis", "scan", "linesearch", "sweep")


def forms(steps, warmup, peak, only=None, tune=True, chk=None):
    """Every form at its workload size.  With a Checker (the oracle leg),
    each form's results are then checked against the oracle: the record's
    "check" entry."""
    import numpy as np
    import torch
    from paper_1710_07358_gb300 import pr, synth
    from paper_1710_07358_gb300.autograd import RowReduce  # noqa: F401  (same kernels as below)
    st = torch.cuda.current_stream()
    k = max(3, min(steps, 30))
    res = {}
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)

    def plain(name, t, op, dtype=None, **kw):
        nb = t.numel() * t.element_size()
        out = pr.reduce(t, op, **kw)
        _, per = time_launches(lambda: pr.reduce(t, op, out=out, **kw), k, warmup, st)
        res[name] = {"GB/s": round(gbs(nb, per), 1), "frac": round(gbs(nb, per) / peak, 4),
                     "us": round(per * 1e3, 2)}
        if chk is not None:
            torch.cuda.synchronize()
            got = chk.value(out)
            x = chk.host(t)
            d = dtype or pr.dtype_name(t)
            if op == "sum" and d in ("f32", "f16", "bf16"):
                res[name]["check"] = chk.sum(x, d, got, kw.get("precision", "plain"))
            elif op == "prod" and d in ("f32", "f64"):
                res[name]["check"] = chk.prod(x, d, got)
            else:
                res[name]["check"] = chk.exact(x, d, op, got)

    want = set(only or FORM_GROUPS)
    n = N_HEAD
    g.manual_seed(synth.config_seed(1))
    if "plain" in want or "precision" in want:
        f32 = torch.rand(n, generator=g, device=dev) * 2 - 1
    if "plain" in want:
        for op in ("sum", "max", "min"):
            plain("f32_%s" % op, f32, op)
        nb = f32.numel() * 4
        _, per = time_launches(lambda: pr.reduce_arg(f32, "max"), k, warmup, st)
        res["f32_argmax"] = {"GB/s": round(gbs(nb, per), 1), "frac": round(gbs(nb, per) / peak, 4),
                             "us": round(per * 1e3, 2)}
        if chk is not None:
            v, i = pr.reduce_arg(f32, "max")
            wv, wi = chk.oracle.argext(chk.host(f32), "f32", "max")
            res["f32_argmax"]["check"] = {"exact": float(v.item()) == wv and int(i.item()) == wi}
        i32 = torch.randint(-(1 << 20), 1 << 20, (n,), generator=g, device=dev, dtype=torch.int32)
        for op in ("sum", "max", "min"):
            plain("i32_%s" % op, i32, op)
        del i32
        u32 = torch.randint(-(1 << 31), (1 << 31) - 1, (n,), generator=g, device=dev,
                            dtype=torch.int32).view(torch.uint32)
        for op in ("and", "or", "xor"):
            plain("u32_%s" % op, u32, op)
        del u32
        f64 = torch.rand(n, generator=g, device=dev, dtype=torch.float64) * 0.002 + 0.999
        plain("f64_prod", f64, "prod")
        del f64
    if "precision" in want:
        for dt, name in ((torch.bfloat16, "bf16"), (torch.float16, "f16")):
            h = torch.randn(n, generator=g, device=dev).to(dt)
            plain("%s_sum" % name, h, "sum", dtype=name)
            plain("%s_sum_compensated" % name, h, "sum", dtype=name, precision="compensated")
            del h
        plain("f32_sum_compensated", f32, "sum", precision="compensated")
        plain("f32_sum_fp64_combine", f32, "sum", precision="fp64_combine")
    if "plain" in want or "precision" in want:
        del f32
    if "illcond" in want:
        ill(res, k, warmup, peak, st)
    if "segmented" in want:
        segmented(res, k, warmup, peak, tune, chk)
    if "fwdbwd" in want:
        fwdbwd(res, k, warmup, peak, st, g, chk)
    if "axis" in want:
        axis(res, k, warmup, peak, st, g, chk)
    if "scan" in want:
        scan(res, k, warmup, peak, st, g, chk)
    if "linesearch" in want:
        linesearch(res, k, warmup, peak, st, g, chk)
    if "sweep" in want:
        sweep(res, k, warmup, peak, st, g)
    return res


SWEEP_SIZES = [1 << e for e in range(10, 31)] + [5_533_214]      # the paper's vector length last
L2_BYTES = 129 << 20


def sweep(res, k, warmup, peak, st, g):
    """The plain fp32 sum from n = 2^10 to 2^30, and the paper's n = 5 533 214.

    Below 4x L2 (n < 2^27) two numbers: "hot_us", the per-call time of a CUDA
    graph of 64 back-to-back calls on L2-resident data (the latency regime);
    and "cold_us" with L2 flushed before every call (a 512 MiB write outside
    the timed region, followed by a 256 MiB read that evicts the written
    lines), from which GB/s.  From 2^27 on the input is at least
    4x L2 and calls are timed back to back.  Every n is a prefix of one 4 GiB
    buffer (aligned like a fresh allocation)."""
    import torch
    from paper_1710_07358_gb300 import pr
    dev = torch.device("cuda")
    g.manual_seed(11)
    big = torch.rand((1 << 30) + 64, generator=g, device=dev) * 2 - 1
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    evict = torch.empty(64 << 20, dtype=torch.float32, device=dev).fill_(1.0)
    out = torch.empty((), dtype=torch.float32, device=dev)
    rows = []
    for n in SWEEP_SIZES:
        x = big[:n]
        nb = 4 * n
        rec = {"n": n}
        if nb < 4 * L2_BYTES:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                pr.prepare(s)
                pr.reduce(x, "sum", out=out, stream=s)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                for _ in range(64):
                    pr.reduce(x, "sum", out=out, stream=s)
            for _ in range(2):
                graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                graph.replay()
            e1.record()
            torch.cuda.synchronize()
            rec["hot_us"] = round(e0.elapsed_time(e1) * 1e3 / (5 * 64), 3)
            per = []
            for _ in range(k + warmup):
                # flush: a 512 MiB write, then a 256 MiB read that evicts its
                # dirty lines, so no write-back overlaps the timed call
                flush.zero_()
                evict.sum()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                pr.reduce(x, "sum", out=out)
                b.record(st)
                per.append((a, b))
            torch.cuda.synchronize()
            # the mean: single event pairs tick in steps of about 2 us, and
            # the launches' phase against those steps varies
            cold = [a.elapsed_time(b) for a, b in per[warmup:]]
            ms = sum(cold) / len(cold)
            rec["cold_us"] = round(ms * 1e3, 3)
        else:
            _, ms = time_launches(lambda: pr.reduce(x, "sum", out=out), k, warmup, st)
            rec["us"] = round(ms * 1e3, 2)
        rec["GB/s"] = round(gbs(nb, ms), 1)
        rec["frac"] = round(gbs(nb, ms) / peak, 4)
        rows.append(rec)
    res["sweep_f32_sum"] = {"l2_rule": "n*4 < 4 x 129 MB: 512 MiB write + 256 MiB read before each cold call; "
                                       "hot = CUDA graph of 64 calls on L2-resident data",
                            "points": rows}
    del big, flush, evict


def scan(res, k, warmup, peak, st, g, chk=None):
    """One-pass prefix scans of n = 2^28 (or the --n-log2 size): uint32 sum (offsets of a counting
    sort: 1 GiB read + 1 GiB written), int32 sum widening to int64 (1 GiB read,
    2 GiB written) and fp32 running max (1 GiB + 1 GiB).  Bandwidth counts the
    bytes read and written, like the copy that sets the measured peak."""
    import torch
    from paper_1710_07358_gb300 import pr
    dev = torch.device("cuda")
    n = N_HEAD                  # 2^28 unless --n-log2 asks for a profiling case
    g.manual_seed(9)
    xi = torch.randint(0, 1 << 8, (n,), generator=g, device=dev, dtype=torch.int32)
    yu = torch.empty(n, dtype=torch.int32, device=dev)

    def put(name, per, nbytes):
        res[name] = {"GB/s": round(gbs(nbytes, per), 1), "frac": round(gbs(nbytes, per) / peak, 4),
                     "us": round(per * 1e3, 2)}

    xu = xi.view(torch.uint32) if hasattr(torch, "uint32") else xi
    _, per = time_launches(lambda: pr.check(pr.pr_scan(xu.data_ptr(), n, pr.DTYPES["u32"], pr.OPS["sum"], 1,
                                                       yu.data_ptr(), st.cuda_stream)), k, warmup, st)
    put("scan_u32_sum_exclusive", per, 2 * n * 4)
    import numpy as np
    if chk is not None:                              # every element against the oracle's loop
        xh = chk.host(xi)
        want = chk.oracle.scan(xh.view(np.uint32), "u32", "sum", True)
        res["scan_u32_sum_exclusive"]["check"] = {"exact": bool(np.array_equal(chk.host(yu).view(np.uint32), want))}
        del want
    y64 = torch.empty(n, dtype=torch.int64, device=dev)
    _, per = time_launches(lambda: pr.scan(xi, "sum", out=y64), k, warmup, st)
    put("scan_i32_sum_to_i64", per, n * 4 + n * 8)
    if chk is not None:
        res["scan_i32_sum_to_i64"]["check"] = {
            "exact": bool(np.array_equal(chk.host(y64), chk.oracle.scan(xh, "i32", "sum", False)))}
        del xh
    del y64, yu
    xf = torch.randn(n, generator=g, device=dev)
    yf = torch.empty_like(xf)
    _, per = time_launches(lambda: pr.scan(xf, "max", out=yf), k, warmup, st)
    put("scan_f32_max", per, 2 * n * 4)
    if chk is not None:
        res["scan_f32_max"]["check"] = {"exact": bool(np.array_equal(
            chk.host(yf).astype(np.float64), chk.oracle.scan(chk.host(xf), "f32", "max", False)))}
    del xf, yf, xi


def linesearch(res, k, warmup, peak, st, g, chk=None):
    """Golden-section (tolerance 1e-6 on [0, 1]: 29 iterations) and Fibonacci
    (31 evaluations) search of the Beckmann objective (BPR, beta 0.15, power
    4) over 2^24 synthetic links: four float32 arrays, 256 MiB per pass, more
    than L2 holds.  One evaluation pass alone is timed first, with 2 and 6
    points; then the searches, where depth D decides D iterations per pass
    over the links.  GB/s counts 16 bytes per link and pass."""
    import torch
    from paper_1710_07358_gb300 import pr, synth
    dev = torch.device("cuda")
    n = 1 << 24
    g.manual_seed(synth.config_seed(7))
    u = lambda lo, hi: torch.rand(n, generator=g, device=dev) * (hi - lo) + lo
    c = u(500.0, 4000.0)
    t0 = u(0.5, 5.0)
    x = c * u(0.2, 1.5)
    y = torch.where(torch.rand(n, generator=g, device=dev) < 0.3, c * u(0.0, 3.0), torch.zeros_like(c))
    d = y - x
    del y
    nb = 16 * n
    for m in (2, 6):
        al = torch.linspace(0.1, 0.9, m, dtype=torch.float64, device=dev)
        ph = torch.empty(m, dtype=torch.float64, device=dev)
        _, per = time_launches(lambda: pr.check(pr.pr_beckmann(x.data_ptr(), d.data_ptr(), t0.data_ptr(),
                                                               c.data_ptr(), n, 0.15, 4, al.data_ptr(), m,
                                                               ph.data_ptr(), st.cuda_stream)), k, warmup, st)
        res["beckmann_pass_%dpts" % m] = {"us": round(per * 1e3, 2), "GB/s": round(gbs(nb, per), 1),
                                          "frac": round(gbs(nb, per) / peak, 4)}
    out = torch.empty(4, dtype=torch.float64, device=dev)
    iters = pr.golden_iterations(0.0, 1.0, 1e-6)
    for method, count in (("golden", iters), ("fibonacci", 31)):
        total = count if method == "golden" else count - 2
        for depth in (1, 2, 3):
            passes = max(1, -(-total // depth))
            _, per = time_launches(lambda: pr.line_search(x, d, t0, c, method=method, count=count, depth=depth,
                                                          result=out), k, warmup, st)
            res["linesearch_%s_d%d" % (method, depth)] = {
                "us": round(per * 1e3, 1), "passes": passes, "GB/s": round(gbs(nb * passes, per), 1),
                "frac": round(gbs(nb * passes, per) / peak, 4), "alpha": round(float(out[2].item()), 7)}
            if chk is not None and depth == 2:
                # phi at the point the search kept, against the oracle's sum
                # of float64 terms, within the evaluation's derived bound
                import numpy as np
                from oracle import linesearch as ols
                arrs = [chk.host(v) for v in (x, d, t0, c)]
                a32, b32 = float(np.float32(out[2].item())), float(np.float32(0.15))
                want = ols.phi(*arrs, b32, 4, a32)
                lin, pw = ols.phi_parts(*arrs, b32, 4, a32)
                bound = 1.001 * 2.0 ** -24 * (8 * float(np.abs(lin).sum()) + 29 * float(np.abs(pw).sum()))
                err = abs(float(out[3].item()) - want)
                width = float(out[1].item()) - float(out[0].item())
                res["linesearch_%s_d%d" % (method, depth)]["check"] = {
                    "phi_abs_err": err, "bound": bound, "ok": err <= bound, "bracket_width": width}
    del x, d, t0, c


def axis(res, k, warmup, peak, st, g, chk=None):
    """Reductions of a non-last axis, 1 GiB each: the middle axis of
    [16, 4096, 4096] fp32 (sum; max with its first index) and its gradient,
    and the first axis of [16384, 16384] (a column reduction)."""
    import torch
    from paper_1710_07358_gb300 import pr
    dev = torch.device("cuda")
    g.manual_seed(7)
    x = torch.randn(16, 4096, 4096, generator=g, device=dev)
    nb = x.numel() * 4

    def put(name, per, nbytes):
        res[name] = {"GB/s": round(gbs(nbytes, per), 1), "frac": round(gbs(nbytes, per) / peak, 4),
                     "us": round(per * 1e3, 2)}

    _, per = time_launches(lambda: pr.reduce_axis(x, "sum", 1), k, warmup, st)
    put("axis_mid_sum", per, nb)
    cols = [(0, 0), (5, 1234), (15, 4095)]           # sampled outputs (slab, column)
    if chk is not None:
        ys = pr.reduce_axis(x, "sum", 1)
        worst = 0.0
        for p, q in cols:
            col = chk.host(x[p, :, q].contiguous())
            r = chk.sum(col, "f32", float(ys[p, q].item()))
            worst = max(worst, r["abs_err"] / r["bound"])
        res["axis_mid_sum"]["check"] = {"sampled_outputs": len(cols), "worst_err_over_bound": worst,
                                        "ok": worst <= 1.0}
    _, per = time_launches(lambda: pr.reduce_axis(x, "max", 1, argidx=True), k, warmup, st)
    put("axis_mid_max_arg", per, nb)
    if chk is not None:
        ym, yi = pr.reduce_axis(x, "max", 1, argidx=True)
        ok = all(chk.oracle.argext(chk.host(x[p, :, q].contiguous()), "f32", "max") ==
                 (float(ym[p, q].item()), int(yi[p, q].item())) for p, q in cols)
        res["axis_mid_max_arg"]["check"] = {"sampled_outputs": len(cols), "exact": ok}
    gout = torch.randn(16, 4096, generator=g, device=dev)
    gi = torch.empty_like(x)
    _, per = time_launches(lambda: pr.reduce_axis_backward("sum", x, 1, gout, out=gi), k, warmup, st)
    put("axis_mid_sum_bwd", per, nb)
    if chk is not None:                              # d(sum)/dx = grad_out broadcast along the axis, exactly
        res["axis_mid_sum_bwd"]["check"] = {"exact": bool(torch.equal(gi, gout[:, None, :].expand_as(gi)))}
    del x, gi
    c = torch.randn(16384, 16384, generator=g, device=dev)
    _, per = time_launches(lambda: pr.reduce_axis(c, "sum", 0), k, warmup, st)
    put("axis_col_sum", per, c.numel() * 4)
    if chk is not None:
        yc = pr.reduce_axis(c, "sum", 0)
        worst = 0.0
        for q in (0, 7777, 16383):
            r = chk.sum(chk.host(c[:, q].contiguous()), "f32", float(yc[q].item()))
            worst = max(worst, r["abs_err"] / r["bound"])
        res["axis_col_sum"]["check"] = {"sampled_outputs": 3, "worst_err_over_bound": worst, "ok": worst <= 1.0}
    del c


def ill(res, k, warmup, peak, st):
    import numpy as np
    import torch
    from paper_1710_07358_gb300 import pr, synth
    dev = torch.device("cuda")

    def plain(name, t, op, **kw):
        nb = t.numel() * t.element_size()
        _, per = time_launches(lambda: pr.reduce(t, op, **kw), k, warmup, st)
        res[name] = {"GB/s": round(gbs(nb, per), 1), "frac": round(gbs(nb, per) / peak, 4),
                     "us": round(per * 1e3, 2)}

    # precision: ill-conditioned fp32 set, error against the exact sum (known by construction)
    x, n_big, exact = synth.ill_conditioned_f32(1 << 26, synth.config_seed(2))
    xt = torch.from_numpy(x).to(dev)
    abs_sum = float(np.abs(x.astype(np.float64)).sum())
    errs = {}
    for prec in ("plain", "fp64_combine", "compensated"):
        v = pr.reduce(xt, "sum", precision=prec).item()
        bound = (2.0 ** -24 if prec == "compensated" else 1e-6) * abs_sum
        errs[prec] = {"result": v, "abs_err": abs(v - exact), "err_over_sum_abs": abs(v - exact) / abs_sum,
                      "bound": bound, "ok": abs(v - exact) <= bound}
    plain("f32_illcond_compensated", xt, "sum", precision="compensated")
    res["illcond_errors"] = {"n": 1 << 26, "exact": exact, "kappa": abs_sum / exact, **errs}
    del xt


def segmented(res, k, warmup, peak, tune=True, chk=None):
    import torch
    from paper_1710_07358_gb300 import pr, synth
    dev = torch.device("cuda")
    # segmented: 4096 log-uniform segments, autotuned, replayed from a CUDA graph
    vals, off = synth.segmented_workload(4096, synth.config_seed(3))
    xv = torch.from_numpy(vals).to(dev)
    ov = torch.from_numpy(off).to(dev)
    seg_bytes = 4 * vals.size + 8 * off.size + 4 * 4096
    for op in ("sum", "max"):
        cfg = pr.autotune("segmented", xv, op, offsets=ov) if tune else \
            pr.get_config("segmented", "f32", op, "plain", 4096)
        out = torch.empty(4096, dtype=torch.float32, device=dev)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            pr.prepare(s)
            pr.check(pr.pr_segmented_reduce(xv.data_ptr(), ov.data_ptr(), 4096, 0, pr.OPS[op], out.data_ptr(),
                                            s.cuda_stream))
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            pr.check(pr.pr_segmented_reduce(xv.data_ptr(), ov.data_ptr(), 4096, 0, pr.OPS[op], out.data_ptr(),
                                            s.cuda_stream))
        _, per = time_launches(graph.replay, k, warmup, torch.cuda.current_stream())
        res["segmented_%s" % op] = {"GB/s": round(gbs(seg_bytes, per), 1), "frac": round(gbs(seg_bytes, per) / peak, 4),
                                    "us": round(per * 1e3, 2), "elements": int(vals.size), "config": cfg,
                                    "graph": True}
        if chk is not None:
            torch.cuda.synchronize()
            res["segmented_%s" % op]["check"] = chk.segments(vals, off, op, out.cpu().numpy())
    del xv, ov


def fwdbwd(res, k, warmup, peak, st, g, chk=None):
    import torch
    from paper_1710_07358_gb300 import pr
    dev = torch.device("cuda")
    # differentiation: [64, 2^20] fp32, forward + backward
    rows, cols = 64, 1 << 20
    xr = torch.randn(rows, cols, generator=g, device=dev)
    xp = torch.rand(rows, cols, generator=g, device=dev) + 0.5
    xp[torch.rand(rows, cols, generator=g, device=dev) < 0.01] = 0.0
    go = torch.linspace(-1, 1, rows, device=dev)
    mat = rows * cols * 4
    for op in ("sum", "max", "prod"):
        xin = xp if op == "prod" else xr

        def fwd():
            if op == "sum":
                return pr.reduce_rows(xin, op), None
            if op == "max":
                return pr.reduce_rows(xin, op, argidx=True)
            return pr.reduce_rows(xin, op, aux=True)

        y, extra = fwd()
        gi = torch.empty_like(xin)

        def bwd():
            if op == "max":
                pr.reduce_backward(op, xin, go, argidx=extra, out=gi)
            elif op == "prod":
                pr.reduce_backward(op, xin, go, aux=extra, out=gi)
            else:
                pr.reduce_backward(op, xin, go, out=gi)

        _, pf = time_launches(fwd, k, warmup, st)
        _, pb = time_launches(bwd, k, warmup, st)
        res["fwd_bwd_%s" % op] = {"fwd_GB/s": round(gbs(mat, pf), 1), "bwd_GB/s": round(gbs(mat, pb), 1),
                                  "fwd_bwd_GB/s": round(gbs(2 * mat, pf + pb), 1),
                                  "frac": round(gbs(2 * mat, pf + pb) / peak, 4),
                                  "us": round((pf + pb) * 1e3, 2)}
        if chk is not None:
            res["fwd_bwd_%s" % op]["check"] = fwdbwd_check(chk, op, xin, go, gi)


def fwdbwd_check(chk, op, xin, go, gi):
    """Sampled rows of the forward against the oracle, and the backward by
    the properties that fix it: sum -> grad_out broadcast; max -> one-hot at
    the first argmax; prod (every row here has two or more zeros) -> 0."""
    import torch
    from paper_1710_07358_gb300 import pr
    rows = (0, 31, 63)
    if op == "sum":
        y = pr.reduce_rows(xin, "sum")
        worst = 0.0
        for r in rows:
            rr = chk.sum(chk.host(xin[r]), "f32", float(y[r].item()))
            worst = max(worst, rr["abs_err"] / rr["bound"])
        return {"sampled_rows": len(rows), "fwd_worst_err_over_bound": worst,
                "bwd_exact": bool(torch.equal(gi, go[:, None].expand_as(gi))), "ok": worst <= 1.0}
    if op == "max":
        y, ai = pr.reduce_rows(xin, "max", argidx=True)
        fwd_ok = all(chk.oracle.argext(chk.host(xin[r]), "f32", "max") == (float(y[r].item()), int(ai[r].item()))
                     for r in rows)
        onehot = torch.zeros_like(gi).scatter_(1, ai[:, None], go[:, None])
        return {"sampled_rows": len(rows), "fwd_exact": fwd_ok, "bwd_exact": bool(torch.equal(gi, onehot))}
    y, ax = pr.reduce_rows(xin, "prod", aux=True)
    _, zc, zi = pr.prod_aux_fields(ax)
    fwd_ok = all(chk.oracle.prod_aux(chk.host(xin[r]), "f32")[1:] == (int(zc[r].item()), int(zi[r].item()))
                 for r in rows)
    return {"sampled_rows": len(rows), "fwd_zero_count_and_index_exact": fwd_ok,
            "fwd_all_zero": bool(torch.all(y == 0)), "bwd_all_zero": int(torch.count_nonzero(gi).item()) == 0}


# --------------------------------------------------------------------------
# Arms
# --------------------------------------------------------------------------

def smi_index(local):
    """nvidia-smi's index of CUDA device `local` (honours CUDA_VISIBLE_DEVICES)."""
    ids = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if local < len(ids) and ids[local].isdigit():
        return int(ids[local])
    return local


def gpu_local_cpus(index):
    """CPUs of the NUMA node the GPU is attached to (sysfs), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        dom, rest = out.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s/local_cpulist" % (int(dom, 16) & 0xffff, rest)
        with open(path) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus & os.sched_getaffinity(0) or None
    except Exception:
        return None


def pinned_near_gpu(x_host, index):
    """Pinned host copy of x_host placed on the GPU's NUMA node: the pages are
    allocated and first touched by this process bound to that node's CPUs."""
    import torch
    cpus = gpu_local_cpus(index)
    old = os.sched_getaffinity(0)
    try:
        if cpus:
            os.sched_setaffinity(0, cpus)
        t = torch.empty(x_host.shape, dtype=torch.from_numpy(x_host[:1]).dtype).pin_memory()
        t.copy_(torch.from_numpy(x_host))
    finally:
        os.sched_setaffinity(0, old)
    return t, sorted(cpus) if cpus else None


def max_over_ranks(v: float, device="cpu") -> float:
    """The largest of every rank's v (one all-reduce MAX; v itself when this
    process is the only rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle on the host cores, same workload and metric (bounded sample per step)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1710_07358_gb300 import synth
    oracle.build()
    x = synth.uniform_f32(N_HEAD, synth.config_seed(1))
    # size each step's sample so that warmup + steps take about two minutes
    probe = x[: 1 << 20]
    t = time.perf_counter()
    oracle.exact_sum(probe, "f32")
    per_elem = max((time.perf_counter() - t) / probe.size, 1e-10)
    total = max(args.steps + args.warmup, 1)
    m = int(min(N_HEAD, max(1 << 16, 120.0 / total / per_elem)))
    sample = x[:m]
    for _ in range(args.warmup):
        oracle.exact_sum(sample, "f32")
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.exact_sum(sample, "f32")
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    v = gbs(m * 4, dt * 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_HEAD, "op": "sum", "dtype": "f32",
                                           "parallelism": "replicas" if world > 1 else "single",
                                           "l2": L2_NOTE},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "model": cpu_model(),
                             "sample": "first %d elements of the n=2^28 workload per step" % m},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1710_07358_gb300 import pr, synth
    peak, peak_src = measured_peaks()

    x_host = synth.uniform_f32(N_HEAD, synth.config_seed(1))
    x = torch.from_numpy(x_host).to(dev)
    out = torch.empty((), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    nbytes = N_HEAD * 4

    def step():
        pr.reduce(x, "sum", out=out)

    # the clock sampler starts first (nvidia-smi needs a moment before its
    # first sample), then the warm-up steps run directly before the timed
    # ones: an idle gap after the warm-up slows the first timed launches
    sampler = ClockSampler(smi_index(dev.index))
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms, per_launch = time_launches(step, args.steps, 0, st)
    clocks = sampler.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms, dev)
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = gbs(nbytes * world, ms_per_step)

    # correctness of the timed result (exactness bound) on rank 0
    res_val = out.item()

    # end to end: pinned host buffer through the C ABI
    e2e = None
    if not args.no_e2e:
        pinned, near = pinned_near_gpu(x_host, smi_index(dev.index))
        ke = max(3, min(args.steps, 10))
        pr.reduce_host(pinned, "sum")
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t = time.perf_counter()
        for _ in range(ke):
            pr.reduce_host(pinned, "sum")
        e2e_s = time.perf_counter() - t
        if world > 1:
            e2e_s = max_over_ranks(e2e_s, dev)
        e2e_s /= ke
        e2e = {"value": round(gbs(nbytes * world, e2e_s * 1e3), 1), "unit": "GB/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": 4, "steps": ke,
               "host_buffer": "pinned, on the GPU's NUMA node (cpus %s)" % (
                   "%d-%d" % (near[0], near[-1]) if near else "unknown")}

    achieved = gbs(nbytes, per_launch)
    cfg = pr.get_config("reduce", "f32", "sum", "plain", N_HEAD)
    plan = pr.reduce_plan(x, "sum")
    traffic = traffic_for("reduce_f32_sum_2^28")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, copy)",
                "kernel": "k_reduce<SumF<LdF32,float>,U=%d,VB=%d,TAIL=%d>" % (
                    cfg["unroll"], cfg["vec_bytes"], 1 if plan["tail_vectors"] else 0),
                "claimed_tail_vectors": plan["tail_vectors"],
                "algorithmic_bytes_per_launch": nbytes, "launch_us": round(per_launch * 1e3, 2)}

    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_HEAD, "op": "sum", "dtype": "f32",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": L2_NOTE, "launch": cfg},
            "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps, "roofline": roofline,
            "result": res_val}
    chk = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle and the chunked multi-core loop,
        # timed on the host cores, then every GPU result of this run checked
        # against the oracle
        model = cpu_model()
        dt = cpu_oracle_sum(x_host)
        line["cpu_baseline"] = {"value": round(gbs(nbytes, dt * 1e3), 4), "unit": "GB/s", "cores": 1,
                                "kind": "oracle", "model": model,
                                "sample": "whole n=2^28 workload once (exact fixed-point sum, one core)"}
        mt, cores = cpu_chunked_baseline(x_host)
        line["cpu_baseline_multicore"] = {"value": round(mt, 2), "unit": "GB/s", "cores": cores,
                                          "kind": "Algorithm 1 per contiguous chunk, float64 accumulators, "
                                                  "chunk sums in order", "model": model,
                                          "sample": "whole n=2^28 workload, best of 5"}
        import oracle
        line["abs_err_vs_exact"] = oracle.sum_error(x_host, "f32", res_val)
        line["err_bound_1e-6_sum_abs"] = 1e-6 * oracle.abs_sum(x_host, "f32")
        chk = Checker()
    if rank == 0 and world == 1 and not args.no_forms:
        del x
        torch.cuda.empty_cache()
        line["forms"] = forms(args.steps, args.warmup, peak, tune=not args.no_tune, chk=chk)
    if chk is not None:
        chk.close()
        bad = sorted(k for k, v in line.get("forms", {}).items() if isinstance(v, dict) and "check" in v and
                     not all(v["check"].get(f, True) for f in ("ok", "exact", "fwd_exact", "bwd_exact",
                                                                "fwd_zero_count_and_index_exact",
                                                                "fwd_all_zero", "bwd_all_zero")))
        line["checks_failed"] = bad
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="segmented form: use the shipped tuning table instead of re-running the autotuner")
    ap.add_argument("--forms-only", default=None,
                    help="comma list of %s: run only these secondary forms (profiling)" % ",".join(FORM_GROUPS))
    ap.add_argument("--n-log2", type=int, default=28,
                    help="headline size 2^k (28 is the measured workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global N_HEAD, WORKLOAD
    if args.n_log2 != 28:
        N_HEAD = 1 << args.n_log2
        WORKLOAD = "plain fp32 sum, n=2^%d uniform[-1,1) (profiling case, not the measured workload)" % args.n_log2
    if args.impl == "reference":
        return run_reference(args)
    if args.forms_only:
        return run_forms_only(args)
    return run_ours(args)


def run_forms_only(args):
    import torch
    torch.cuda.set_device(0)
    peak, _ = measured_peaks()
    only = [f.strip() for f in args.forms_only.split(",") if f.strip()]
    print(json.dumps({"forms": forms(args.steps, args.warmup, peak, only, tune=not args.no_tune)}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
