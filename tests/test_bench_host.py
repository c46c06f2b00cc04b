"""Host logic of bench.py that needs no GPU: the oracle checks it records next
to every form (they must accept right results and flag wrong ones), the
multi-core CPU baseline and the CPU model it reports, and the sweep's sizes."""
import os

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import synth

bench = pytest.importorskip("bench")


@pytest.fixture(scope="module")
def chk():
    c = bench.Checker()
    yield c
    c.close()


def test_sum_check_accepts_within_bound_and_flags_beyond(chk):
    x = synth.uniform_f32(200003, 1)
    exact = oracle.exact_sum(x, "f32")
    bound = 1e-6 * oracle.abs_sum(x, "f32")
    assert chk.sum(x, "f32", exact)["ok"]
    assert chk.sum(x, "f32", exact + 0.5 * bound)["ok"]
    r = chk.sum(x, "f32", exact + 2 * bound)
    assert not r["ok"] and r["abs_err"] > r["bound"]
    # compensated: the tighter 2^-24 bound
    assert not chk.sum(x, "f32", exact + 4 * 2.0 ** -24 * oracle.abs_sum(x, "f32"), "compensated")["ok"]


def test_exact_and_product_checks(chk):
    xi = synth.uniform_i32(100000, 2)
    want = oracle.reduce(xi, "i32", "sum")
    assert chk.exact(xi, "i32", "sum", want)["exact"]
    assert not chk.exact(xi, "i32", "sum", want + 1)["exact"]
    xf = synth.uniform_f32(1000, 3)
    assert chk.exact(xf, "f32", "max", oracle.reduce(xf, "f32", "max"))["exact"]
    assert not chk.exact(xf, "f32", "max", 2.0)["exact"]
    d = synth.uniform_f64(5000, 4)
    p = oracle.reduce(d, "f64", "prod")
    assert chk.prod(d, "f64", p)["ok"]
    assert not chk.prod(d, "f64", p * (1 + 1e-9))["ok"]


def test_segment_checks_count_every_segment(chk):
    vals, off = synth.segmented_workload(50, 5, max_len=3000)
    sums = np.array([oracle.exact_sum(vals[off[k]:off[k + 1]], "f32") for k in range(50)], dtype=np.float32)
    r = chk.segments(vals, off, "sum", sums)
    assert r["segments"] == 50 and r["ok"] and r["worst_err_over_bound"] <= 1.0
    bad = sums.copy()
    seg = vals[off[7]:off[8]]
    bad[7] += np.float32(10 * 1e-6 * oracle.abs_sum(seg, "f32") + 1e-3)
    assert not chk.segments(vals, off, "sum", bad)["ok"]
    maxes = np.array([oracle.reduce(vals[off[k]:off[k + 1]], "f32", "max") for k in range(50)], dtype=np.float32)
    assert chk.segments(vals, off, "max", maxes)["mismatches"] == 0
    maxes[3] = -1.0
    assert chk.segments(vals, off, "max", maxes)["mismatches"] == 1


def test_multicore_baseline_and_cpu_model():
    x = synth.uniform_f32(1 << 20, 6)
    v, cores = bench.cpu_chunked_baseline(x, reps=2)
    assert v > 0 and cores == len(os.sched_getaffinity(0))
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_sweep_sizes_span_the_configuration():
    sizes = bench.SWEEP_SIZES
    assert sizes[0] == 1 << 10 and max(sizes) == 1 << 30 and 5_533_214 in sizes
    assert all(1 << e in sizes for e in range(10, 31))


def test_kernel_hash_ignores_comments_only():
    """The traffic record's hash reads the kernel sources' code: comments and
    spacing do not change it, code and string literals do."""
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "a//b /*x*/";\n'
    code = bench._code_only(src)
    assert code == 'int a = 1; const char* s = "a//b /*x*/";'
    assert bench._code_only(src.replace("// note", "// another note")) == code
    assert bench._code_only(src.replace("int a = 1;", "int   a = 1;")) == code
    assert bench._code_only(src.replace("a = 1", "a = 2")) != code
    assert len(bench.kernel_hash()) == 16
