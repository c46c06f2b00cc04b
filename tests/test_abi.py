"""C-ABI checks that need no GPU: the library loads, exports every function
include/pr.h declares, and rejects bad arguments on the host with the
documented status before anything is enqueued."""
import ctypes
import os
import re

import pytest

from paper_1710_07358_gb300 import pr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OK, INVALID, UNSUPPORTED, CUDA = 0, 1, 2, 3
F32, F16, BF16, F64, I32, U32, I64 = range(7)
SUM, PROD, MAX, MIN, AND, OR, XOR = range(7)
PLAIN, COMP, F64C = range(3)
FAKE = 0x10000      # an aligned address that is never dereferenced (validation fails first)


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(pr.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pr.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_python_binding_mirrors_c_names():
    for n in declared_functions():
        assert callable(getattr(pr, n)), n


def test_version_and_status_strings(L):
    assert pr.pr_version().startswith("pr ")
    for code, name in pr.STATUS.items():
        assert pr.pr_status_string(code) == name


def test_out_dtype_table(L):
    table = {(F32, SUM): F32, (F16, SUM): F32, (BF16, SUM): F32, (F16, MAX): F16, (BF16, MIN): BF16,
             (F16, PROD): F32, (F64, PROD): F64, (I32, SUM): I64, (I32, MAX): I32, (I32, PROD): I32,
             (U32, SUM): U32, (U32, XOR): U32, (I64, SUM): I64}
    for (d, o), want in table.items():
        assert pr.pr_out_dtype(d, o) == want


def _msg():
    return pr.pr_last_error_message()


@pytest.mark.parametrize("args,status,needle", [
    ((FAKE, -1, F32, SUM, FAKE, None), INVALID, "n must be"),
    ((None, 10, F32, SUM, FAKE, None), INVALID, "x is NULL"),
    ((FAKE, 10, F32, SUM, None, None), INVALID, "out is NULL"),
    ((FAKE, 10, F32, AND, FAKE, None), UNSUPPORTED, "bitwise"),
    ((FAKE, 10, BF16, XOR, FAKE, None), UNSUPPORTED, "bitwise"),
    ((FAKE, 10, 99, SUM, FAKE, None), INVALID, "dtype"),
    ((FAKE, 10, F32, 42, FAKE, None), INVALID, "op"),
    ((FAKE + 2, 10, F32, SUM, FAKE, None), INVALID, "aligned"),
    ((FAKE + 4, 10, F64, MAX, FAKE, None), INVALID, "aligned"),
])
def test_reduce_rejects(L, args, status, needle):
    assert pr.pr_reduce(*args) == status
    assert needle in _msg()


def test_reduce_ex_precision_and_out_dtype_rules(L):
    assert pr.pr_reduce_ex(FAKE, 10, I32, SUM, COMP, I64, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_ex(FAKE, 10, F32, MAX, F64C, F32, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_ex(FAKE, 10, F64, SUM, COMP, F64, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_ex(FAKE, 10, F32, SUM, PLAIN, F64, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_ex(FAKE, 10, F32, SUM, 7, F32, FAKE, None) == INVALID


def test_segmented_rejects(L):
    assert pr.pr_segmented_reduce(FAKE, FAKE, -1, F32, SUM, FAKE, None) == INVALID
    assert pr.pr_segmented_reduce(FAKE, None, 4, F32, SUM, FAKE, None) == INVALID
    assert pr.pr_segmented_reduce(None, FAKE, 4, F32, SUM, FAKE, None) == INVALID
    assert pr.pr_segmented_reduce(FAKE, FAKE, 4, F32, SUM, None, None) == INVALID
    assert pr.pr_segmented_reduce_aux(FAKE, FAKE, 4, F32, SUM, PLAIN, FAKE, FAKE, None, None) == UNSUPPORTED
    assert pr.pr_segmented_reduce_aux(FAKE, FAKE, 4, F32, MAX, PLAIN, FAKE, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_segmented_reduce_aux(FAKE, FAKE, 4, F16, PROD, PLAIN, FAKE, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_segmented_reduce(FAKE, FAKE, 4, F32, OR, FAKE, None) == UNSUPPORTED
    # zero segments: nothing to do, nothing enqueued
    assert pr.pr_segmented_reduce(None, None, 0, F32, SUM, None, None) == OK


def test_rows_and_backward_reject(L):
    assert pr.pr_reduce_rows(FAKE, -1, 4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_rows(FAKE, 2 ** 40, 2 ** 40, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_rows(None, 4, 4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_backward(SUM, I32, FAKE, 4, 4, FAKE, None, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_backward(AND, F32, FAKE, 4, 4, FAKE, None, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_backward(MAX, F32, None, 4, 4, FAKE, None, None, FAKE, None) == INVALID
    assert pr.pr_reduce_backward(PROD, F32, None, 4, 4, FAKE, None, FAKE, FAKE, None) == INVALID
    assert pr.pr_reduce_backward(SUM, F32, None, 0, 4, None, None, None, None, None) == OK


def test_axis_rejects(L):
    assert pr.pr_reduce_axis(FAKE, -1, 4, 4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_axis(FAKE, 2, 4, -4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_axis(FAKE, 2 ** 40, 2 ** 20, 2 ** 10, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_axis(None, 2, 4, 4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    assert pr.pr_reduce_axis(FAKE, 2, 4, 4, F32, SUM, PLAIN, None, None, None, None) == INVALID
    assert pr.pr_reduce_axis(FAKE, 2, 4, 4, F32, XOR, PLAIN, FAKE, None, None, None) == UNSUPPORTED
    assert pr.pr_reduce_axis(FAKE, 2, 4, 4, F32, SUM, PLAIN, FAKE, FAKE, None, None) == UNSUPPORTED
    assert pr.pr_reduce_axis(FAKE, 2, 4, 4, I32, PROD, PLAIN, FAKE, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_axis(FAKE + 2, 2, 4, 4, F32, SUM, PLAIN, FAKE, None, None, None) == INVALID
    # nothing to compute: no outputs
    assert pr.pr_reduce_axis(None, 0, 4, 4, F32, SUM, PLAIN, None, None, None, None) == OK
    assert pr.pr_reduce_axis(None, 3, 4, 0, F32, SUM, PLAIN, None, None, None, None) == OK
    assert pr.pr_reduce_axis_backward(SUM, I32, FAKE, 2, 4, 4, FAKE, None, None, FAKE, None) == UNSUPPORTED
    assert pr.pr_reduce_axis_backward(MAX, F32, None, 2, 4, 4, FAKE, None, None, FAKE, None) == INVALID
    assert pr.pr_reduce_axis_backward(PROD, F32, None, 2, 4, 4, FAKE, None, FAKE, FAKE, None) == INVALID
    assert pr.pr_reduce_axis_backward(SUM, F32, None, 2, 4, -1, FAKE, None, None, FAKE, None) == INVALID
    assert pr.pr_reduce_axis_backward(SUM, F32, None, 2, 0, 4, None, None, None, None, None) == OK
    best = pr.pr_config()
    assert pr.pr_autotune_axis(None, 2, 4, 4, F32, SUM, PLAIN, None, ctypes.byref(best)) == INVALID
    assert pr.pr_autotune_axis(FAKE, 2, 4, 1, F32, SUM, PLAIN, None, ctypes.byref(best)) == INVALID
    assert pr.pr_autotune_axis(FAKE, 2, 4, 4, F32, AND, PLAIN, None, ctypes.byref(best)) == UNSUPPORTED
    # the axis kind has its own configurations
    c = pr.pr_config(64, 4, 2, 32)
    assert pr.pr_set_config(4, F32, MAX, PLAIN, 1 << 20, ctypes.byref(c)) == OK
    got = pr.pr_config()
    assert pr.pr_get_config(4, F32, MAX, PLAIN, 1 << 20, ctypes.byref(got)) == OK and got.as_dict() == c.as_dict()


def test_scan_rejects(L):
    assert pr.pr_scan(FAKE, -1, I32, SUM, 0, FAKE, None) == INVALID
    assert pr.pr_scan(None, 4, I32, SUM, 0, FAKE, None) == INVALID
    assert pr.pr_scan(FAKE, 4, I32, SUM, 0, None, None) == INVALID
    assert pr.pr_scan(FAKE, 4, F32, SUM, 0, FAKE, None) == UNSUPPORTED
    assert pr.pr_scan(FAKE, 4, BF16, PROD, 1, FAKE, None) == UNSUPPORTED
    assert pr.pr_scan(FAKE, 4, 99, SUM, 0, FAKE, None) == INVALID
    assert pr.pr_scan(FAKE + 2, 4, I32, MAX, 0, FAKE, None) == INVALID
    assert pr.pr_scan(FAKE, 4, I32, SUM, 0, FAKE + 4, None) == INVALID   # int64 output alignment
    assert pr.pr_scan(None, 0, I32, SUM, 0, None, None) == OK
    assert pr.pr_scan(FAKE, 1 << 45, U32, SUM, 0, FAKE, None) == INVALID   # 2^32 tiles of 32 KB
    assert pr.pr_check_bounded_wait(0, None) == INVALID


def test_host_path_rejects(L):
    assert pr.pr_reduce_host(None, 5, F32, SUM, FAKE, None) == INVALID
    assert pr.pr_reduce_host(FAKE, 5, F32, SUM, None, None) == INVALID
    assert pr.pr_reduce_host(FAKE, 5, F32, XOR, FAKE, None) == UNSUPPORTED


def test_config_roundtrip_and_validation(L):
    c = pr.pr_config(512, 2, 4, 16)
    assert pr.pr_set_config(0, F32, SUM, PLAIN, 1 << 20, ctypes.byref(c)) == OK
    got = pr.pr_config()
    assert pr.pr_get_config(0, F32, SUM, PLAIN, (1 << 20) + 5, ctypes.byref(got)) == OK
    assert got.as_dict() == c.as_dict()
    for bad in ((100, 2, 4, 16), (512, 0, 4, 16), (512, 2, 3, 16), (512, 2, 4, 8), (2048, 1, 4, 16)):
        assert pr.pr_set_config(0, F32, SUM, PLAIN, 1, ctypes.byref(pr.pr_config(*bad))) == INVALID
    # the segmented kernel runs blocks of at most 512 threads
    assert pr.pr_set_config(1, F32, SUM, PLAIN, 1, ctypes.byref(pr.pr_config(1024, 1, 4, 32))) == INVALID
    assert pr.pr_set_config(1, F32, SUM, PLAIN, 1, ctypes.byref(pr.pr_config(512, 1, 4, 32))) == OK


def test_valid_call_without_a_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    # validation passes, the CUDA runtime then reports the missing device
    assert pr.pr_reduce(FAKE, 10, F32, SUM, FAKE, None) == CUDA
    with pytest.raises(pr.PrError):
        pr.check(pr.pr_reduce(FAKE, 10, F32, SUM, FAKE, None))


def test_line_search_rejections():
    """Argument checks of pr_beckmann and pr_line_search (all on the host)."""
    F = FAKE
    ok = (F, F, F, F, 100, 0.15, 4)
    assert pr.pr_beckmann(F, F, F, F, -1, 0.15, 4, F, 2, F, None) == INVALID
    assert pr.pr_beckmann(None, F, F, F, 100, 0.15, 4, F, 2, F, None) == INVALID
    assert pr.pr_beckmann(F + 2, F, F, F, 100, 0.15, 4, F, 2, F, None) == INVALID      # 4-byte alignment
    assert pr.pr_beckmann(F, F, F, F, 100, -1.0, 4, F, 2, F, None) == INVALID          # beta < 0
    assert pr.pr_beckmann(F, F, F, F, 100, float("nan"), 4, F, 2, F, None) == INVALID
    assert pr.pr_beckmann(F, F, F, F, 100, 0.15, 0, F, 2, F, None) == INVALID          # power
    assert pr.pr_beckmann(F, F, F, F, 100, 0.15, 17, F, 2, F, None) == INVALID
    assert pr.pr_beckmann(*ok, F, 0, F, None) == INVALID                                # m
    assert pr.pr_beckmann(*ok, F, 17, F, None) == INVALID
    assert pr.pr_beckmann(*ok, None, 2, F, None) == INVALID
    assert pr.pr_beckmann(*ok, F + 4, 2, F, None) == INVALID                            # 8-byte alignment
    assert pr.pr_line_search(*ok, 1.0, 1.0, 0, 10, 2, F, None) == INVALID               # lo < hi
    assert pr.pr_line_search(*ok, 0.0, float("inf"), 0, 10, 2, F, None) == INVALID
    assert pr.pr_line_search(*ok, 0.0, 1.0, 2, 10, 2, F, None) == INVALID               # method
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, -1, 2, F, None) == INVALID              # golden iterations
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, 201, 2, F, None) == INVALID
    assert pr.pr_line_search(*ok, 0.0, 1.0, 1, 2, 2, F, None) == INVALID               # Fibonacci evaluations
    assert pr.pr_line_search(*ok, 0.0, 1.0, 1, 79, 2, F, None) == INVALID
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, 10, 0, F, None) == INVALID              # depth
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, 10, 4, F, None) == INVALID
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, 10, 2, None, None) == INVALID
    assert pr.pr_line_search(*ok, 0.0, 1.0, 0, 10, 2, F + 4, None) == INVALID


def test_golden_iteration_count_closed_form(L):
    """pr_golden_iterations returns the smallest K with (hi - lo) r^K <= tol,
    r = (sqrt 5 - 1) / 2: the bracket after K iterations is within tol and
    the one after K - 1 is not."""
    import math
    r = (math.sqrt(5.0) - 1.0) / 2.0
    for lo, hi in ((0.0, 1.0), (-3.0, 5.0), (0.25, 0.2500001), (10.0, 1e6)):
        for tol in (1e-12, 1e-9, 1e-6, 1e-3, 0.5, 100.0, 1e7):
            k = pr.golden_iterations(lo, hi, tol)
            assert (hi - lo) * r ** k <= tol
            assert k == 0 or (hi - lo) * r ** (k - 1) > tol
    assert pr.golden_iterations(0.0, 1.0, 1e-6) == 29            # the benchmark's search: r^29 = 8.7e-7
    k = ctypes.c_int32(-1)
    for bad in ((1.0, 1.0, 1e-3), (0.0, 1.0, 0.0), (0.0, 1.0, -1.0), (0.0, float("inf"), 1e-3),
                (0.0, 1.0, float("nan")), (0.0, 1.0, 1e-300)):
        assert pr.pr_golden_iterations(*bad, ctypes.byref(k)) == INVALID
    assert pr.pr_golden_iterations(0.0, 1.0, 1e-3, None) == INVALID


def test_fault_hook_arguments_and_validation_order(L):
    """The host-side fault hook: bad arguments are refused; argument checks run
    before it, so rejected calls neither fire nor consume an armed fault."""
    pending = ctypes.c_int32(7)
    assert pr.pr_debug_inject_fault(3, 0, ctypes.byref(pending)) == INVALID
    assert pr.pr_debug_inject_fault(-1, 0, None) == INVALID
    assert pr.pr_debug_inject_fault(1, -1, None) == INVALID
    assert pr.inject_fault("none") is False
    for site in ("launch", "alloc"):
        assert pr.inject_fault(site, after=2) is False
        assert pr.pr_reduce(FAKE, -1, F32, SUM, FAKE, None) == INVALID
        assert pr.pr_segmented_reduce(FAKE, None, 4, F32, SUM, FAKE, None) == INVALID
        assert pr.pr_scan(None, 4, I32, SUM, 0, FAKE, None) == INVALID
        assert pr.pr_reduce_backward(MAX, F32, None, 4, 4, FAKE, None, None, FAKE, None) == INVALID
        assert pr.pr_line_search(FAKE, FAKE, FAKE, FAKE, 100, 0.15, 4, 1.0, 1.0, 0, 10, 2, FAKE, None) == INVALID
        assert pr.inject_fault("none") is True            # still armed: nothing consumed it
        assert pr.inject_fault("none") is False


def test_reduce_plan_rejects(L):
    """The launch-plan query validates like the reductions it describes, on the
    host, before it touches a device."""
    g, b, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    refs = (ctypes.byref(g), ctypes.byref(b), ctypes.byref(t))
    assert pr.pr_debug_reduce_plan(FAKE, -1, F32, SUM, 0, 0, None, *refs) == INVALID
    assert pr.pr_debug_reduce_plan(None, 4, F32, SUM, 0, 0, None, *refs) == INVALID
    assert pr.pr_debug_reduce_plan(FAKE, 4, 99, SUM, 0, 0, None, *refs) == INVALID
    assert pr.pr_debug_reduce_plan(FAKE, 4, F32, SUM, 0, 1, None, *refs) == UNSUPPORTED   # arg needs MAX / MIN
    assert pr.pr_debug_reduce_plan(FAKE, 4, F32, 4, 0, 0, None, *refs) == UNSUPPORTED     # AND on floats
