"""The autotuner on the GPU: what it keeps is one of its candidates, becomes
the configuration in use, and gives results the oracle accepts, the same bits
on every repeat; the tuned table survives a save / load round trip keyed by
the GPU's name and is refused on a GPU of another name."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import pr, synth
from gpu_helpers import to_device, values_of, same_float, sum_bound

pytestmark = pytest.mark.gpu

UNROLLS = (2, 4)
VEC_BYTES = (16, 32)


def is_candidate(kind, c):
    """The candidate space pr_autotune walks (block 64 is tried for axis
    reductions only; the segmented kernel is built for at most 512 threads)."""
    blocks = (128, 256, 512) if kind == "segmented" else (128, 256, 512, 1024)
    return (c["block"] in blocks and c["blocks_per_sm"] in (1, 2, 4, 8) and c["block"] * c["blocks_per_sm"] <= 2048
            and c["unroll"] in UNROLLS and c["vec_bytes"] in VEC_BYTES)


@pytest.fixture
def keep_configs():
    """Restore the configurations a test tunes (the table is process-wide)."""
    saved = []

    def remember(kind, dtype, op, n):
        saved.append((kind, dtype, op, n, pr.get_config(kind, dtype, op, "plain", n)))
    yield remember
    for kind, dtype, op, n, c in saved:
        pr.set_config(kind, dtype, op, "plain", n, c)


@pytest.mark.parametrize("dtype,op", [("f32", "sum"), ("f32", "max"), ("i32", "sum"), ("u32", "xor")])
def test_autotune_reduce_keeps_a_candidate_and_stays_exact(dtype, op, keep_configs):
    n = (1 << 22) + 3
    x = {"f32": synth.uniform_f32, "i32": synth.uniform_i32, "u32": synth.random_u32}[dtype](n, 70)
    t = to_device(x, dtype, 1)
    keep_configs("reduce", dtype, op, n)
    best = pr.autotune("reduce", t, op)
    assert is_candidate("reduce", best), best
    assert pr.get_config("reduce", dtype, op, "plain", n) == best
    od = pr.out_dtype_name(dtype, op)
    first = values_of(pr.reduce(t, op), od)[0]
    if dtype == "f32" and op == "sum":
        assert oracle.sum_error(x, dtype, first) <= sum_bound(x, dtype)
    elif dtype == "f32":
        assert same_float(first, oracle.reduce(x, dtype, op))
    else:
        assert first == oracle.reduce(x, dtype, op)
    for _ in range(3):                                    # a fixed configuration fixes the bits
        again = values_of(pr.reduce(t, op), od)[0]
        assert again == first


def test_autotune_segmented_keeps_a_candidate_and_stays_exact(keep_configs):
    nseg = 300
    off = synth.offsets_from_lengths(synth.segment_lengths(nseg, 71, 100000))
    x = synth.normal_f32(int(off[-1]), 72)
    t = to_device(x, "f32")
    import torch
    o = torch.from_numpy(off).cuda()
    for op in ("sum", "max"):
        keep_configs("segmented", "f32", op, nseg)
        best = pr.autotune("segmented", t, op, offsets=o)
        assert is_candidate("segmented", best), best
        assert pr.get_config("segmented", "f32", op, "plain", nseg) == best
        got = values_of(pr.segmented_reduce(t, o, op), "f32")
        for s in range(nseg):
            seg = x[off[s]:off[s + 1]]
            if op == "sum":
                assert oracle.sum_error(seg, "f32", got[s]) <= sum_bound(seg, "f32"), s
            else:
                assert same_float(got[s], oracle.reduce(seg, "f32", op)), s
        assert values_of(pr.segmented_reduce(t, o, op), "f32") == got


def test_tune_save_load_round_trip(tmp_path, keep_configs):
    import torch
    n = 1 << 20
    keep_configs("reduce", "f32", "min", n)
    keep_configs("reduce", "i32", "max", n)
    a = dict(block=256, blocks_per_sm=4, unroll=4, vec_bytes=16)
    b = dict(block=1024, blocks_per_sm=1, unroll=2, vec_bytes=32)
    pr.set_config("reduce", "f32", "min", "plain", n, a)
    pr.set_config("reduce", "i32", "max", "plain", n, b)
    path = str(tmp_path / "table.json")
    pr.check(pr.pr_tune_save(path))
    with open(path) as f:
        table = json.load(f)                              # the file is valid JSON
    assert table["gpu"] == torch.cuda.get_device_name()
    keys = {(e["kind"], e["dtype"], e["op"], e["precision"], e["bucket"]) for e in table["entries"]}
    assert (0, pr.DTYPES["f32"], pr.OPS["min"], 0, 20) in keys
    # change the configurations in use, then restore them from the file
    pr.set_config("reduce", "f32", "min", "plain", n, b)
    pr.set_config("reduce", "i32", "max", "plain", n, a)
    pr.check(pr.pr_tune_load(path))
    assert pr.get_config("reduce", "f32", "min", "plain", n) == a
    assert pr.get_config("reduce", "i32", "max", "plain", n) == b
    x = synth.uniform_f32(n + 9, 73)
    assert same_float(values_of(pr.reduce(to_device(x, "f32"), "min"), "f32")[0], oracle.reduce(x, "f32", "min"))
    # a table made on a GPU of another name is refused and changes nothing
    table["gpu"] = "not " + table["gpu"]
    for e in table["entries"]:
        e["block"] = 128
    other = str(tmp_path / "other.json")
    with open(other, "w") as f:
        f.write(json.dumps(table).replace("{\"kind\"", "\n {\"kind\""))
    assert pr.pr_tune_load(other) == 1 and "another GPU" in pr.pr_last_error_message()
    assert pr.get_config("reduce", "f32", "min", "plain", n) == a
    assert os.path.exists(path)
