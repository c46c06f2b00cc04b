"""Pins for the CPU oracle: each test checks it against something the paper or
the mathematics fixes (a worked example, a closed form, exact rational
arithmetic, an independent correctly-rounded summation, brute force over all
orders, finite differences), never against the oracle itself."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1710_07358_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32, M64 = 2 ** 32, 2 ** 64


def _exact(a):
    return sum((Fraction(float(v)) for v in np.asarray(a, dtype=np.float64)), Fraction(0))


def _decode(a, dtype):
    """Element values as float64 through numpy's own converters (independent of oracle.c)."""
    if dtype == "bf16":
        return (np.asarray(a, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if dtype == "f16":
        return np.asarray(a).view(np.float16).astype(np.float64)
    return np.asarray(a).astype(np.float64)


# --------------------------------------------------------------------------
# The paper's worked example (Section 1.1 footnote): 1.5 + 4^50 - 4^50
# --------------------------------------------------------------------------

def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([c.strip() for c in line.split("|")])
    return rows


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_footnote_absorption_example(dtype):
    np_t = np.float32 if dtype == "f32" else np.float64
    for order, loop_val, exact_val in _golden_rows("footnote_absorption.txt"):
        terms = []
        for t in order.split(","):
            terms.append(float(eval(t.replace("^", "**"))))
        x = np.array(terms, dtype=np_t)
        # Algorithm 1 in the printed order gives the printed floating-point value...
        if dtype == "f32":
            acc = np.float32(0)
            for v in x:
                acc = np.float32(acc + v)
            assert float(acc) == float(loop_val)
        assert oracle.sum_f64_loop(x, dtype) == float(loop_val)
        # ...and the exact sum is 1.5 in every order.
        assert oracle.exact_sum(x, dtype) == float(exact_val)
        assert oracle.reduce(x, dtype, "sum") == float(exact_val)


# --------------------------------------------------------------------------
# Exact float sum: against exact rational arithmetic and math.fsum
# --------------------------------------------------------------------------

def _mixed_floats(rng, n, dtype):
    mags = rng.uniform(-40, 40, size=n)
    vals = rng.choice([-1.0, 1.0], size=n) * (2.0 ** mags) * rng.random(n)
    if dtype == "f32":
        a = vals.astype(np.float32)
        a[: n // 10] = np.float32(1e-45) * rng.integers(1, 50, size=n // 10)  # subnormals
        return a
    if dtype == "f64":
        a = vals.copy()
        a[: n // 10] = 5e-324 * rng.integers(1, 50, size=n // 10)
        return a
    if dtype == "f16":
        return np.clip(vals, -6e4, 6e4).astype(np.float16)
    return synth.f32_to_bf16_bits(vals.astype(np.float32))


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16"])
def test_exact_sum_matches_rational(dtype):
    rng = np.random.default_rng(1)
    for n in (0, 1, 2, 3, 17, 200):
        a = _mixed_floats(rng, n, dtype)
        ex = _exact(_decode(a, dtype))
        assert oracle.exact_sum(a, dtype) == float(ex)
        assert oracle.abs_sum(a, dtype) == float(sum(abs(Fraction(float(v))) for v in _decode(a, dtype)))
        r = float(rng.standard_normal())
        assert oracle.sum_error(a, dtype, r) == float(abs(ex - Fraction(r)))


def test_exact_sum_rounding_ties_and_cancellation():
    # ties at the 53-bit boundary: 2^53 + 1 -> even (2^53), 2^53 + 3 -> 2^53 + 4
    for parts, want in [([2.0 ** 53, 1.0], 2.0 ** 53), ([2.0 ** 53, 3.0], 2.0 ** 53 + 4),
                        ([2.0 ** 53, 1.0, 2.0 ** -60], 2.0 ** 53 + 2),
                        ([1e308, 1e308, -1e308], 1e308), ([1e308, 1e308], math.inf),
                        ([5e-324, -5e-324, 5e-324], 5e-324), ([-1.0, 0.25], -0.75)]:
        assert oracle.exact_sum(np.array(parts), "f64") == want


def test_exact_sum_matches_fsum_large():
    rng = np.random.default_rng(2)
    for dtype in ("f32", "f64"):
        a = (rng.standard_normal(1_000_000) * 10.0 ** rng.integers(-8, 8, 1_000_000))
        a = a.astype(np.float32 if dtype == "f32" else np.float64)
        assert oracle.exact_sum(a, dtype) == math.fsum(a.astype(np.float64).tolist())


def test_exact_sum_special_values():
    f = lambda *v: np.array(v, dtype=np.float32)
    assert math.isnan(oracle.exact_sum(f(1, np.nan, 2), "f32"))
    assert oracle.exact_sum(f(1, np.inf, 2), "f32") == math.inf
    assert oracle.exact_sum(f(-np.inf, 2), "f32") == -math.inf
    assert math.isnan(oracle.exact_sum(f(np.inf, -np.inf), "f32"))


def test_alg1_loop_within_worst_case_bound():
    rng = np.random.default_rng(3)
    a = rng.uniform(-1, 1, 200_000).astype(np.float32)
    n = a.size
    err = oracle.sum_error(a, "f32", oracle.sum_f64_loop(a, "f32"))
    assert err <= (n - 1) * 2.0 ** -53 * oracle.abs_sum(a, "f32")


def test_half_and_bfloat16_decoding_all_patterns():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    for dtype in ("f16", "bf16"):
        want = _decode(bits, dtype)
        got = np.array([oracle.sum_f64_loop(bits[i:i + 1], dtype) for i in range(65536)])
        same = (got == want) | (np.isnan(got) & np.isnan(want))
        assert same.all(), dtype


# --------------------------------------------------------------------------
# Integer and bitwise combiners: closed forms and brute force
# --------------------------------------------------------------------------

def _xor_upto(m):
    return [m, 1, m + 1, 0][m % 4]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 31, 32, 33, 1000, 65537])
def test_integer_closed_forms(n):
    iota = np.arange(n, dtype=np.int64)
    assert oracle.reduce(iota.astype(np.int32), "i32", "sum") == n * (n - 1) // 2
    assert oracle.reduce(iota, "i64", "sum") == n * (n - 1) // 2
    assert oracle.reduce(iota.astype(np.uint32), "u32", "sum") == (n * (n - 1) // 2) % M32
    assert oracle.reduce(iota.astype(np.uint32), "u32", "xor") == _xor_upto(n - 1)
    assert oracle.reduce(iota.astype(np.int32), "i32", "xor") == _xor_upto(n - 1)
    perm = np.random.default_rng(n).permutation(n)
    for dt, t in (("i32", np.int32), ("u32", np.uint32), ("i64", np.int64)):
        assert oracle.reduce(perm.astype(t), dt, "min") == 0
        assert oracle.reduce(perm.astype(t), dt, "max") == n - 1
    for c in (0, 1, 3, 0x5A5A5A5A, 0xFFFFFFFF):
        const = np.full(n, c, dtype=np.uint32)
        assert oracle.reduce(const, "u32", "and") == c
        assert oracle.reduce(const, "u32", "or") == c
        assert oracle.reduce(const, "u32", "xor") == (c if n % 2 else 0)
        assert oracle.reduce(const, "u32", "sum") == (c * n) % M32
        assert oracle.reduce(const, "u32", "prod") == pow(c, n, M32)
    for c in (-7, 3, 2 ** 20):
        const = np.full(n, c, dtype=np.int32)
        assert oracle.reduce(const, "i32", "sum") == c * n
        p = pow(c % M32, n, M32)
        assert oracle.reduce(const, "i32", "prod") == (p - M32 if p >= 2 ** 31 else p)


def _wrap(v, bits, signed):
    v %= 2 ** bits
    return v - 2 ** bits if signed and v >= 2 ** (bits - 1) else v


def _py_combine(op, a, b):
    return {"sum": a + b, "prod": a * b, "max": max(a, b), "min": min(a, b),
            "and": a & b, "or": a | b, "xor": a ^ b}[op]


@pytest.mark.parametrize("dtype", ["i32", "u32", "i64"])
def test_integer_brute_force_every_order(dtype):
    rng = np.random.default_rng(4)
    t = {"i32": np.int32, "u32": np.uint32, "i64": np.int64}[dtype]
    info = np.iinfo(t)
    for n in range(0, 7):
        x = rng.integers(info.min, info.max, size=n, dtype=t, endpoint=True)
        for op in oracle.OPS:
            bits, signed = (64, True) if (dtype == "i64" or (dtype == "i32" and op == "sum")) else \
                (32, dtype == "i32")
            ident = oracle.identity(dtype, op)
            want = oracle.reduce(x, dtype, op)
            for order in itertools.permutations(range(n)):
                acc = ident
                for i in order:
                    acc = _py_combine(op, acc, int(x[i]))
                if op in ("sum", "prod"):
                    acc = _wrap(acc, bits, signed)
                assert acc == want, (dtype, op, n, order)


def test_int32_sum_widens_to_int64():
    x = np.full(4, 2 ** 31 - 1, dtype=np.int32)
    assert oracle.reduce(x, "i32", "sum") == 4 * (2 ** 31 - 1)


@pytest.mark.parametrize("where", list(range(0, 40)) + list(range(4096 - 40, 4096)))
def test_planted_bits(where):
    n = 4096
    ones = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    bit = 1 << (where % 32)
    assert oracle.reduce(synth.plant(ones, where, 0xFFFFFFFF ^ bit), "u32", "and") == 0xFFFFFFFF ^ bit
    zeros = np.zeros(n, dtype=np.uint32)
    assert oracle.reduce(synth.plant(zeros, where, bit), "u32", "or") == bit
    assert oracle.reduce(synth.plant(zeros, where, bit), "u32", "xor") == bit


# --------------------------------------------------------------------------
# Float max / min: planted extrema, NaN and signed zeros
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "bf16", "i32", "u32", "i64"])
def test_planted_extremum_first_index(dtype):
    n = 2000
    rng = np.random.default_rng(5)
    for where in (0, 1, 37, n // 2, n - 2, n - 1):
        if dtype in ("f32", "f64"):
            base = rng.uniform(-1, 1, n).astype(np.float32 if dtype == "f32" else np.float64)
            hi, lo = 2.0, -2.0
        elif dtype == "f16":
            base = rng.uniform(-1, 1, n).astype(np.float16)
            hi, lo = np.float16(2.0), np.float16(-2.0)
        elif dtype == "bf16":
            base = synth.f32_to_bf16_bits(rng.uniform(-1, 1, n).astype(np.float32))
            hi, lo = synth.f32_to_bf16_bits(np.array([2.0, -2.0], np.float32))
        else:
            t = {"i32": np.int32, "u32": np.uint32, "i64": np.int64}[dtype]
            base = rng.integers(10, 1000, size=n).astype(t)
            hi, lo = t(5000), t(1)
        x = synth.plant(synth.plant(base, where, hi), n - 1 - where if n - 1 - where != where else 0, hi)
        first = min(where, n - 1 - where) if n - 1 - where != where else min(where, 0)
        v, i = oracle.argext(x, dtype, "max")
        assert i == first and v == float(_decode(np.array([hi]), dtype)[0] if dtype in ("f16", "bf16") else hi)
        y = synth.plant(base, where, lo)
        v, i = oracle.argext(y, dtype, "min")
        assert i == where


def test_float_maxmin_nan_and_signed_zero():
    f = lambda *v: np.array(v, dtype=np.float32)
    assert math.isnan(oracle.reduce(f(1, np.nan, 3), "f32", "max"))
    assert math.isnan(oracle.reduce(f(1, np.nan, 3), "f32", "min"))
    v, i = oracle.argext(f(1, np.nan, 3, np.nan), "f32", "max")
    assert math.isnan(v) and i == 1
    for order in ([-0.0, 0.0], [0.0, -0.0]):
        mx = oracle.reduce(f(*order), "f32", "max")
        mn = oracle.reduce(f(*order), "f32", "min")
        assert mx == 0.0 and not math.copysign(1, mx) < 0
        assert mn == 0.0 and math.copysign(1, mn) < 0
    assert oracle.argext(f(-0.0, 0.0, 0.0), "f32", "max")[1] == 1
    assert oracle.argext(f(0.0, -0.0, -0.0), "f32", "min")[1] == 1
    assert oracle.reduce(f(-np.inf, -np.inf), "f32", "max") == -math.inf
    assert oracle.argext(f(), "f32", "max") == (-math.inf, -1)


# --------------------------------------------------------------------------
# Product: exact rationals, special values, no intermediate overflow
# --------------------------------------------------------------------------

def _exact_prod(vals):
    p = Fraction(1)
    for v in vals:
        p *= Fraction(float(v))
    return p


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
def test_prod_matches_rational(dtype):
    rng = np.random.default_rng(6)
    for n in (0, 1, 2, 5, 64, 300):
        v = rng.uniform(0.5, 2.0, n) * rng.choice([-1, 1], n)
        a = {"f64": v, "f32": v.astype(np.float32), "f16": v.astype(np.float16),
             "bf16": synth.f32_to_bf16_bits(v.astype(np.float32))}[dtype]
        want = float(_exact_prod(_decode(a, dtype)))
        got = oracle.reduce(a, dtype, "prod")
        assert got == want or abs(got - want) <= 2.0 ** -52 * abs(want)


def test_prod_closed_forms_and_special_values():
    for c, n in ((2.0, 1000), (0.5, 1074), (-2.0, 3), (1.0 + 2 ** -20, 4096)):
        want = float(Fraction(c) ** n)
        assert oracle.reduce(np.full(n, c), "f64", "prod") == want
    # no intermediate overflow: 2^1000 * 2^1000 * 2^-1000 = 2^1000
    assert oracle.reduce(np.array([2.0 ** 1000, 2.0 ** 1000, 2.0 ** -1000]), "f64", "prod") == 2.0 ** 1000
    f = lambda *v: np.array(v, dtype=np.float64)
    z = oracle.reduce(f(3.0, -0.0, 2.0), "f64", "prod")
    assert z == 0 and math.copysign(1, z) < 0
    assert oracle.reduce(f(3.0, -np.inf), "f64", "prod") == -math.inf
    assert math.isnan(oracle.reduce(f(np.inf, 0.0), "f64", "prod"))
    assert math.isnan(oracle.reduce(f(np.nan, 1.0), "f64", "prod"))
    assert oracle.reduce(f(), "f64", "prod") == 1.0


def test_prod_aux_and_except():
    rng = np.random.default_rng(7)
    x = rng.uniform(0.5, 1.5, 50)
    x[[3, 17, 40]] = 0.0
    p_nz, zc, zi = oracle.prod_aux(x, "f64")
    assert zc == 3 and zi == 3
    assert p_nz == float(_exact_prod(v for v in x if v != 0))
    y = rng.uniform(-1.5, 1.5, 40)
    for i in (0, 7, 39):
        want = float(_exact_prod(np.delete(y, i)))
        got = oracle.prod_except(y, "f64", i)
        assert abs(got - want) <= 2.0 ** -52 * abs(want)


# --------------------------------------------------------------------------
# Gradients: finite differences in float64 pin the gradient oracle
# --------------------------------------------------------------------------

def _fd(f, x, i, h):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


@pytest.mark.parametrize("op", ["sum", "max", "min", "prod"])
def test_gradient_oracle_vs_finite_differences(op):
    rng = np.random.default_rng(8)
    x = rng.uniform(0.5, 1.5, (2, 60))
    if op == "prod":
        x[1, 5] = 0.0              # one zero: only that coordinate has a non-zero gradient
    g = np.array([1.25, -0.5])
    G = oracle.grad(x, "f64", op, g)
    for r in range(2):
        f = lambda v: oracle.reduce(v, "f64", op) * g[r]
        srt = np.sort(x[r])
        gap = min(srt[-1] - srt[-2], srt[1] - srt[0])
        h = min(1e-3, gap / 4)
        for i in range(x.shape[1]):
            fd = _fd(f, x[r].copy(), i, h)
            assert abs(fd - G[r, i]) <= 1e-9 * max(1.0, abs(G[r, i])), (op, r, i)
    if op == "prod":
        assert np.count_nonzero(G[1]) == 1 and G[1, 5] != 0


# --------------------------------------------------------------------------
# Segmented form
# --------------------------------------------------------------------------

def test_segmented_identities_and_totals():
    x = np.arange(100, dtype=np.int32)
    off = np.array([0, 0, 10, 10, 55, 100, 100])
    s = oracle.segmented(x, off, "i32", "sum")
    assert s == [0, 45, 0, sum(range(10, 55)), sum(range(55, 100)), 0]
    assert sum(s) == 99 * 100 // 2
    assert oracle.segmented(x, off, "i32", "max")[0] == -(2 ** 31)
    assert oracle.segmented(x.astype(np.float32), off, "f32", "min")[2] == math.inf
    assert oracle.segmented(x.view(np.uint32), off, "u32", "and")[0] == 0xFFFFFFFF
    am = oracle.segmented_argext(x.astype(np.float32), off, "f32", "max")
    assert am[1] == (9.0, 9) and am[4] == (99.0, 44) and am[0] == (-math.inf, -1)


# --------------------------------------------------------------------------
# Workload generators that the tolerances depend on
# --------------------------------------------------------------------------

@pytest.mark.parametrize("outer,n,inner", [(3, 17, 5), (1, 40, 1), (4, 1, 9), (2, 6, 13)])
def test_axis_oracle_matches_library_reductions(outer, n, inner):
    """Reductions along the middle axis, pinned to numpy's axis reductions on
    exact (integer) data: a transposed or mis-strided slice fails here."""
    rng = np.random.default_rng(outer * 100 + n * 10 + inner)
    xi = rng.integers(-1000, 1000, size=outer * n * inner).astype(np.int32)
    x3 = xi.reshape(outer, n, inner).astype(np.int64)
    assert oracle.axis(xi, "i32", "sum", outer, n, inner) == list(x3.sum(axis=1).reshape(-1))
    assert oracle.axis(xi, "i32", "max", outer, n, inner) == list(x3.max(axis=1).reshape(-1))
    assert oracle.axis(xi, "i32", "min", outer, n, inner) == list(x3.min(axis=1).reshape(-1))
    xu = rng.integers(0, 2 ** 32, size=outer * n * inner, dtype=np.uint64).astype(np.uint32)
    want = np.bitwise_xor.reduce(xu.reshape(outer, n, inner), axis=1).reshape(-1)
    assert oracle.axis(xu, "u32", "xor", outer, n, inner) == [int(v) for v in want]
    # first index of the extremum along the axis: numpy's argmax / argmin take the first too
    am = oracle.axis_argext(xi, "i32", "max", outer, n, inner)
    assert [i for _, i in am] == list(x3.argmax(axis=1).reshape(-1))
    an = oracle.axis_argext(xi, "i32", "min", outer, n, inner)
    assert [i for _, i in an] == list(x3.argmin(axis=1).reshape(-1))
    # float sums: each output is the exact sum of its column
    xf = rng.standard_normal(outer * n * inner).astype(np.float32)
    cols = xf.reshape(outer, n, inner).transpose(0, 2, 1).reshape(-1, n)
    assert oracle.axis(xf, "f32", "sum", outer, n, inner) == [math.fsum(float(v) for v in c) for c in cols]


@pytest.mark.parametrize("dtype,op", [("i32", "sum"), ("u32", "sum"), ("i64", "sum"), ("i32", "max"), ("i32", "min"),
                                      ("u32", "max"), ("i64", "min"), ("u32", "xor"), ("i32", "and"), ("i64", "or"),
                                      ("u32", "prod")])
def test_scan_oracle_matches_library_prefixes(dtype, op):
    """Prefix scans pinned to numpy's accumulate on exact integer data (sums and
    products wrap in the output type), and to the reduction of each prefix."""
    rng = np.random.default_rng(len(dtype) + len(op))
    n = 1000
    if dtype == "i32":
        x = rng.integers(-2 ** 31, 2 ** 31, size=n).astype(np.int32)
    elif dtype == "u32":
        x = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    else:
        x = rng.integers(-2 ** 63, 2 ** 63 - 1, size=n, dtype=np.int64)
    ufunc = {"sum": np.add, "max": np.maximum, "min": np.minimum, "xor": np.bitwise_xor, "and": np.bitwise_and,
             "or": np.bitwise_or, "prod": np.multiply}[op]
    wide = x.astype(np.int64) if (dtype == "i32" and op == "sum") else x
    with np.errstate(over="ignore"):
        want = ufunc.accumulate(wide, dtype=wide.dtype)
    got = oracle.scan(x, dtype, op)
    assert np.array_equal(got, want)
    ex = oracle.scan(x, dtype, op, exclusive=True)
    assert ex[0] == oracle.identity(dtype, op) and np.array_equal(ex[1:], want[:-1])
    for i in (0, 1, 7, 500, n - 1):
        assert int(got[i]) == oracle.reduce(x[:i + 1], dtype, op)


def test_scan_oracle_float_extremes():
    x = np.array([1.0, -0.0, 0.0, 3.0, np.nan, 5.0], dtype=np.float32)
    assert list(oracle.scan(x, "f32", "max"))[:4] == [1.0, 1.0, 1.0, 3.0]
    assert all(math.isnan(v) for v in oracle.scan(x, "f32", "max")[4:])
    mn = oracle.scan(np.array([0.0, -0.0, 0.0], dtype=np.float32), "f32", "min")
    assert [math.copysign(1.0, v) for v in mn] == [1.0, -1.0, -1.0]      # -0 < +0
    ex = oracle.scan(x, "f32", "min", exclusive=True)
    assert ex[0] == math.inf and ex[1] == 1.0
    # every prefix's result is the reduction of that prefix
    r = synth.normal_f32(300, 3)
    got = oracle.scan(r, "f32", "max")
    assert all(got[i] == oracle.reduce(r[:i + 1], "f32", "max") for i in range(300))


def test_axis_oracle_empty_axis_and_rows():
    assert oracle.axis(np.zeros(0, np.float32), "f32", "max", 2, 0, 3) == [-math.inf] * 6
    assert oracle.axis(np.zeros(0, np.int32), "i32", "sum", 2, 0, 3) == [0] * 6
    # inner == 1 is the row reduction
    x = synth.normal_f32(5 * 7, 4)
    assert oracle.axis(x, "f32", "sum", 5, 7, 1) == oracle.segmented(x, np.arange(6) * 7, "f32", "sum")


def test_ill_conditioned_set_cancels_exactly():
    # the exact sum is fixed by construction (pairs cancel, m copies of 2^-10)
    x, n_big, exact = synth.ill_conditioned_f32(2 ** 20, 5)
    assert oracle.exact_sum(x, "f32") == exact
    assert np.count_nonzero(np.abs(x) > 1e7) == n_big
    kappa = oracle.abs_sum(x, "f32") / exact
    assert 5e9 <= kappa <= 2e10
    xs, nb, ex = synth.ill_conditioned_f32(2 ** 16, 5, stress=True)
    assert oracle.exact_sum(xs, "f32") == ex and nb >= 2 ** 15 - 2 ** 13


def test_uniform_generators_stay_in_range():
    a = synth.uniform_f32(1 << 16, 9)
    assert a.min() >= -1.0 and a.max() < 1.0
    d = synth.uniform_f64(1 << 16, 9)
    assert d.min() >= 0.999 and d.max() < 1.001
    lens = synth.segment_lengths(4096, 3)
    assert lens.min() >= 1 and lens.max() <= 2 ** 20


# --------------------------------------------------------------------------
# Table 2's bandwidth column is n*4 bytes / time with GB = 1e9 bytes; the
# benchmark's bandwidth helper must reproduce it.
# --------------------------------------------------------------------------

def test_bandwidth_formula_reproduces_table2():
    from paper_1710_07358_gb300.metrics import gbs
    for F, t_ms, bw, pct in _golden_rows("paper_table2.txt"):
        assert abs(gbs(synth.PAPER_N * 4, float(t_ms) * 1e-3) - float(bw)) < 1e-6
        # the usage column is bandwidth / a peak of ~332.8 GB/s
        assert abs(float(bw) / 332.75 * 100 - float(pct)) < 0.02


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 17])
def test_chunked_multicore_baseline(threads):
    """The multi-core CPU baseline: one thread is Algorithm 1 itself; integer
    valued inputs sum exactly in any order and any chunking; otherwise the
    result lies within the worst case of any double summation order,
    (n - 1) 2^-53 sum |x|, of the exact sum."""
    n = 100003
    x = np.random.default_rng(threads).uniform(-1, 1, n).astype(np.float32)
    got = oracle.sum_f64_chunked(x, "f32", threads)
    if threads == 1:
        assert got == oracle.sum_f64_loop(x, "f32")
    assert abs(got - oracle.exact_sum(x, "f32")) <= (n - 1) * 2.0 ** -53 * oracle.abs_sum(x, "f32")
    ints = np.random.default_rng(threads + 50).integers(-1000, 1000, n).astype(np.float32)
    assert oracle.sum_f64_chunked(ints, "f32", threads) == float(ints.astype(np.int64).sum())
    assert oracle.sum_f64_chunked(x[:0], "f32", threads) == 0.0
    assert oracle.sum_f64_chunked(x[:5], "f32", threads) == pytest.approx(float(x[:5].astype(np.float64).sum()))
