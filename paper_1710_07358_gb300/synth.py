"""Seeded synthetic inputs shaped like the workloads the library is measured on.

This module only draws numbers; it contains no reduction arithmetic and is
shared by the CUDA-path tests, the oracle tests and the benchmark so that both
sides see identical inputs.  Every generator is a pure function of its seed
(numpy PCG64), so x86-64 and AArch64 hosts produce the same bytes.

Workloads (the paper's own vector is n = 5,533,214 int32/fp32 elements,
Section 4):
  plain sweep:   fp32 U[-1,1), int32 U[-2^20,2^20), uint32 random bits,
                 fp64 U[0.999,1.001)
  precision:     bf16 / fp16 N(0,1); fp32 ill-conditioned (+-1e8 pairs and
                 +-N(0,1)*1e-3 pairs that cancel exactly, plus copies of 2^-10;
                 condition ~1e10)
  batching:      segment lengths ceil(exp(U(0, ln 2^20))) -> CSR int64 offsets,
                 fp32 N(0,1) values
  differentiation: [64, 2^20] fp32 N(0,1); product rows U[0.5,1.5) with 1 %
                 exact zeros
  line search:   a road network's links: capacities U[500, 4000), free-flow
                 times U[0.5, 5), flows x = c U[0.2, 1.5), an all-or-nothing
                 auxiliary flow y (30 % of links loaded with c U[0, 3), the
                 rest 0) and the direction d = y - x
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20171020
PAPER_N = 5_533_214


def config_seed(i: int) -> int:
    return BASE_SEED + i


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_f32(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """fp32 uniform on [lo, hi): (hi-lo)*u + lo with u drawn directly as fp32 in [0,1)."""
    u = _rng(seed).random(n, dtype=np.float32)
    out = u * np.float32(hi - lo) + np.float32(lo)
    return np.minimum(out, np.nextafter(np.float32(hi), np.float32(lo)))


def uniform_f64(n: int, seed: int, lo: float = 0.999, hi: float = 1.001) -> np.ndarray:
    u = _rng(seed).random(n, dtype=np.float64)
    return np.minimum(u * (hi - lo) + lo, np.nextafter(hi, lo))


def uniform_i32(n: int, seed: int, lo: int = -(2 ** 20), hi: int = 2 ** 20) -> np.ndarray:
    return _rng(seed).integers(lo, hi, size=n, dtype=np.int32)


def random_u32(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(0, 2 ** 32, size=n, dtype=np.uint32)


def random_i64(n: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(-(2 ** 63), 2 ** 63 - 1, size=n, dtype=np.int64)


def normal_f32(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return (_rng(seed).standard_normal(n, dtype=np.float32) * np.float32(scale)).astype(np.float32)


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round fp32 to bfloat16 (nearest, ties to even); returns the 16-bit patterns."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    nan = np.isnan(a)
    out = rounded.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def normal_bf16(n: int, seed: int) -> np.ndarray:
    """bf16 N(0,1) as uint16 bit patterns."""
    return f32_to_bf16_bits(normal_f32(n, seed))


def normal_f16(n: int, seed: int) -> np.ndarray:
    """fp16 N(0,1) (numpy float16, rounded to nearest)."""
    return normal_f32(n, seed).astype(np.float16)


def ill_conditioned_f32(n: int, seed: int, kappa: float = 1e10, stress: bool = False):
    """fp32 values whose exact sum is tiny relative to sum|x|, known by construction.

    * big values in exact pairs (+B_k, -B_k), B_k = fp32(1e8*(1+u_k)), u_k ~ U[0,1);
    * small values in exact pairs (+s_i, -s_i), s_i = fp32(N(0,1)*1e-3);
    * m copies of 2^-10 (~1e-3), so the exact sum is m * 2^-10.
    All elements are permuted with the seed.  m = min(8192, n/8) and the number
    of big pairs is chosen so that sum|x| / (m 2^-10) ~ kappa (E|B| = 1.5e8).
    With stress=True half of the elements are big (condition ~1e15).
    Returns (values, number of big elements, exact sum).
    """
    rng = _rng(seed)
    m = max(1, min(8192, n // 8))
    exact = m * 2.0 ** -10
    if stress:
        n_big = ((n - m) // 2) & ~1
    else:
        n_big = 2 * max(1, int(round(kappa * exact / (2.0 * 1.5e8))))
        n_big = min(n_big, ((n - m) // 2) & ~1)
    n_pairs = (n - m - n_big) // 2
    m = n - n_big - 2 * n_pairs                  # absorbs an odd remainder
    exact = m * 2.0 ** -10
    small = (rng.standard_normal(n_pairs, dtype=np.float32) * np.float32(1e-3)).astype(np.float32)
    b = (np.float32(1e8) * (np.float32(1.0) + rng.random(n_big // 2, dtype=np.float32))).astype(np.float32)
    vals = np.concatenate([small, -small, b, -b, np.full(m, 2.0 ** -10, dtype=np.float32)])
    perm = rng.permutation(n)
    return vals[perm].astype(np.float32), n_big, exact


def segment_lengths(nseg: int, seed: int, max_len: int = 2 ** 20) -> np.ndarray:
    """Log-uniform lengths ceil(exp(U(0, ln max_len))) in [1, max_len]."""
    u = _rng(seed).random(nseg)
    return np.clip(np.ceil(np.exp(u * math.log(max_len))), 1, max_len).astype(np.int64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    """CSR offsets (int64, nseg+1 entries, starting at 0)."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def segmented_workload(nseg: int, seed: int, max_len: int = 2 ** 20):
    """(fp32 N(0,1) values, int64 offsets) for nseg log-uniform segments."""
    off = offsets_from_lengths(segment_lengths(nseg, seed, max_len))
    return normal_f32(int(off[-1]), seed + 1000), off


def rows_normal(rows: int, cols: int, seed: int) -> np.ndarray:
    return normal_f32(rows * cols, seed).reshape(rows, cols)


def prod_rows(rows: int, cols: int, seed: int, zero_frac: float = 0.01) -> np.ndarray:
    """[rows, cols] fp32 U[0.5,1.5) with a fraction of elements set exactly to 0."""
    x = uniform_f32(rows * cols, seed, 0.5, 1.5)
    z = _rng(seed + 7).random(rows * cols) < zero_frac
    x[z] = 0.0
    return x.reshape(rows, cols)


def plant(x: np.ndarray, idx: int, value) -> np.ndarray:
    """Copy of x with x[idx] = value (for planted-extremum / planted-bit cases)."""
    y = np.array(x, copy=True)
    y.reshape(-1)[idx] = value
    return y


def network_links(n: int, seed: int):
    """float32 (x, d, t0, c) of n links: flows, direction y - x, free-flow
    times and capacities of a Frank-Wolfe step (see the module docstring)."""
    rng = _rng(seed)
    c = rng.uniform(500.0, 4000.0, n).astype(np.float32)
    t0 = rng.uniform(0.5, 5.0, n).astype(np.float32)
    x = (c * rng.uniform(0.2, 1.5, n)).astype(np.float32)
    y = np.where(rng.uniform(size=n) < 0.3, c * rng.uniform(0.0, 3.0, n), 0.0).astype(np.float32)
    return x, (y - x).astype(np.float32), t0, c
