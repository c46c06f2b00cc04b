"""Pins of the line-search oracle against what calculus and the textbook
searches fix, independent of the oracle's own formulas: the derivative of
phi is the BPR link cost along d (fundamental theorem of calculus), p = 1
makes phi a quadratic (constant second difference, closed-form minimiser),
golden-section brackets shrink by r per evaluation and Fibonacci brackets end
at (hi - lo) / F_N, and a dense grid agrees with both searches."""
import math

import numpy as np
import pytest

from oracle import linesearch as ls


def network(n, seed, p_zero_flow=0.0):
    """Synthetic links: capacities, free-flow times, current flows and an
    all-or-nothing direction d = y - x (y: flows of the auxiliary solution)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.uniform(500.0, 4000.0, n).astype(np.float32)
    t0 = rng.uniform(0.5, 5.0, n).astype(np.float32)
    x = (c * rng.uniform(0.2, 1.5, n)).astype(np.float32)
    y = np.where(rng.uniform(size=n) < 0.3, c * rng.uniform(0.0, 3.0, n), 0.0).astype(np.float32)
    if p_zero_flow:
        x[rng.uniform(size=n) < p_zero_flow] = 0.0
    return x, (y - x).astype(np.float32), t0, c


def link_cost(x, d, t0, c, beta, p, alpha):
    """sum_i t0 (1 + beta (v/c)^p) d_i: the cost of each link, along d."""
    x, d, t0, c = (np.asarray(a, dtype=np.float64) for a in (x, d, t0, c))
    v = x + alpha * d
    return math.fsum((t0 * (1.0 + beta * (v / c) ** p) * d).tolist())


@pytest.mark.parametrize("p", [1, 2, 4])
def test_derivative_is_the_link_cost(p):
    x, d, t0, c = network(2000, 1)
    for alpha in (0.0, 0.3, 0.9):
        h = 1e-4
        fd = (ls.phi(x, d, t0, c, 0.15, p, alpha + h) - ls.phi(x, d, t0, c, 0.15, p, alpha - h)) / (2 * h)
        want = link_cost(x, d, t0, c, 0.15, p, alpha)
        assert abs(fd - want) <= 1e-6 * abs(want) + 1e-6


def test_quadratic_case_second_difference_and_minimiser():
    x, d, t0, c = network(3000, 2)
    beta = 0.15
    # constant second difference h^2 * beta * sum t0 d^2 / c
    curv = beta * math.fsum((t0.astype(np.float64) * d.astype(np.float64) ** 2 / c.astype(np.float64)).tolist())
    for alpha, h in ((0.1, 0.05), (0.6, 0.2)):
        sd = ls.phi(x, d, t0, c, beta, 1, alpha + h) - 2 * ls.phi(x, d, t0, c, beta, 1, alpha) \
            + ls.phi(x, d, t0, c, beta, 1, alpha - h)
        assert abs(sd - h * h * curv) <= 1e-8 * abs(ls.phi(x, d, t0, c, beta, 1, alpha)) + 1e-9
    # the closed-form minimiser zeroes the derivative (the link cost along d)
    a_star = ls.quadratic_minimizer(x, d, t0, c, beta)
    scale = math.fsum(np.abs(t0.astype(np.float64) * d).tolist())
    assert abs(link_cost(x, d, t0, c, beta, 1, a_star)) <= 1e-9 * scale


def test_golden_section_widths_and_evaluations():
    f = lambda a: (a - 0.3) ** 2
    for iters in (0, 1, 5, 30):
        a, b, ev = ls.golden_section(f, 0.0, 1.0, iters)
        assert len(ev) == iters + 2
        assert abs((b - a) - ls.GOLDEN ** iters) <= 1e-12
        assert a - 1e-12 <= 0.3 <= b + 1e-12
    assert ls.golden_iterations(0.0, 1.0, 1e-6) == 29     # r^28 > 1e-6 >= r^29
    assert ls.golden_iterations(0.0, 1.0, 2.0) == 0
    # a point evaluated once is reused, never recomputed: all points distinct
    _, _, ev = ls.golden_section(f, 0.0, 1.0, 20)
    assert len({round(p, 15) for p, _ in ev}) == len(ev)


def test_golden_section_monotone_goes_to_the_end():
    a, b, _ = ls.golden_section(lambda t: t, -2.0, 3.0, 40)
    assert abs(a + 2.0) < 1e-7 and b + 2.0 < 1e-7 + 5 * ls.GOLDEN ** 40
    a, b, _ = ls.golden_section(lambda t: -t, -2.0, 3.0, 40)
    assert abs(b - 3.0) < 1e-7


@pytest.mark.parametrize("n_eval", [3, 4, 5, 10, 25])
def test_fibonacci_width_and_evaluations(n_eval):
    f = lambda a: (a - 0.3) ** 2
    a, b, ev = ls.fibonacci_search(f, 0.0, 1.0, n_eval)
    assert len(ev) == n_eval
    u = 1.0 / ls.fibonacci(n_eval)
    assert u * (1 - 1e-9) <= b - a <= 1.1 * u * (1 + 1e-9)
    assert a - 1e-12 <= 0.3 <= b + 1e-12
    assert [ls.fibonacci(k) for k in range(8)] == [1, 1, 2, 3, 5, 8, 13, 21]


def test_fibonacci_beats_golden_for_the_same_evaluations():
    f = lambda a: (a - 0.77) ** 2
    for n in (6, 12, 20):
        fa, fb, _ = ls.fibonacci_search(f, 0.0, 1.0, n)
        ga, gb, _ = ls.golden_section(f, 0.0, 1.0, n - 2)
        assert fb - fa < gb - ga


@pytest.mark.parametrize("p", [1, 4])
def test_searches_agree_with_dense_grid(p):
    x, d, t0, c = network(1500, 3 + p)
    beta = 0.15
    hi = 4.0 if p == 1 else 1.0                # both minimisers interior (about 2.97 and 0.59)
    grid = np.linspace(0.0, hi, 2001)
    step = grid[1] - grid[0]
    vals = [ls.phi(x, d, t0, c, beta, p, g) for g in grid]
    k = int(np.argmin(vals))
    assert 0 < k < len(grid) - 1
    f = lambda a: ls.phi(x, d, t0, c, beta, p, a)
    a, b, _ = ls.golden_section(f, 0.0, hi, ls.golden_iterations(0.0, hi, 1e-6))
    assert a - step <= grid[k] <= b + step
    fa, fb, _ = ls.fibonacci_search(f, 0.0, hi, 30)
    assert fa - step <= grid[k] <= fb + step
    if p == 1:
        a_star = ls.quadratic_minimizer(x, d, t0, c, beta)
        assert a - 1e-9 <= a_star <= b + 1e-9
        assert abs(a_star - grid[k]) <= step


@pytest.mark.parametrize("p", [1, 4, 6])
def test_phi_parts_split_each_term(p):
    """The linear and power parts add up to the term (sharing its sign when
    p + 1 is odd, or where v >= 0), and their derivatives along d are the
    free-flow cost sum t0 d and the congestion cost sum t0 beta (v / c)^p d."""
    x, d, t0, c = network(3000, 5)
    for alpha in (0.0, 0.4, 2.5):
        lin, pw = ls.phi_parts(x, d, t0, c, 0.15, p, alpha)
        t = ls.phi_terms(x, d, t0, c, 0.15, p, alpha)
        assert np.allclose(lin + pw, t, rtol=1e-15, atol=0)
        same = (lin >= 0) if p % 2 else np.ones_like(lin, dtype=bool)
        assert np.all((np.abs(lin) + np.abs(pw))[same] <= np.abs(t)[same] * (1 + 1e-15))
    h, a0 = 1e-4, 0.3
    part = lambda a, k: math.fsum(ls.phi_parts(x, d, t0, c, 0.15, p, a)[k].tolist())
    x64, d64, t64, c64 = (np.asarray(v, dtype=np.float64) for v in (x, d, t0, c))
    v = x64 + a0 * d64
    want_lin = math.fsum((t64 * d64).tolist())
    want_pw = math.fsum((t64 * 0.15 * (v / c64) ** p * d64).tolist())
    assert (part(a0 + h, 0) - part(a0 - h, 0)) / (2 * h) == pytest.approx(want_lin, rel=1e-7)
    assert (part(a0 + h, 1) - part(a0 - h, 1)) / (2 * h) == pytest.approx(want_pw, rel=1e-6)
