"""CPU oracle for the line search that uses the reduction as its inner step.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests, the smoke
check and the benchmark's CPU legs are its only callers.

Section 1 names golden-section and Fibonacci search among the consumers of a
reduction, and Section 5 places the golden-ratio method inside the traffic
assignment step: there each evaluation of the objective is one sum over every
link of the network.  The objective here is that step's objective, the
Beckmann function of BPR link costs along a search direction:

    phi(alpha) = sum_i t0_i * (v_i + beta * c_i / (p + 1) * (v_i / c_i)^(p + 1)),
    v_i = x_i + alpha * d_i,

with x, d, t0, c float32 arrays (flows, direction, free-flow times,
capacities), beta >= 0 and an integer power p >= 1.  Each term is evaluated in
float64 from the float32 inputs and the terms are summed with ``math.fsum``
(correctly rounded), so phi is the float64 rounding of the exact sum of the
float64 terms.

Both searches keep a bracket [a, b] with two interior points lo < hi and
their values; each iteration compares the two values, keeps the part of the
bracket around the better point (ties keep [lo, b]), reuses the retained
point, and evaluates one new point.  The point positions are computed in
plain float64 operations, in the order written, so that another
implementation using the same operations places the same points.

Parity is pinned in the tests by closed forms (p = 1 makes phi a quadratic),
by the textbook bracket widths, and by brute force over a dense grid.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0          # r = 1 / golden ratio


def phi_terms(x, d, t0, c, beta: float, p: int, alpha: float) -> np.ndarray:
    """float64 terms of phi(alpha) from the float32 inputs."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    d = np.asarray(d, dtype=np.float32).astype(np.float64)
    t0 = np.asarray(t0, dtype=np.float32).astype(np.float64)
    c = np.asarray(c, dtype=np.float32).astype(np.float64)
    v = x + float(alpha) * d
    q = v / c
    return t0 * (v + float(beta) * c / (p + 1) * q ** (p + 1))


def phi_parts(x, d, t0, c, beta: float, p: int, alpha: float):
    """The two parts of every term, in float64: the linear part t0 v and the
    power part t0 beta c / (p + 1) (v / c)^(p + 1).  Both have the sign of v,
    so |term| = |linear| + |power|; an evaluation's error bound weighs the
    two parts differently (the power part takes more roundings)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    d = np.asarray(d, dtype=np.float32).astype(np.float64)
    t0 = np.asarray(t0, dtype=np.float32).astype(np.float64)
    c = np.asarray(c, dtype=np.float32).astype(np.float64)
    v = x + float(alpha) * d
    return t0 * v, t0 * float(beta) * c / (p + 1) * (v / c) ** (p + 1)


def phi(x, d, t0, c, beta: float, p: int, alpha: float) -> float:
    """The objective at alpha: correctly rounded sum of the float64 terms."""
    return math.fsum(phi_terms(x, d, t0, c, beta, p, alpha).tolist())


def golden_iterations(lo: float, hi: float, tol: float) -> int:
    """Iterations after the first two evaluations until the bracket is at most
    tol wide: the smallest K >= 0 with (hi - lo) * r^K <= tol."""
    if hi - lo <= tol:
        return 0
    return int(math.ceil(math.log(tol / (hi - lo)) / math.log(GOLDEN) - 1e-12))


def fibonacci(k: int) -> float:
    """F_0 = F_1 = 1, F_k = F_{k-1} + F_{k-2}, by float64 additions (exact up
    to F_77, then IEEE-rounded)."""
    a, b = 1.0, 1.0
    for _ in range(k - 1):
        a, b = b, a + b
    return b if k >= 1 else 1.0


def golden_section(f, lo: float, hi: float, iters: int):
    """Golden-section search (Kiefer 1953) of f on [lo, hi] with `iters`
    iterations after the two initial evaluations.  Points of the bracket
    [a, b]: b - r (b - a) and a + r (b - a).  Returns (a, b, evaluations) with
    evaluations the list of (alpha, f(alpha)) in the order made."""
    a, b = float(lo), float(hi)
    x1 = b - GOLDEN * (b - a)
    x2 = a + GOLDEN * (b - a)
    f1, f2 = f(x1), f(x2)
    ev = [(x1, f1), (x2, f2)]
    for _ in range(iters):
        if f1 < f2:
            b = x2
            x2, f2 = x1, f1
            x1 = b - GOLDEN * (b - a)
            f1 = f(x1)
            ev.append((x1, f1))
        else:
            a = x1
            x1, f1 = x2, f2
            x2 = a + GOLDEN * (b - a)
            f2 = f(x2)
            ev.append((x2, f2))
    return a, b, ev


def fibonacci_search(f, lo: float, hi: float, n_eval: int):
    """Fibonacci search of f on [lo, hi] with n_eval >= 3 evaluations.

    With L = hi - lo and unit u = L / F_N (N = n_eval), bracket j (j = 1..N-2,
    lower end a_j) has its points at a_j + F_{N-j-1} u and a_j + F_{N-j} u;
    the retained point of one bracket is exactly one point of the next, so
    each elimination costs one evaluation.  Bracket N-1 is 2u wide and its two
    points would coincide (both u past its lower end); the last evaluation is
    made a tenth of u from the retained point instead (below it when it
    becomes the upper point, above it otherwise), and the final comparison
    leaves a bracket u or 1.1 u wide.  Returns (a, b, evaluations)."""
    N = int(n_eval)
    a, b = float(lo), float(hi)
    u = (b - a) / fibonacci(N)
    x1 = a + fibonacci(N - 2) * u
    x2 = a + fibonacci(N - 1) * u
    f1, f2 = f(x1), f(x2)
    ev = [(x1, f1), (x2, f2)]
    for j in range(1, N - 1):
        last = j == N - 2
        if f1 < f2:
            b = x2
            x2, f2 = x1, f1
            x1 = (x2 - 0.1 * u) if last else (a + fibonacci(N - j - 2) * u)
            f1 = f(x1)
            ev.append((x1, f1))
        else:
            a = x1
            x1, f1 = x2, f2
            x2 = (x1 + 0.1 * u) if last else (a + fibonacci(N - j - 1) * u)
            f2 = f(x2)
            ev.append((x2, f2))
    # the last comparison only shrinks the bracket
    if f1 < f2:
        b = x2
    else:
        a = x1
    return a, b, ev


def quadratic_minimizer(x, d, t0, c, beta: float) -> float:
    """Closed form for p = 1: phi is a quadratic in alpha,
    phi'(alpha) = sum t0 d (1 + beta v / c), zero at
    alpha* = -(sum t0 d + beta sum t0 x d / c) / (beta sum t0 d^2 / c)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    d = np.asarray(d, dtype=np.float32).astype(np.float64)
    t0 = np.asarray(t0, dtype=np.float32).astype(np.float64)
    c = np.asarray(c, dtype=np.float32).astype(np.float64)
    num = math.fsum((t0 * d).tolist()) + beta * math.fsum((t0 * x * d / c).tolist())
    den = beta * math.fsum((t0 * d * d / c).tolist())
    return -num / den
