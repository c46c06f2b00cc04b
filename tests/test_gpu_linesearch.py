"""Parity of the line search on the reduction (golden-section and Fibonacci
search of the Beckmann objective) with the oracle: every evaluation within
its error bound, the same sequence of points as the one-by-one search
whatever the speculation depth, the oracle's bracket wherever every
comparison is decided by more than the evaluation error, and convergence to
the minimiser otherwise."""
import math

import numpy as np
import pytest

from oracle import linesearch as ols
from paper_1710_07358_gb300 import pr, synth

pytestmark = pytest.mark.gpu

BETA = 0.15
B32 = float(np.float32(BETA))          # the kernel receives beta as float32; the oracle evaluates at it too
U = 2.0 ** -24


def eval_bound(arrs, p, a32):
    """Error bound of one evaluation, derived from the kernel's operations
    (u = 2^-24, first order, times 1.001 for the higher-order terms):
      linear part t0 v:   v = fma(alpha, d, x), fma(B, v^4, t0) or t0 * v,
                          the last product or fma: 3 u
      power part:         power 4 (B = t0 (beta / 5) rcp(c)^4 with an
                          approximate reciprocal within 2 u, v^4 by two
                          squarings, fma, product): 24 u; other powers (a
                          correctly rounded rcp(c), q = v rcp(c), p products,
                          t0 kb c, fma): 4 p + 7 u
      summation:          eight terms pairwise (3 u), Kahan (2 u), float64
                          combines (below 2^-45): 5 u of sum |term|
    so |phi_gpu - phi| <= u (8 sum |t0 v| + (c_p + 5) sum |power part|)."""
    lin, pw = ols.phi_parts(*arrs, B32, p, a32)
    cp = 24 if p == 4 else 4 * p + 7
    # numpy's pairwise float64 sums of non-negative values err by far less
    # than the 2^-40 added here, so the bound stays an upper bound
    up = 1.0 + 2.0 ** -40
    return 1.001 * U * (8 * float(np.abs(lin).sum()) + (cp + 5) * float(np.abs(pw).sum())) * up + 1e-300


def dev(arrs, offset=0):
    """CUDA float32 copies, `offset` elements past a 16-byte boundary."""
    import torch
    out = []
    for a in arrs:
        buf = torch.zeros(a.size + offset, dtype=torch.float32, device="cuda")
        buf[offset:] = torch.from_numpy(a).cuda()
        out.append(buf[offset:])
    return out


@pytest.mark.parametrize("n", [0, 1, 3, 7, 1000, 100003, (1 << 20) + 5])
@pytest.mark.parametrize("p", [1, 4, 6])
def test_evaluation_within_bound(n, p):
    arrs = synth.network_links(n, 10 + n % 97)
    alphas = np.array([0.0, 0.125, 0.3, 0.5, 0.77, 1.0, 2.5], dtype=np.float64)
    import torch
    from gpu_helpers import Guarded
    g = Guarded(alphas.size, torch.float64)
    got = pr.beckmann(*dev(arrs), alphas, BETA, p, out=g.tensor)
    got = g.check().cpu().numpy()
    for k, al in enumerate(alphas):
        a32 = float(np.float32(al))                       # the kernel evaluates at float32(alpha)
        want = ols.phi(*arrs, B32, p, a32)
        bound = eval_bound(arrs, p, a32)
        assert abs(got[k] - want) <= bound, (n, p, al, got[k], want, bound)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_evaluation_unaligned_and_sixteen_points(offset):
    arrs = synth.network_links(50021, 20 + offset)
    alphas = np.linspace(0.0, 1.0, 16)
    got = pr.beckmann(*dev(arrs, offset), alphas, BETA, 4).cpu().numpy()
    aligned = pr.beckmann(*dev(arrs), alphas, BETA, 4).cpu().numpy()
    for k, al in enumerate(alphas):
        want = ols.phi(*arrs, B32, 4, float(np.float32(al)))
        bound = eval_bound(arrs, 4, float(np.float32(al)))
        assert abs(got[k] - want) <= bound and abs(aligned[k] - want) <= bound


def test_evaluation_at_the_benchmark_size():
    n = 1 << 24
    arrs = synth.network_links(n, synth.config_seed(7))
    alphas = np.array([0.25, 0.6], dtype=np.float64)
    got = pr.beckmann(*dev(arrs), alphas, BETA, 4).cpu().numpy()
    for k, al in enumerate(alphas):
        want = ols.phi(*arrs, B32, 4, float(np.float32(al)))
        assert abs(got[k] - want) <= eval_bound(arrs, 4, float(np.float32(al)))


def gpu_search(arrs, p, lo, hi, method, count, depth, offset=0):
    r = pr.line_search(*dev(arrs, offset), lo=lo, hi=hi, beta=BETA, power=p, method=method, count=count,
                       depth=depth)
    return r.cpu().numpy()


def oracle_search(arrs, p, lo, hi, method, count):
    f = lambda al: ols.phi(*arrs, B32, p, float(np.float32(al)))
    if method == "golden":
        return ols.golden_section(f, lo, hi, count)
    return ols.fibonacci_search(f, lo, hi, count)


def min_margin(ev, arrs, p, method):
    """Smallest |f1 - f2| / (bound(x1) + bound(x2)) over the comparisons the
    search made (replayed from its evaluation list; Fibonacci also compares
    the last two points to shrink its final bracket).  Above 1, every
    comparison the kernel makes goes the oracle's way."""
    bd = {x: eval_bound(arrs, p, float(np.float32(x))) for x, _ in ev}
    worst = math.inf
    (x1, f1), (x2, f2) = ev[0], ev[1]
    for xn, fn in ev[2:]:
        worst = min(worst, abs(f1 - f2) / (bd[x1] + bd[x2]))
        if f1 < f2:
            x2, f2 = x1, f1
            x1, f1 = xn, fn
        else:
            x1, f1 = x2, f2
            x2, f2 = xn, fn
    if method == "fibonacci":
        worst = min(worst, abs(f1 - f2) / (bd[x1] + bd[x2]))
    return worst


def assert_same_search(arrs, p, hi, method, count, depths=(1, 2, 3)):
    a, b, ev = oracle_search(arrs, p, 0.0, hi, method, count)
    # every comparison is decided by more than the two evaluations' error
    # bounds: the kernel must take the same branches, place the same float64
    # points and end with the same bracket, bit for bit
    assert min_margin(ev, arrs, p, method) > 1.0
    for depth in depths:
        got = gpu_search(arrs, p, 0.0, hi, method, count, depth)
        assert got[0] == a and got[1] == b, (depth, got[:2], (a, b))
        assert got[2] in [x for x, _ in ev] and a <= got[2] <= b
        a32 = float(np.float32(got[2]))
        assert abs(got[3] - ols.phi(*arrs, B32, p, a32)) <= eval_bound(arrs, p, a32)


@pytest.mark.parametrize("method,count", [("golden", 10), ("golden", 0), ("golden", 1), ("fibonacci", 3),
                                          ("fibonacci", 10)])
@pytest.mark.parametrize("p,hi", [(1, 4.0), (4, 1.0)])
def test_search_matches_oracle_exactly(method, count, p, hi):
    assert_same_search(synth.network_links(30011, 31 + p), p, hi, method, count)


@pytest.mark.slow
def test_search_at_the_benchmark_size_matches_oracle_exactly():
    """2^24 links (256 MiB per pass, more than L2 holds), power 4: ten
    golden-section iterations, bracket for bracket with the oracle at every
    depth."""
    assert_same_search(synth.network_links(1 << 24, synth.config_seed(7)), 4, 1.0, "golden", 10)


@pytest.mark.parametrize("method,count", [("golden", 40), ("fibonacci", 40)])
@pytest.mark.parametrize("p", [1, 4])
def test_search_converges_to_the_minimiser(method, count, p):
    arrs = synth.network_links(20011, 41 + p)
    hi = 4.0 if p == 1 else 1.0
    got = gpu_search(arrs, p, 0.0, hi, method, count, 2)
    a, b = got[0], got[1]
    if p == 1:
        star = ols.quadratic_minimizer(*arrs, B32)
    else:
        f = lambda al: ols.phi(*arrs, B32, p, al)
        oa, ob, _ = ols.golden_section(f, 0.0, hi, 60)
        star = (oa + ob) / 2
    # where phi is flat to within the evaluation error, any point is as good:
    # |phi(s + w) - phi(s)| ~ phi''(s) w^2 / 2 = eps sum|terms|
    h = 1e-3
    f2 = (ols.phi(*arrs, B32, p, star + h) - 2 * ols.phi(*arrs, B32, p, star) + ols.phi(*arrs, B32, p, star - h)) / h**2
    eps = eval_bound(arrs, p, star)
    flat = math.sqrt(2 * eps / f2)
    assert a - flat - 1e-9 <= star <= b + flat + 1e-9, (a, b, star, flat)
    # the textbook width, plus the rounding of float64 positions near |alpha| <= hi
    width = hi * ols.GOLDEN ** count if method == "golden" else 1.1 * hi / ols.fibonacci(count)
    assert b - a <= width + 64 * hi * 2.0 ** -52


def test_depth_and_alignment_do_not_change_the_search():
    arrs = synth.network_links(70001, 51)
    ref = gpu_search(arrs, 4, 0.0, 1.0, "golden", 35, 1)
    for depth in (2, 3):
        assert np.array_equal(gpu_search(arrs, 4, 0.0, 1.0, "golden", 35, depth), ref)
    # unaligned arrays take the scalar loads: a different float32 evaluation
    # order per thread, so only the bracket's convergence is compared
    un = gpu_search(arrs, 4, 0.0, 1.0, "golden", 35, 2, offset=1)
    assert abs((un[0] + un[1]) - (ref[0] + ref[1])) / 2 <= 1e-3


def test_monotone_objective_ends_at_the_lower_end():
    x, d, t0, c = synth.network_links(10007, 61)
    d = np.abs(d)                                     # every link only gains flow: phi increases
    got = gpu_search((x, d, t0, c), 4, 0.0, 1.0, "golden", 30, 2)
    assert got[0] == 0.0 and got[1] <= ols.GOLDEN ** 30 * (1 + 1e-9)


def test_no_links_and_graph_replay():
    import torch
    e = [np.zeros(0, dtype=np.float32)] * 4
    got = gpu_search(e, 4, 0.0, 1.0, "golden", 5, 2)       # phi = 0: every comparison a tie
    a, b, _ = ols.golden_section(lambda al: 0.0, 0.0, 1.0, 5)
    assert got[0] == a and got[1] == b and got[3] == 0.0
    arrs = dev(synth.network_links(40009, 71))
    s = torch.cuda.Stream()
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        pr.line_search(*arrs, method="fibonacci", count=20, depth=3, result=res, stream=s)
    s.synchronize()
    want = res.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pr.line_search(*arrs, method="fibonacci", count=20, depth=3, result=res, stream=s)
    for _ in range(3):
        res.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(res, want)
    assert pr.last_device_error() == 0
