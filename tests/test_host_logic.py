"""Host-side arithmetic of the library that needs no device: the Gauss-Legendre
rule behind the drive samples, and the choice of Taylor degree and squaring
count for U_n = exp(-i Hbar_n).  CPU only; the library is built and loaded, but
no context is created."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2411_09982_gb300 import magnus as M

DEGREES = {2: 1, 4: 2, 6: 3, 9: 4, 12: 5, 16: 6, 18: 5}   # degree -> matrix products


def split_beta(d):
    """Digit width of the split product: largest beta <= 8 with 2^(2 beta - 1) 2d <= 2^24."""
    return max(b for b in range(2, 9) if 2.0 ** (2 * b - 1) * 2 * d <= 2.0 ** 24)


def unit_roundoff(prec, L, d):
    return 2.0 ** -53 if prec == M.MG_PREC_FP64 else max(2.0 ** -53, 2.0 ** (-split_beta(d) * L))


def tail_over_theta_exact(m, theta):
    """sum_{j>m} theta^j / j! divided by theta, in rational arithmetic (80 terms: the
    rest is below 1e-60 of the sum for theta <= 40)."""
    t = Fraction(theta)
    term = Fraction(1)
    for j in range(1, m + 1):
        term = term * t / j
    s = Fraction(0)
    for j in range(m + 1, m + 81):
        term = term * t / j
        s += term
    return s / t


def theta_by_bisection(m, u):
    """Largest theta with tail/theta <= u, by bisection on a log-space float evaluation."""
    def ratio(th):
        return math.fsum(math.exp(j * math.log(th) - math.lgamma(j + 1)) for j in range(m + 1, m + 81)) / th
    lo, hi = 1e-6, 40.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ratio(mid) <= u else (lo, mid)
    return lo


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8, 16, 33, 64])
def test_quadrature_rule_is_gauss_legendre_on_host(P):
    """The rule integrates x^k exactly on [-1, 1] for k <= 2P - 1 (the defining property,
    up to rounding of the sum), and agrees with numpy's leggauss within the error of the
    latter (2.3e-15 in the weights at P = 64, against 40-digit Newton nodes)."""
    x, w = M.mg_quadrature_nodes(P)
    assert np.all(np.diff(x) > 0) and np.all(w > 0)
    for k in range(2 * P):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(math.fsum(w * x ** k) - exact) <= 4e-15, (k, math.fsum(w * x ** k), exact)
    xr, wr = np.polynomial.legendre.leggauss(P)
    np.testing.assert_allclose(x, xr, atol=4e-15, rtol=0)
    np.testing.assert_allclose(w, wr, atol=4e-15, rtol=0)


@pytest.mark.parametrize("prec,L,d", [(M.MG_PREC_FP64, 6, 30), (M.MG_PREC_SPLIT, 6, 729), (M.MG_PREC_SPLIT, 4, 64),
                                      (M.MG_PREC_SPLIT, 8, 4096), (M.MG_PREC_SPLIT, 2, 30)])
def test_taylor_theta_is_the_largest_within_the_remainder_bound(prec, L, d):
    """theta_m: the truncated series errs by at most u relative at 1-norm theta (exact
    rational check), and by more than u just above it."""
    u = unit_roundoff(prec, L, d)
    seen = set()
    for norm in [1e-3, 0.3, 1.0, 2.5, 6.0, 40.0, 1e3]:
        m, s, th = M.mg_taylor_choice(norm, prec, L, d)
        if m in seen:
            continue
        seen.add(m)
        assert tail_over_theta_exact(m, th) <= Fraction(u) * (1 + Fraction(1, 10 ** 12)), (m, th)
        above = th * (1 + 1e-9)
        assert tail_over_theta_exact(m, above) > Fraction(u), (m, th)
        assert th == pytest.approx(theta_by_bisection(m, u), rel=1e-10)


@pytest.mark.parametrize("prec,L,d", [(M.MG_PREC_FP64, 6, 30), (M.MG_PREC_SPLIT, 6, 729), (M.MG_PREC_SPLIT, 4, 100)])
def test_taylor_choice_minimises_products(prec, L, d):
    """(m, s) minimises products(m) + s over the offered degrees (18 on the split path
    only), ties to fewer squarings, and s is the least with norm1 / 2^s <= theta_m."""
    u = unit_roundoff(prec, L, d)
    offered = {m: c for m, c in DEGREES.items() if m != 18 or prec == M.MG_PREC_SPLIT}
    thetas = {m: theta_by_bisection(m, u) for m in offered}
    rng = np.random.default_rng(11)
    norms = [0.0, 1e-12, 1e-4] + list(10.0 ** rng.uniform(-3, 5, 300))
    for norm in norms:
        # skip norms within 1e-8 of a switching point, where float rounding of theta decides
        if any(abs(norm / (t * 2.0 ** k) - 1) < 1e-8 for t in thetas.values() for k in range(0, 40)):
            continue
        m, s, th = M.mg_taylor_choice(norm, prec, L, d)
        assert m in offered, m
        assert norm * 2.0 ** -s <= th and (s == 0 or norm * 2.0 ** -(s - 1) > th), (norm, m, s, th)

        def least_s(t):
            k = 0
            while norm * 2.0 ** -k > t:
                k += 1
            return k
        costs = {mm: offered[mm] + least_s(t) for mm, t in thetas.items()}
        best = min(costs.values())
        assert costs[m] == best, (norm, m, s, costs)
        assert s == min(least_s(thetas[mm]) for mm in offered if costs[mm] == best), (norm, m, s, costs)


def test_taylor_choice_small_norms_take_low_degrees_and_no_squaring():
    assert M.mg_taylor_choice(0.0, M.MG_PREC_FP64, 6, 30)[:2] == (2, 0)
    m, s, _ = M.mg_taylor_choice(1e-9, M.MG_PREC_FP64, 6, 30)
    assert s == 0 and m <= 4
    # a coarser unit roundoff never needs a higher degree or more squarings at the same norm
    for norm in [0.5, 3.0, 50.0]:
        m64, s64, _ = M.mg_taylor_choice(norm, M.MG_PREC_FP64, 6, 30)
        for L in (2, 4, 6):
            m_l, s_l, _ = M.mg_taylor_choice(norm, M.MG_PREC_SPLIT, L, 729)
            assert DEGREES[m_l] + s_l <= DEGREES[m64] + s64


@pytest.mark.parametrize("args", [(-1.0, 0, 6, 30), (float("nan"), 0, 6, 30), (float("inf"), 0, 6, 30),
                                  (1.0, 1, 1, 30), (1.0, 1, 9, 30), (1.0, 2, 6, 30), (1.0, 0, 6, 0),
                                  (1.0, 0, 6, 4097)])
def test_taylor_choice_rejects_invalid_arguments(args):
    with pytest.raises(M.MagnusError):
        M.mg_taylor_choice(*args)


def test_node_samples_follow_the_header_node_map():
    """The binding's drive samples sit at t0 + n dt + (1 + x_p) dt / 2 (the node map the
    header documents), N x P x K contiguous; with them, (dt/2) sum_p w_p u(t_{n,p})
    integrates a polynomial drive of degree <= 2P - 1 exactly over every interval."""
    import oracle
    import workloads as W
    wl = W.config(0, N=12)
    samples, w = M.node_samples(wl)
    assert samples.shape == (wl.N, wl.P, wl.K) and samples.flags["C_CONTIGUOUS"]
    x, _ = M.mg_quadrature_nodes(wl.P)
    np.testing.assert_allclose(samples, wl.drive(oracle.node_times(wl.t0, wl.dt, wl.N, x)), rtol=0, atol=1e-15)
    # a cubic drive u(t) = t^3: the integral over [t_n, t_n + dt] is exact
    wl3 = W.Workload("cubic", wl.H0, wl.Hk, lambda t: (t ** 3)[..., None], 0.5, 0.25, 6, wl.P, None)
    s3, w3 = M.node_samples(wl3)
    c = 0.5 * wl3.dt * (s3[..., 0] * w3[None, :]).sum(axis=1)
    tn = wl3.t0 + wl3.dt * np.arange(wl3.N)
    np.testing.assert_allclose(c, ((tn + wl3.dt) ** 4 - tn ** 4) / 4, rtol=1e-14, atol=0)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8, 16])
def test_second_order_weights_satisfy_their_exact_identities(P):
    """M[p][q] = int_0^1 l_p(s1) int_0^{s1} l_q(s2): its row sums are int_0^1 l_p(s) s ds =
    (w_p/2) s_p, its column sums int_0^1 l_q(s)(1 - s) ds = (w_q/2)(1 - s_q), and
    M[p][q] + M[q][p] is the full square's integral (w_p/2)(w_q/2) (Gauss-Legendre is
    exact for these degrees); the stored sums equal the matrix's."""
    Mw, C, R = M.mg_second_order_weights(P)
    x, w = np.polynomial.legendre.leggauss(P)
    s, h = 0.5 * (1.0 + x), 0.5 * w
    np.testing.assert_allclose(Mw.sum(axis=1), h * s, atol=1e-14, rtol=0)
    np.testing.assert_allclose(Mw.sum(axis=0), h * (1.0 - s), atol=1e-14, rtol=0)
    np.testing.assert_allclose(Mw + Mw.T, np.outer(h, h), atol=1e-14, rtol=0)
    np.testing.assert_allclose(R, Mw.sum(axis=1), atol=1e-15, rtol=0)
    np.testing.assert_allclose(C, Mw.sum(axis=0), atol=1e-15, rtol=0)


@pytest.mark.parametrize("P", [2, 3, 5])
def test_second_order_weights_by_exact_integration(P):
    """Small P: each entry by exact rational integration of the Lagrange polynomials on
    the same (double) nodes, to the rounding of the result."""
    Mw, _, _ = M.mg_second_order_weights(P)
    s = [Fraction(v) for v in 0.5 * (1.0 + np.polynomial.legendre.leggauss(P)[0])]

    def mul(a, b):
        out = [Fraction(0)] * (len(a) + len(b) - 1)
        for i, u in enumerate(a):
            for j, v in enumerate(b):
                out[i + j] += u * v
        return out

    def integ(a):   # antiderivative vanishing at 0
        return [Fraction(0)] + [c / (k + 1) for k, c in enumerate(a)]

    ell = []
    for p in range(P):
        poly = [Fraction(1)]
        for r in range(P):
            if r != p:
                poly = mul(poly, [-s[r] / (s[p] - s[r]), 1 / (s[p] - s[r])])
        ell.append(poly)
    for p in range(P):
        for q in range(P):
            val = float(sum(integ(mul(ell[p], integ(ell[q])))))   # evaluated at s1 = 1
            assert abs(Mw[p, q] - val) <= 4e-16, (p, q, Mw[p, q], val)


@pytest.mark.parametrize("d,nops,density", [(1, 1, 1.0), (7, 3, 0.2), (40, 5, 0.05), (33, 2, 0.0)])
def test_csr_pattern_is_the_union_with_the_diagonal(d, nops, density):
    """The action path's CSR form: the pattern is exactly the union of the operators'
    nonzeros plus the diagonal, columns ascending per row, diag pointing at (i, i), and
    every operator's values scattered back on the pattern reproduce it exactly."""
    rng = np.random.default_rng(d * 10 + nops)
    ops = (rng.normal(size=(nops, d, d)) + 1j * rng.normal(size=(nops, d, d))) * (rng.uniform(size=(nops, d, d)) < density)
    ops[0, 0, d - 1] = 0.5j   # an entry with a zero real part still counts
    rowptr, col, diag, val = M.mg_csr_pattern(ops)
    want = (ops != 0).any(axis=0) | np.eye(d, dtype=bool)
    got = np.zeros((d, d), bool)
    for i in range(d):
        cols = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        got[i, cols] = True
        assert col[diag[i]] == i and rowptr[i] <= diag[i] < rowptr[i + 1]
    assert np.array_equal(got, want) and rowptr[-1] == want.sum()
    for k in range(nops):
        dense = np.zeros((d, d), complex)
        for i in range(d):
            dense[i, col[rowptr[i]:rowptr[i + 1]]] = val[k, rowptr[i]:rowptr[i + 1]]
        assert np.array_equal(dense, ops[k])


def test_split_digits_follow_the_exactness_bound():
    """beta is the largest digit width with 2^(2 beta - 1) 2d <= 2^24 (the two leading
    accumulator levels stay exact over K = 2d terms), checked by brute force; the digit
    count is the smallest carrying the requested bits, clamped to 2..8."""
    for d in (1, 2, 16, 30, 64, 255, 256, 729, 1024, 1025, 2048, 4096):
        beta, L = M.mg_split_digits(d, 42)
        ok = [b for b in range(2, 9) if 2.0 ** (2 * b - 1) * 2 * d <= 2.0 ** 24]
        assert beta == max(ok)
        assert L == min(8, max(2, -(-42 // beta)))
    assert M.mg_split_digits(729)[0] == 7 and M.mg_split_digits(729)[1] == 6
    assert M.mg_split_digits(1025) == (6, 7) and M.mg_split_digits(4096) == (6, 7)
    for bad in ((0, 42), (4097, 42), (64, 0), (64, 65)):
        with pytest.raises(M.MagnusError):
            M.mg_split_digits(*bad)
