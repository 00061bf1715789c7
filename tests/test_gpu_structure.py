"""Split products that use the structure of real operators (mg_ctx_set_structure).

With real operators (H0 and b + b^dag drives in a real basis) every first-order Hbar_n is
real (Eq. magnus-first-order-term with real coefficients c_{k,n}), so the exponent
X_n = -i 2^-s (Hbar_n - tau_n I) is purely imaginary, X^2 and X^6 are real and X^3 is
imaginary (bit 0: the products of these powers skip the zero half of A's K axis and, where
B has a zero part, multiply one B plane into one output half), and with real symmetric
operators every polynomial in X is complex symmetric (bit 1: the products of the
exponential compute the tiles on and below the diagonal and mirror the rest).  The digit
products bit 0 skips are exact zeros: those results must equal the full products' in every
product configuration (one CTA or CTA pairs, stage depths, digit layouts, digit counts).
With bit 1 every U_n is exactly symmetric and every result meets the oracle within the
stated 1e-6.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.fixture(scope="module")
def ctx():
    M.load()
    c = M.Context(0)
    yield c
    c.close()


def _evolve(ctx, wl, structure, L=6, taylor=None, order=1, N=None):
    """One mg_evolve of the workload; returns (result, report, counted gemm flops)."""
    ctx.set_structure(structure)
    ctx.enable_gemm_timing(True)
    ctx.gemm_stats(reset=True)
    N = wl.N if N is None else N
    samples, w = M.node_samples(wl, N)
    p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, L)
    if order != 1:
        p.set_magnus_order(order)
    if taylor is not None:
        p.set_taylor(taylor)
    p.set_controls(N, wl.P, wl.t0, wl.dt, w, cuda(samples))
    if wl.psi0 is None:
        out = torch.empty((wl.d, wl.d), dtype=torch.complex128, device="cuda")
        rep = p.evolve(M.MG_OUT_PROPAGATOR, None, out)
    else:
        out = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
        rep = p.evolve(M.MG_OUT_STATE, cuda(wl.psi0), out)
    torch.cuda.synchronize()
    flops = ctx.gemm_stats(reset=True)["flops"]
    ctx.enable_gemm_timing(False)
    ctx.set_structure(True)
    p.close()
    return out.cpu().numpy(), rep, flops


def _restore(ctx):
    ctx.set_stage_k(32)
    ctx.set_digit_pairs(0)
    ctx.set_cta_pairs(None)


# d = 300: three row tiles of 128 (the last ragged), five column tiles of 64 (ragged),
# each half of K 320 deep (a whole number of 64-deep stages)
_D300 = dict(nt=6, nr=50, N=12, T=6.0, sigma=2.0, omega0=0.2, unitary=True, name="tr300")


@pytest.mark.parametrize("L,stage_k,digit_pairs,cta_pairs", [
    (6, 32, 0, None),     # the default: one CTA per tile at three row tiles
    (6, 32, 0, True),     # CTA pairs: the power products in the pairs' real mode
    (6, 16, 0, True),
    (6, 32, 2, True),     # paired digit layout on CTA pairs
    (6, 16, 0, False),
    (6, 32, 1, False),    # paired digit layout, 16-deep stages
    (6, 32, 2, False),    # paired digit layout, 32-deep stages of 128-byte rows
    (5, 32, 0, None),
    (3, 64, 0, False),    # 64-deep stages (128-byte rows)
    (8, 32, 0, False),    # eight digits take 16-deep stages
])
def test_structured_products_equal_full_products(ctx, L, stage_k, digit_pairs, cta_pairs):
    wl = W.transmon_resonator(**_D300)
    ctx.set_stage_k(stage_k)
    ctx.set_digit_pairs(digit_pairs)
    ctx.set_cta_pairs(cta_pairs)
    try:
        on, rep_on, f_on = _evolve(ctx, wl, 1, L)
        off, rep_off, f_off = _evolve(ctx, wl, 0, L)
        sym, rep_sym, f_sym = _evolve(ctx, wl, 3, L)
        sym2, _, _ = _evolve(ctx, wl, 2, L)
    finally:
        _restore(ctx)
    assert np.array_equal(on, off), np.abs(on - off).max()
    # zero-part skipping is exact on symmetric products too, where the operands' zero
    # halves and planes are not even written
    assert np.array_equal(sym, sym2), np.abs(sym - sym2).max()
    # three of the degree-18 polynomial's products (X X, X^2 X, X^3 X^3) per interval take
    # 2 d^3 instead of 8 d^3 (degree 18 wherever the digits carry 30 bits or more)
    if L >= 5:
        assert f_on == pytest.approx(f_off - 18.0 * wl.d ** 3 * wl.N, rel=1e-12)
    else:
        assert f_on < f_off
    assert f_sym < f_on
    # the oracle bound from six digits (this job's ||Hbar_n||_1 ~ 1e3 takes ten squarings,
    # which five digits' 35 bits do not carry to 1e-6)
    if L >= 6:
        ref = oracle.evolve_workload(wl)
        for got in (on, sym):
            err = np.abs(got - ref).max()
            assert err <= 1e-6, err


@pytest.mark.parametrize("nt,nr,N", [(8, 64, 6), (8, 100, 3)])
def test_default_pairs_real_mode(ctx, nt, nr, N):
    """d = 512 (four row tiles) and d = 800 (seven): CTA pairs by default, the power
    products in the real mode (128-column tiles of one output half), ragged edges."""
    wl = W.transmon_resonator(nt=nt, nr=nr, N=N, T=0.5 * N, sigma=0.5, omega0=0.2, unitary=True, name="trpairs")
    on, _, f_on = _evolve(ctx, wl, 1)
    off, _, f_off = _evolve(ctx, wl, 0)
    sym, _, f_sym = _evolve(ctx, wl, 3)
    sym2, _, _ = _evolve(ctx, wl, 2)
    assert np.array_equal(on, off), np.abs(on - off).max()
    assert np.array_equal(sym, sym2), np.abs(sym - sym2).max()
    assert f_sym < f_on < f_off
    ref = oracle.evolve_workload(wl)
    for got in (on, sym):
        assert np.abs(got - ref).max() <= 1e-6, np.abs(got - ref).max()


_SYM_BY_TILING = {}


@pytest.mark.parametrize("cta_pairs", [False, True])
def test_symmetric_products_give_exactly_symmetric_exponentials(ctx, cta_pairs):
    """One interval: U_0 = exp(-i Hbar_0) is complex symmetric; with bit 1 every product of
    its exponential copies the entries above the diagonal from below it, so U_0 = U_0^T
    exactly, the same on single CTAs and CTA pairs, and it differs from the full
    products' U_0 by their rounding only."""
    wl = W.transmon_resonator(**_D300)
    ctx.set_cta_pairs(cta_pairs)
    try:
        sym, _, f_sym = _evolve(ctx, wl, 3, N=1)
        full, _, f_full = _evolve(ctx, wl, 0, N=1)
    finally:
        _restore(ctx)
    assert np.array_equal(sym, sym.T)
    _SYM_BY_TILING[cta_pairs] = sym
    if len(_SYM_BY_TILING) == 2:
        assert np.array_equal(_SYM_BY_TILING[False], _SYM_BY_TILING[True])
    assert np.abs(sym - full).max() <= 1e-9, np.abs(sym - full).max()
    assert f_sym < 0.6 * f_full
    ref = oracle.evolve_workload(wl, n_intervals=1)
    assert np.abs(sym - ref).max() <= 1e-8


def test_state_workload_and_trace(ctx):
    """The d = 30 workload (state output) and the report agree with and without skipping."""
    wl = W.config(0, N=200)
    on, rep_on, f_on = _evolve(ctx, wl, 1)
    off, rep_off, f_off = _evolve(ctx, wl, 0)
    sym, rep_sym, f_sym = _evolve(ctx, wl, 3)
    assert np.array_equal(on, off)
    assert rep_on["max_squarings"] == rep_off["max_squarings"] == rep_sym["max_squarings"]
    assert f_sym < f_on < f_off
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6
    assert np.abs(sym - ref).max() <= 1e-6


def test_paterson_stockmeyer_powers(ctx):
    """The Paterson-Stockmeyer forms' powers X^j = X^{j-1} X skip too (MG_TAYLOR_PS)."""
    wl = W.transmon_resonator(nt=4, nr=36, N=10, T=5.0, sigma=2.0, omega0=0.2, unitary=True, name="tr144")
    on, _, f_on = _evolve(ctx, wl, 1, taylor=M.MG_TAYLOR_PS)
    off, _, f_off = _evolve(ctx, wl, 0, taylor=M.MG_TAYLOR_PS)
    sym, _, f_sym = _evolve(ctx, wl, 3, taylor=M.MG_TAYLOR_PS)
    assert np.array_equal(on, off)
    assert f_sym < f_on < f_off
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6
    assert np.abs(sym - ref).max() <= 1e-6


def test_complex_operators_take_full_products(ctx):
    """An operator with a nonzero imaginary part (a Y-quadrature drive i(b^dag - b)) keeps
    every product in full: the counted work is the same either way."""
    base = W.transmon_resonator(nt=3, nr=40, N=8, T=4.0, sigma=1.5, omega0=0.2, unitary=True, name="tr120y")
    Hk = base.Hk.copy()
    # i (b - b^dag) has the same support as b + b^dag and is Hermitian with imaginary entries
    low = np.tril(Hk[0], -1)
    Hk[0] = 1j * (low - low.T)
    wl = W.Workload("tr120y", base.H0, Hk, base.drive, base.t0, base.T, base.N, base.P, None)
    on, _, f_on = _evolve(ctx, wl, 3)
    off, _, f_off = _evolve(ctx, wl, 0)
    assert f_on == f_off
    assert np.array_equal(on, off)
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6


def test_second_order_term_takes_full_products(ctx):
    """The second-order term adds -(i/2)[H_j, H_k] (imaginary for real operators): full products."""
    wl = W.transmon_resonator(nt=3, nr=12, N=20, T=10.0, sigma=3.0, omega0=0.1, name="tr36")
    on, _, f_on = _evolve(ctx, wl, 3, order=2)
    off, _, f_off = _evolve(ctx, wl, 0, order=2)
    assert f_on == f_off
    assert np.array_equal(on, off)


def test_batch_of_real_plans(ctx):
    """mg_evolve_batch over uneven real jobs (one padded dimension per group) skips too, and
    each job equals its full-product result and the oracle."""
    rng = np.random.default_rng(41)
    jobs = [W.random_instance(rng, name=f"j{i}", N_range=(10, 30), d_range=(40, 200)) for i in range(5)]
    jobs[1].psi0 = None
    results = {}
    for structure in (1, 0, 3):
        ctx.set_structure(structure)
        plans, outs, ins, kinds = [], [], [], []
        for wl in jobs:
            samples, w = M.node_samples(wl)
            p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, 6)
            p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
            plans.append(p)
            if wl.psi0 is None:
                kinds.append(M.MG_OUT_PROPAGATOR)
                ins.append(None)
                outs.append(torch.empty((wl.d, wl.d), dtype=torch.complex128, device="cuda"))
            else:
                kinds.append(M.MG_OUT_STATE)
                ins.append(cuda(wl.psi0))
                outs.append(torch.empty(wl.d, dtype=torch.complex128, device="cuda"))
        status = M.mg_evolve_batch(ctx, plans, kinds, ins, outs)
        torch.cuda.synchronize()
        assert list(status) == [0] * len(jobs)
        results[structure] = [o.cpu().numpy() for o in outs]
        for p in plans:
            p.close()
    ctx.set_structure(3)
    for wl, a, b, c in zip(jobs, results[1], results[0], results[3]):
        assert np.array_equal(a, b), wl.name
        ref = oracle.evolve_workload(wl)
        assert np.abs(a - ref).max() <= 1e-6, wl.name
        assert np.abs(c - ref).max() <= 1e-6, wl.name


def test_structure_option_rejects_other_values(ctx):
    for bad in (-1, 4):
        with pytest.raises(M.MagnusError) as e:
            M._check(M.load().mg_ctx_set_structure(ctx.h, bad), "mg_ctx_set_structure")
        assert e.value.code == M.MG_EINVAL
