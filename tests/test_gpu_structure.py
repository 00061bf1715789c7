"""Split products that leave out the exactly-zero parts of real operators' powers.

With real operators (H0 and b + b^dag drives in a real basis) every first-order Hbar_n is
real (Eq. magnus-first-order-term with real coefficients c_{k,n}), so the exponent
X_n = -i 2^-s (Hbar_n - tau_n I) is purely imaginary, X^2 and X^6 are real and X^3 is
imaginary.  The products of these powers (mg_ctx_set_structure, on by default) skip the
zero half of A's K axis and, where B has a zero part, multiply one B plane into one output
half.  The skipped digit products are exact zeros: every result must equal the full
product's, in every product configuration (one CTA or CTA pairs, stage depths, digit
layouts, digit counts), and meet the oracle within the stated 1e-6.
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


def _evolve(ctx, wl, structure, L=6, taylor=None, order=1):
    """One mg_evolve of the workload; returns (result, report, counted gemm flops)."""
    ctx.set_structure(structure)
    ctx.enable_gemm_timing(True)
    ctx.gemm_stats(reset=True)
    samples, w = M.node_samples(wl)
    p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, L)
    if order != 1:
        p.set_magnus_order(order)
    if taylor is not None:
        p.set_taylor(taylor)
    p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
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
    (6, 32, 0, True),     # CTA pairs for the full products (structured ones stay on one CTA)
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
        on, rep_on, f_on = _evolve(ctx, wl, True, L)
        off, rep_off, f_off = _evolve(ctx, wl, False, L)
    finally:
        _restore(ctx)
    assert np.array_equal(on, off), np.abs(on - off).max()
    # three of the degree-18 polynomial's products (X X, X^2 X, X^3 X^3) per interval take
    # 2 d^3 instead of 8 d^3 (degree 18 wherever the digits carry 30 bits or more)
    if L >= 5:
        assert f_on == pytest.approx(f_off - 18.0 * wl.d ** 3 * wl.N, rel=1e-12)
    else:
        assert f_on < f_off
    # the oracle bound from six digits (this job's ||Hbar_n||_1 ~ 1e3 takes ten squarings,
    # which five digits' 35 bits do not carry to 1e-6)
    if L >= 6:
        ref = oracle.evolve_workload(wl)
        err = np.abs(on - ref).max()
        assert err <= 1e-6, err


def test_state_workload_and_trace(ctx):
    """The d = 30 workload (state output) and the report agree with and without skipping."""
    wl = W.config(0, N=200)
    on, rep_on, f_on = _evolve(ctx, wl, True)
    off, rep_off, f_off = _evolve(ctx, wl, False)
    assert np.array_equal(on, off)
    assert rep_on["max_squarings"] == rep_off["max_squarings"]
    assert f_on < f_off
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6


def test_paterson_stockmeyer_powers(ctx):
    """The Paterson-Stockmeyer forms' powers X^j = X^{j-1} X skip too (MG_TAYLOR_PS)."""
    wl = W.transmon_resonator(nt=4, nr=36, N=10, T=5.0, sigma=2.0, omega0=0.2, unitary=True, name="tr144")
    on, _, f_on = _evolve(ctx, wl, True, taylor=M.MG_TAYLOR_PS)
    off, _, f_off = _evolve(ctx, wl, False, taylor=M.MG_TAYLOR_PS)
    assert np.array_equal(on, off)
    assert f_on < f_off
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6


def test_complex_operators_take_full_products(ctx):
    """An operator with a nonzero imaginary part (a Y-quadrature drive i(b^dag - b)) keeps
    every product in full: the counted work is the same either way."""
    base = W.transmon_resonator(nt=3, nr=40, N=8, T=4.0, sigma=1.5, omega0=0.2, unitary=True, name="tr120y")
    Hk = base.Hk.copy()
    # i (b - b^dag) has the same support as b + b^dag and is Hermitian with imaginary entries
    low = np.tril(Hk[0], -1)
    Hk[0] = 1j * (low - low.T)
    wl = W.Workload("tr120y", base.H0, Hk, base.drive, base.t0, base.T, base.N, base.P, None)
    on, _, f_on = _evolve(ctx, wl, True)
    off, _, f_off = _evolve(ctx, wl, False)
    assert f_on == f_off
    assert np.array_equal(on, off)
    ref = oracle.evolve_workload(wl)
    assert np.abs(on - ref).max() <= 1e-6


def test_second_order_term_takes_full_products(ctx):
    """The second-order term adds -(i/2)[H_j, H_k] (imaginary for real operators): full products."""
    wl = W.transmon_resonator(nt=3, nr=12, N=20, T=10.0, sigma=3.0, omega0=0.1, name="tr36")
    on, _, f_on = _evolve(ctx, wl, True, order=2)
    off, _, f_off = _evolve(ctx, wl, False, order=2)
    assert f_on == f_off
    assert np.array_equal(on, off)


def test_batch_of_real_plans(ctx):
    """mg_evolve_batch over uneven real jobs (one padded dimension per group) skips too, and
    each job equals its full-product result and the oracle."""
    rng = np.random.default_rng(41)
    jobs = [W.random_instance(rng, name=f"j{i}", N_range=(10, 30), d_range=(40, 200)) for i in range(5)]
    jobs[1].psi0 = None
    results = {}
    for structure in (True, False):
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
    ctx.set_structure(True)
    for wl, a, b in zip(jobs, results[True], results[False]):
        assert np.array_equal(a, b), wl.name
        ref = oracle.evolve_workload(wl)
        assert np.abs(a - ref).max() <= 1e-6, wl.name


def test_structure_option_rejects_other_values(ctx):
    for bad in (-1, 2):
        with pytest.raises(M.MagnusError) as e:
            M._check(M.load().mg_ctx_set_structure(ctx.h, bad), "mg_ctx_set_structure")
        assert e.value.code == M.MG_EINVAL
