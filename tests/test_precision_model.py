"""The NumPy model of the split-precision arithmetic (tests/precision_model.py),
checked against the mathematics it restates, and its predictions for the
tolerance question: which digit counts keep whole evolutions within 1e-6 of the
FP64 oracle.  CPU only."""
import numpy as np
import pytest

import oracle
import precision_model as PM
import workloads as W


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("d,L", [(7, 3), (30, 6), (129, 5)])
def test_digits_reconstruct_the_fixed_point_value(d, L):
    """2^(E+1-beta) sum_s q_s 2^(-beta s) is the entry rounded to the grid 2^(E+1-beta L)
    (error at most half a grid step); every digit is in the balanced range and exact in BF16."""
    rng = np.random.default_rng(d)
    A = rand_c(rng, (d, d)) * np.exp2(rng.integers(-20, 20, d))[:, None]
    beta = PM.split_beta(d)
    for axis, scale_axis in ((1, -1), (0, -2)):
        vr, vi, E = PM.digits(A, L, beta, axis)
        Eb = np.expand_dims(E, scale_axis)
        for v, part in ((vr, A.real), (vi, A.imag)):
            q = v * np.exp2(beta * np.arange(L))[:, None, None]
            assert np.array_equal(q, np.round(q)) and np.abs(q).max() <= 2 ** (beta - 1)
            assert np.all(np.abs(part) < np.exp2(Eb))
            rec = np.exp2(Eb + 1 - beta) * v.sum(axis=0)
            assert np.all(np.abs(rec - part) <= np.exp2(Eb - beta * L))
            bits = v.astype(np.float32).view(np.uint32)
            assert np.all(v.astype(np.float32) == v) and np.all(bits & 0xFFFF == 0)


def test_product_of_small_integers_is_exact():
    """Entries that fit in one digit and sums that fit the level-0 accumulator: exact."""
    rng = np.random.default_rng(2)
    d = 40
    A = rng.integers(-8, 9, (2, d, d)) + 1j * rng.integers(-8, 9, (2, d, d))
    B = rng.integers(-8, 9, (2, d, d)) + 1j * rng.integers(-8, 9, (2, d, d))
    for L in (2, 4):
        C = PM.df_value(PM.split_product(A, B, L))
        assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("d", [64, 129])
@pytest.mark.parametrize("accumulate", ["nearest", "zero"])
def test_product_within_the_digit_bound(d, accumulate):
    """The digit truncation plus FP32 rounding of the level->=3 accumulator stays within the
    bound the GPU tests use, for every L, and falls with L until the FP32 floor."""
    rng = np.random.default_rng(d)
    A, B = rand_c(rng, (d, d)), rand_c(rng, (d, d))
    ref = A @ B
    beta = PM.split_beta(d)
    ma = np.abs(np.stack([A.real, A.imag])).max()
    mb = np.abs(np.stack([B.real, B.imag])).max()
    errs = []
    for L in range(2, 8):
        err = np.abs(PM.df_value(PM.split_product(A, B, L, accumulate=accumulate)) - ref).max()
        bound = (L + 2) * 2 * d * (2 * ma) * (2 * mb) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta)) \
            + 1e-13 * d * ma * mb
        assert err <= bound, (L, err, bound)
        errs.append(err)
    for L in range(2, 5):   # truncation-dominated: about 2^-beta per extra digit
        assert errs[L - 1] < errs[L - 2] * 2.0 ** (4 - beta), errs


@pytest.mark.parametrize("allow18", [False, True])
def test_expm_model_matches_eigendecomposition(allow18):
    """The modelled split exponential, by Paterson-Stockmeyer or by the degree-18
    five-product scheme, against the oracle's exp(-i H) (eigendecomposition)."""
    rng = np.random.default_rng(4)
    d = 24
    H = np.stack([0.4 * (a + a.conj().T) for a in rand_c(rng, (3, d, d))])
    ref = np.stack([oracle.expm_minus_i(h) for h in H])
    errs = {}
    for L in (3, 6):
        U, (m, _) = PM.expm_split(H, L, allow18=allow18)
        assert (m == 18) == allow18
        errs[L] = np.abs(PM.df_value(U) - ref).max()
    assert errs[6] < 1e-10 and errs[3] > 100 * errs[6], errs


def test_expm_model_of_a_diagonal_is_the_exact_phase():
    d = 9
    lam = np.linspace(-3.0, 3.0, d)
    U, _ = PM.expm_split(np.diag(lam).astype(complex)[None], 6)
    np.testing.assert_allclose(PM.df_value(U)[0], np.diag(np.exp(-1j * lam)), atol=1e-12, rtol=0)


def test_config0_tolerance_reached_from_five_digits():
    """The d = 30 transmon-resonator workload, first 200 intervals: the model predicts
    errors within 1e-6 of the oracle from L = 5 digits on, and well above it at L = 3,
    so the 1e-6 tolerance separates the digit counts."""
    wl = W.config(0, N=200)
    ref, parts = oracle.evolve_workload(wl, return_parts=True)
    errs = {}
    for L in (3, 5, 6):
        psi, _ = PM.evolve_state_split(parts["Hbar"], wl.psi0, L)
        errs[L] = np.abs(psi - ref).max()
    assert errs[3] > 1e-5 and errs[5] < 1e-7 and errs[6] < errs[5], errs


def test_a_separate_level3_accumulator_lowers_the_floor():
    """With truncating accumulation, the shared level->=3 accumulator sets the error floor
    from L = 6 on; keeping level 3 apart (five accumulators) lowers it by well over 10x."""
    rng = np.random.default_rng(9)
    d = 64
    A, B = rand_c(rng, (d, d)), rand_c(rng, (d, d))
    ref = A @ B
    e4 = np.abs(PM.df_value(PM.split_product(A, B, 7, groups=4)) - ref).max()
    e5 = np.abs(PM.df_value(PM.split_product(A, B, 7, groups=5)) - ref).max()
    e4_l6 = np.abs(PM.df_value(PM.split_product(A, B, 6, groups=4)) - ref).max()
    assert e4 > 0.5 * e4_l6 and e5 < e4 / 10, (e4_l6, e4, e5)


def test_three_pass_tf32_products_cannot_reach_the_split_tolerance():
    """The interface sketch's TF32x3 mode: products hi hi + hi lo + lo hi of TF32 halves,
    accumulated in one FP32 accumulator, carry about 2^-22 of relative error per product
    (the FP32 accumulator, not the operand halves, sets it), 10^4 times the 6-digit split
    product's; over 200 intervals of the d = 30 workload the modelled state misses the
    stated 1e-6 while the 5-digit split stays two orders inside it."""
    rng = np.random.default_rng(17)
    d = 64
    A, B = rand_c(rng, (d, d)), rand_c(rng, (d, d))
    ref = A @ B
    rel_tf = np.abs(PM.tf32x3_product(A, B) - ref).max() / np.abs(ref).max()
    rel_l6 = np.abs(PM.df_value(PM.split_product(A, B, 6)) - ref).max() / np.abs(ref).max()
    assert 1e-8 < rel_tf < 1e-5 and rel_l6 < 1e-4 * rel_tf, (rel_tf, rel_l6)
    wl = W.config(0, N=200)
    ref_psi, parts = oracle.evolve_workload(wl, return_parts=True)
    psi = np.asarray(wl.psi0, dtype=np.complex128)
    for H in parts["Hbar"]:
        tau = np.trace(H).real / wl.d
        psi = PM.expm_tf32x3(H - tau * np.eye(wl.d), tau) @ psi
    err_tf = np.abs(psi - ref_psi).max()
    assert err_tf > 1e-6, err_tf
