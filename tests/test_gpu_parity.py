"""GPU parity of every step of the path against the CPU FP64 oracle (through the C ABI).

Tolerances (written per test):
  * FP64 mode: the oracle's own rounding level, ~1e-13 relative per product,
    and the stated max-abs bound 1e-11 on whole evolutions.
  * split mode: a product with L digits of beta bits errs by about
    (L + 2) * 2d * 2^{-beta L} * max|A| * max|B| in the worst case; whole
    evolutions must meet the stated max-abs bound 1e-6.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    M.load()
    c = M.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rand_c(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


def rand_herm(rng, d, scale=1.0):
    a = rand_c(rng, (d, d))
    return scale * 0.5 * (a + a.conj().T)


def split_beta(d):
    for beta in range(8, 1, -1):
        if 2.0 ** (2 * beta - 1) * 2 * d <= 2.0 ** 24:
            return beta
    return 2


# ----------------------------------------------------------------------------
# quadrature and the first-order term
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 5, 8, 16, 33, 64])
def test_quadrature_nodes_match_leggauss(P):
    x, w = M.mg_quadrature_nodes(P)
    xr, wr = oracle.gauss_legendre(P)
    # numpy's own weights err by up to 2.3e-15 at P = 64 (numpy 2.5)
    np.testing.assert_allclose(x, xr, atol=4e-15, rtol=0)
    np.testing.assert_allclose(w, wr, atol=4e-15, rtol=0)


def test_coefficients_match_oracle(ctx):
    wl = W.config(1, N=300)
    samples, w = M.node_samples(wl, 300)
    c = torch.empty((300, wl.K), dtype=torch.float64, device="cuda")
    M.mg_coefficients(ctx, 300, wl.P, wl.K, wl.dt, cuda(w), cuda(samples), c)
    torch.cuda.synchronize()
    ref = oracle.drive_coefficients(samples, oracle.gauss_legendre(wl.P)[1], wl.dt)
    np.testing.assert_allclose(c.cpu().numpy(), ref, atol=1e-16, rtol=1e-13)


@pytest.mark.parametrize("d,K,N", [(1, 0, 3), (30, 1, 19), (45, 3, 8), (129, 2, 9)])
def test_build_omega_matches_oracle(ctx, d, K, N):
    rng = np.random.default_rng(d + K)
    H0 = rand_herm(rng, d, 3.0)
    Hk = np.stack([rand_herm(rng, d) for _ in range(K)]) if K else np.zeros((0, d, d), complex)
    c = rng.normal(size=(N, K)) * 0.1
    dt = 0.05
    Hbar = torch.empty((N, d, d), dtype=torch.complex128, device="cuda")
    tau = torch.empty(N, dtype=torch.float64, device="cuda")
    nrm = torch.empty(N, dtype=torch.float64, device="cuda")
    M.mg_build_omega(ctx, N, d, K, dt, cuda(H0), cuda(Hk) if K else None, cuda(c) if K else None, Hbar, tau, nrm)
    torch.cuda.synchronize()
    for n in range(N):
        ref = oracle.first_order_term(H0, Hk, c[n], dt)
        np.testing.assert_allclose(Hbar[n].cpu().numpy(), ref, atol=1e-14, rtol=0)
        t = np.trace(ref).real / d
        assert abs(tau[n].item() - t) < 1e-14
        # the 1-norm only selects the squaring count: the kernel returns an upper bound
        # within 2^-19 relative (FP32 magnitudes widened by 2^-20, summed in FP64)
        exact = np.linalg.norm(ref - t * np.eye(d), 1)
        assert exact * (1 - 1e-12) <= nrm[n].item() <= exact * (1 + 2.0 ** -19) + 1e-300


# ----------------------------------------------------------------------------
# matrix products
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d,batch", [(1, 3), (7, 2), (30, 5), (64, 2), (65, 3), (129, 2), (200, 1)])
def test_cgemm_fp64(ctx, d, batch):
    rng = np.random.default_rng(d)
    A, B = rand_c(rng, (batch, d, d)), rand_c(rng, (batch, d, d))
    C = torch.empty((batch, d, d), dtype=torch.complex128, device="cuda")
    M.mg_cgemm(ctx, batch, d, cuda(A), cuda(B), C, M.MG_PREC_FP64)
    torch.cuda.synchronize()
    np.testing.assert_allclose(C.cpu().numpy(), A @ B, atol=1e-13 * d, rtol=0)


@pytest.mark.parametrize("d", [1, 5, 16, 30])
def test_cgemm_split_exact_on_small_integers(ctx, d):
    """Integer entries |a| <= 3 are one exact digit: the split product must equal the exact one bit for bit,
    also right after a product with more digits has left nonzero accumulators behind in TMEM."""
    rng = np.random.default_rng(100 + d)
    X = cuda(rand_c(rng, (4, 200, 200)))
    M.mg_cgemm(ctx, 4, 200, X, X, torch.empty_like(X), M.MG_PREC_SPLIT, 8)
    A = rng.integers(-3, 4, (2, d, d)) + 1j * rng.integers(-3, 4, (2, d, d))
    B = rng.integers(-3, 4, (2, d, d)) + 1j * rng.integers(-3, 4, (2, d, d))
    C = torch.empty((2, d, d), dtype=torch.complex128, device="cuda")
    M.mg_cgemm(ctx, 2, d, cuda(A), cuda(B), C, M.MG_PREC_SPLIT, 2)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), A @ B)


@pytest.mark.parametrize("d,L", [(30, 2), (30, 4), (30, 6), (64, 6), (129, 3), (129, 6), (200, 8), (300, 5),
                                 (729, 6)])
def test_cgemm_split_within_digit_bound(ctx, d, L):
    rng = np.random.default_rng(7 * d + L)
    batch = 2
    A, B = rand_c(rng, (batch, d, d)), rand_c(rng, (batch, d, d))
    C = torch.empty((batch, d, d), dtype=torch.complex128, device="cuda")
    M.mg_cgemm(ctx, batch, d, cuda(A), cuda(B), C, M.MG_PREC_SPLIT, L)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    ref = A @ B
    beta = split_beta(d)
    ma = np.abs(np.stack([A.real, A.imag])).max()
    mb = np.abs(np.stack([B.real, B.imag])).max()
    # digit truncation plus the FP32 rounding of the level->=3 accumulator
    bound = (L + 2) * 2 * d * (2 * ma) * (2 * mb) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta)) \
        + 1e-13 * d * ma * mb
    err = np.abs(got - ref).max()
    assert err <= bound, (err, bound)
    # and it is a real approximation: the error falls with every digit
    if L >= 4:
        assert err <= 1e-5 * np.abs(ref).max()


# ----------------------------------------------------------------------------
# exponential
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d,scale", [(1, 3.0), (2, 1.0), (30, 0.5), (30, 8.0), (100, 2.0), (129, 0.05)])
def test_expm_fp64_matches_oracle(ctx, d, scale):
    rng = np.random.default_rng(d)
    A = np.stack([rand_herm(rng, d, scale) for _ in range(3)])
    U = torch.empty_like(cuda(A))
    sq = torch.zeros(3, dtype=torch.int32, device="cuda")
    M.mg_expm(ctx, 3, d, cuda(A), U, M.MG_PREC_FP64, 6, sq)
    torch.cuda.synchronize()
    for b in range(3):
        ref = oracle.expm_minus_i(A[b])
        nrm = np.linalg.norm(A[b] - np.trace(A[b]).real / d * np.eye(d), 1)
        np.testing.assert_allclose(U[b].cpu().numpy(), ref, atol=5e-15 * d * max(1.0, nrm), rtol=0)


@pytest.mark.parametrize("d,L", [(30, 6), (100, 5), (129, 7), (256, 6)])
def test_expm_split_matches_oracle(ctx, d, L):
    rng = np.random.default_rng(d + L)
    A = np.stack([rand_herm(rng, d, 0.3) for _ in range(2)])
    U = torch.empty_like(cuda(A))
    M.mg_expm(ctx, 2, d, cuda(A), U, M.MG_PREC_SPLIT, L)
    torch.cuda.synchronize()
    beta = split_beta(d)
    for b in range(2):
        ref = oracle.expm_minus_i(A[b])
        err = np.abs(U[b].cpu().numpy() - ref).max()
        # ~10 products, each with digit truncation 2d 2^{-beta L} and an FP32-accumulation
        # floor of the level->=3 accumulator measured at about 2e-14 d^1.5 (relative)
        assert err < 100 * (2 * d * 2.0 ** (-beta * L) + 2e-14 * d ** 1.5), err


def test_expm_diagonal_is_exact_phase(ctx):
    lam = np.linspace(-20, 20, 33)
    A = np.diag(lam).astype(np.complex128)[None]
    U = torch.empty_like(cuda(A))
    M.mg_expm(ctx, 1, 33, cuda(A), U, M.MG_PREC_FP64, 6)
    torch.cuda.synchronize()
    np.testing.assert_allclose(np.diag(U[0].cpu().numpy()), np.exp(-1j * lam), atol=1e-13, rtol=0)
    off = U[0].cpu().numpy() - np.diag(np.diag(U[0].cpu().numpy()))
    assert np.abs(off).max() == 0.0


# ----------------------------------------------------------------------------
# propagation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("N,d,prec", [(1, 5, 0), (2, 5, 0), (37, 12, 0), (37, 12, 1), (64, 40, 1)])
def test_propagate_tree_matches_sequential_product(ctx, N, d, prec):
    rng = np.random.default_rng(N * d)
    Us = np.stack([oracle.expm_minus_i(rand_herm(rng, d, 0.7)) for _ in range(N)])
    out = torch.empty((d, d), dtype=torch.complex128, device="cuda")
    M.mg_propagate(ctx, N, d, cuda(Us), M.MG_OUT_PROPAGATOR, None, out, 0, prec, 6)
    torch.cuda.synchronize()
    ref = oracle.propagate_unitary(Us)
    tol = 1e-12 if prec == 0 else 1e-9
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=tol, rtol=0)
    psi = torch.empty(d, dtype=torch.complex128, device="cuda")
    psi0 = W.basis_state(d, 1)
    M.mg_propagate(ctx, N, d, cuda(Us), M.MG_OUT_STATE, cuda(psi0), psi, 0, prec, 6)
    torch.cuda.synchronize()
    np.testing.assert_allclose(psi.cpu().numpy(), oracle.propagate_state(Us, psi0), atol=1e-12, rtol=0)


@pytest.mark.parametrize("d,prec", [(24, M.MG_PREC_FP64), (24, M.MG_PREC_SPLIT), (300, M.MG_PREC_FP64)])
def test_reorth_removes_scale_drift(ctx, d, prec):
    """Propagators scaled by (1 + 1e-6) make the product drift by (1 + 1e-6)^N.  The polar
    factor of c V (c > 0, V unitary) is V, so re-orthonormalising every R intervals (N a
    multiple of R) takes the product back to that of the unitaries, and renormalising psi
    takes the state back to the unit-norm result."""
    rng = np.random.default_rng(d + 100 * prec)
    N, R, eps = 32, 8, 1e-6
    Us = np.stack([oracle.expm_minus_i(rand_herm(rng, d, 0.7)) for _ in range(N)])
    psi0 = W.basis_state(d, 1)
    ref_U, ref_psi = oracle.propagate_unitary(Us), oracle.propagate_state(Us, psi0)
    Ud = cuda((1.0 + eps) * Us)
    tol_U = 1e-11 if prec == M.MG_PREC_FP64 else 1e-9
    for reorth in (0, R):
        U = torch.empty((d, d), dtype=torch.complex128, device="cuda")
        M.mg_propagate(ctx, N, d, Ud, M.MG_OUT_PROPAGATOR, None, U, reorth, prec, 6)
        psi = torch.empty(d, dtype=torch.complex128, device="cuda")
        M.mg_propagate(ctx, N, d, Ud, M.MG_OUT_STATE, cuda(psi0), psi, reorth, prec, 6)
        torch.cuda.synchronize()
        err_U = np.abs(U.cpu().numpy() - ref_U).max()
        err_psi = np.abs(psi.cpu().numpy() - ref_psi).max()
        if reorth:
            assert err_U <= tol_U and err_psi <= 1e-12, (err_U, err_psi)
        else:   # the drift the step removes is there: 3.2e-5 relative
            assert err_U > 1e-5 * np.abs(ref_U).max() and err_psi > 1e-5 * np.abs(ref_psi).max(), (err_U, err_psi)


@pytest.mark.parametrize("prec,L,tol", [(M.MG_PREC_FP64, 6, 1e-11), (M.MG_PREC_SPLIT, 6, 1e-6)])
def test_evolve_with_reorth_matches_oracle(ctx, prec, L, tol):
    """Whole evolutions with re-orthonormalisation every 7 intervals (no chunk or tree level
    aligns with 7) give the oracle's result, for a state and for a full propagator."""
    for wl in (W.config(0, N=100), W.transmon_resonator(nt=3, nr=10, N=60, unitary=True)):
        out, rep = M.evolve_workload(ctx, wl, prec, L, reorth_every=7)
        ref = oracle.evolve_workload(wl)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= tol, (wl.name, err)


# ----------------------------------------------------------------------------
# whole evolutions
# ----------------------------------------------------------------------------
def test_evolve_transmon_resonator_d30_fp64(ctx):
    """The d = 30 workload (1000 intervals, 16 points, psi0 = |0,0>) within 1e-11 of the oracle."""
    wl = W.config(0)
    psi, rep = M.evolve_workload(ctx, wl, M.MG_PREC_FP64)
    ref = oracle.evolve_workload(wl)
    err = np.abs(psi.cpu().numpy() - ref).max()
    assert err <= 1e-11, err
    assert rep["unitarity_defect"] < 1e-12


@pytest.mark.parametrize("L", [5, 6])
def test_evolve_transmon_resonator_d30_split(ctx, L):
    wl = W.config(0)
    psi, rep = M.evolve_workload(ctx, wl, M.MG_PREC_SPLIT, L)
    ref = oracle.evolve_workload(wl)
    err = np.abs(psi.cpu().numpy() - ref).max()
    assert err <= 1e-6, err


@pytest.mark.parametrize("prec,L,tol", [(0, 6, 1e-11), (1, 6, 1e-6), (1, 7, 1e-6)])
def test_evolve_chain_d729_prefix(ctx, prec, L, tol):
    """The d = 729 chain (full propagator) on its first 24 intervals."""
    wl = W.config(1)
    n = 24
    U, rep = M.evolve_workload(ctx, wl, prec, L, N=n)
    ref = oracle.evolve_workload(wl, n_intervals=n)
    err = np.abs(U.cpu().numpy() - ref).max()
    assert err <= tol, err


def test_evolve_constant_hamiltonian_exact(ctx):
    """Time-independent H: U(T) = exp(-i H T) for any number of intervals (ragged tree of 13)."""
    rng = np.random.default_rng(3)
    d = 21
    H0 = rand_herm(rng, d, 2.0)
    wl = W.Workload("const", H0, np.zeros((1, d, d), complex) + rand_herm(rng, d)[None], W.ConstantDrive(np.array([0.3])),
                    0.0, 1.7, 13, 4, None)
    U, _ = M.evolve_workload(ctx, wl, M.MG_PREC_FP64)
    ref = oracle.expm_minus_i(wl.T * (wl.H0 + 0.3 * wl.Hk[0]))
    np.testing.assert_allclose(U.cpu().numpy(), ref, atol=1e-12, rtol=0)


def test_evolve_host_pointers_match_device(ctx):
    wl = W.config(0, N=50)
    samples, w = M.node_samples(wl)
    plan = M.Plan(ctx, wl.H0, wl.Hk)  # host operators
    plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, torch.from_numpy(samples))
    out_h = torch.empty(wl.d, dtype=torch.complex128).pin_memory()
    plan.evolve(M.MG_OUT_STATE, torch.from_numpy(wl.psi0), out_h, host=True)
    ref = oracle.evolve_workload(wl)
    assert np.abs(out_h.numpy() - ref).max() <= 1e-11


# ----------------------------------------------------------------------------
# many uneven jobs in shared launches (mg_evolve_batch)
# ----------------------------------------------------------------------------
def _ref_and_tol(wl, prec):
    """The oracle's result and the bound a GPU result must meet.

    Split mode: the stated 1e-6, flat.  FP64 mode: the stated 1e-11, or, for the random
    jobs with very long intervals (|Hbar_n|_1 up to ~1e4 rad), 4 u |Hbar|_1 N (u = 2^-53)
    if that is larger -- the rounding scale of any FP64 evolution of these jobs: the oracle
    itself and its evolution through scipy's expm differ by up to that bound
    (test_oracle_self_consistency_on_high_norm_instances)."""
    ref, parts = oracle.evolve_workload(wl, return_parts=True)
    if prec == M.MG_PREC_SPLIT:
        return ref, 1e-6
    hmax = max(np.abs(h).sum(axis=0).max() for h in parts["Hbar"])
    return ref, max(1e-11, 4 * 2.0 ** -53 * hmax * wl.N)


def _small_jobs(seed=21, n=10):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        wl = W.random_instance(rng, name=f"job{i}", N_range=(5, 40), d_range=(16, 110))
        if i % 3 == 2:
            wl.psi0 = None   # full propagator
        jobs.append(wl)
    # a few fixed odd sizes
    jobs.append(W.transmon_resonator(nt=3, nr=7, N=17, name="d21"))
    jobs.append(W.transmon_resonator(nt=2, nr=3, N=9, name="d6", unitary=True))
    return jobs


@pytest.mark.parametrize("prec,L,tol,reorth", [(0, 6, 1e-11, 0), (1, 6, 1e-6, 0), (0, 6, 1e-11, 5), (1, 6, 1e-6, 5)])
def test_evolve_batch_matches_oracle_per_job(ctx, prec, L, tol, reorth):
    """Every job of an uneven batch against the oracle, also with re-orthonormalisation
    every 5 intervals (which moves a result by its unitarity defect only)."""
    jobs = _small_jobs()
    plans, outs, ins, kinds = [], [], [], []
    for wl in jobs:
        samples, w = M.node_samples(wl)
        p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), prec, L)
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
    try:
        status = M.mg_evolve_batch(ctx, plans, kinds, ins, outs, reorth)
        torch.cuda.synchronize()
        assert status == [0] * len(jobs)
        worst = []
        for wl, o in zip(jobs, outs):
            ref, t = _ref_and_tol(wl, prec)
            err = np.abs(o.cpu().numpy() - ref).max()
            worst.append((err / t, wl.name, wl.d, wl.N, err, t))
            assert err <= t, (wl.name, wl.d, wl.N, err, t)
        r, name, d, n, err, t = max(worst)
        print(f"batch prec={prec} reorth={reorth}: worst job {name} (d={d}, N={n}) error {err:.2e}, bound {t:.2e}")
    finally:
        for p in plans:
            p.close()


def test_evolve_batch_result_same_alone_and_in_mix(ctx):
    """A job's result does not depend on the other jobs of the batch (within the split tolerance)."""
    jobs = _small_jobs(seed=5, n=8)
    target = W.transmon_resonator(nt=4, nr=9, N=33, name="target")
    alone, _ = M.evolve_workload(ctx, target, M.MG_PREC_SPLIT, 6)
    plans, outs, ins, kinds = [], [], [], []
    for wl in jobs[:4] + [target] + jobs[4:]:
        samples, w = M.node_samples(wl)
        p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_SPLIT, 6)
        p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
        plans.append(p)
        state = wl.psi0 is not None
        kinds.append(M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR)
        ins.append(cuda(wl.psi0) if state else None)
        outs.append(torch.empty(wl.d if state else (wl.d, wl.d), dtype=torch.complex128, device="cuda"))
    M.mg_evolve_batch(ctx, plans, kinds, ins, outs)
    torch.cuda.synchronize()
    assert np.abs(outs[4].cpu().numpy() - alone.cpu().numpy()).max() <= 1e-6
    for p in plans:
        p.close()


def test_evolve_batch_nonfinite_job_fails_alone(ctx):
    jobs = _small_jobs(seed=9, n=4)
    plans, outs, ins, kinds = [], [], [], []
    for i, wl in enumerate(jobs):
        samples, w = M.node_samples(wl)
        if i == 1:
            samples = samples.copy()
            samples[2, 3, 0] = np.nan
        p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_FP64)
        p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
        plans.append(p)
        state = wl.psi0 is not None
        kinds.append(M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR)
        ins.append(cuda(wl.psi0) if state else None)
        outs.append(torch.empty(wl.d if state else (wl.d, wl.d), dtype=torch.complex128, device="cuda"))
    status = M.mg_evolve_batch(ctx, plans, kinds, ins, outs)
    torch.cuda.synchronize()
    assert status[1] == M.MG_ENONFINITE
    for i, (wl, o) in enumerate(zip(jobs, outs)):
        if i == 1:
            continue
        assert status[i] == 0
        ref, t = _ref_and_tol(wl, M.MG_PREC_FP64)
        assert np.abs(o.cpu().numpy() - ref).max() <= t
    for p in plans:
        p.close()


def test_evolve_nonfinite_samples_rejected(ctx):
    wl = W.config(0, N=20)
    samples, w = M.node_samples(wl)
    samples[3, 0, 0] = np.inf
    p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk))
    p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
    out = torch.empty(wl.d, dtype=torch.complex128, device="cuda")
    with pytest.raises(M.MagnusError) as e:
        p.evolve(M.MG_OUT_STATE, cuda(wl.psi0), out)
    assert e.value.code == M.MG_ENONFINITE
    p.close()


def test_plan_rejects_non_hermitian_operator(ctx):
    rng = np.random.default_rng(0)
    H0 = rand_c(rng, (5, 5))
    with pytest.raises(M.MagnusError) as e:
        M.Plan(ctx, cuda(H0), cuda(rand_herm(rng, 5)[None]), flags=M.MG_FLAG_CHECK_HERMITIAN)
    assert e.value.code == M.MG_ENOTHERM


# ----------------------------------------------------------------------------
# second-order Magnus term (Eq. magnus-avg, commutator line)
# ----------------------------------------------------------------------------
def _second_order_cases():
    return [
        W.transmon_resonator(nt=3, nr=2, T=2.0, sigma=0.5, omega0=0.4, N=20, P=16, name="tr6"),
        W.transmon_chain(n_sites=3, levels=2, J=0.05, seed=7, omega0_max=0.3, T=4.0, sigma=1.0, N=12, P=16,
                         unitary=True, name="chain8_K3"),
    ]


@pytest.mark.parametrize("prec,L,tol", [(0, 6, 1e-11), (1, 6, 1e-8)])
def test_second_order_magnus_matches_oracle(ctx, prec, L, tol):
    for wl in _second_order_cases():
        out, rep = M.evolve_workload(ctx, wl, prec, L, order=2)
        ref2 = oracle.evolve_workload_second_order(wl)
        ref1 = oracle.evolve_workload(wl)
        got = out.cpu().numpy()
        assert np.abs(got - ref2).max() <= tol, (wl.name, np.abs(got - ref2).max())
        # the commutator term matters for these drives: order 1 is far away
        assert np.abs(ref2 - ref1).max() > 1e3 * tol


# ----------------------------------------------------------------------------
# action-based state path with sparse operators (MG_FLAG_STATE_ACTION)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("order", [1, 2])
def test_action_state_path_matches_oracle(ctx, order):
    diag = W.config(0, N=50)   # commuting diagonal operators: Gershgorin's interval is the spectrum
    diag.H0 = np.diag(np.diag(diag.H0))
    diag.Hk = np.diag(np.arange(diag.d, dtype=np.complex128))[None]
    cases = [W.config(0, N=120), W.transmon_resonator(nt=3, nr=2, T=2.0, sigma=0.5, omega0=0.4, N=20, P=16),
             W.transmon_chain(n_sites=3, levels=3, J=0.02, seed=4, omega0_max=0.2, T=5.0, sigma=1.2, N=30, P=16,
                              unitary=False), diag]
    for wl in cases:
        out, _ = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, order=order, flags=M.MG_FLAG_STATE_ACTION)
        ref = oracle.evolve_workload(wl) if order == 1 else oracle.evolve_workload_second_order(wl)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= 1e-11, (wl.name, err)


def test_action_state_path_cluster_matches_oracle(ctx):
    # large sparse jobs run as one thread block cluster per job (rows split over the
    # CTAs, ragged last block); d = 729 chain and d = 512 three-site 8-level chain
    cases = [W.transmon_chain(n_sites=6, levels=3, J=0.01, seed=1, omega0_max=0.05, T=1.0, sigma=0.3, N=8,
                              P=16, unitary=False, name="chain729_state"),
             W.transmon_chain(n_sites=3, levels=8, J=0.02, seed=5, omega0_max=0.1, T=0.8, sigma=0.3, N=6, P=8,
                              all_to_all=True, unitary=False, name="a2a512_state")]
    for wl in cases:
        out, rep = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, flags=M.MG_FLAG_STATE_ACTION)
        assert rep["action_ctas"] >= 2, (wl.name, rep["action_ctas"])
        ref = oracle.evolve_workload(wl)
        err = np.abs(out.cpu().numpy() - ref).max()
        assert err <= 1e-11, (wl.name, err)


def test_action_state_path_in_batch(ctx):
    jobs = _small_jobs(seed=31, n=6)
    plans, outs, ins, kinds = [], [], [], []
    for wl in jobs:
        samples, w = M.node_samples(wl)
        state = wl.psi0 is not None
        p = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_FP64, 6, M.MG_FLAG_STATE_ACTION)
        p.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
        plans.append(p)
        kinds.append(M.MG_OUT_STATE if state else M.MG_OUT_PROPAGATOR)
        ins.append(cuda(wl.psi0) if state else None)
        outs.append(torch.empty(wl.d if state else (wl.d, wl.d), dtype=torch.complex128, device="cuda"))
    try:
        status = M.mg_evolve_batch(ctx, plans, kinds, ins, outs)
        torch.cuda.synchronize()
        assert status == [0] * len(jobs)
        for wl, o in zip(jobs, outs):
            ref, t = _ref_and_tol(wl, M.MG_PREC_FP64)
            err = np.abs(o.cpu().numpy() - ref).max()
            assert err <= t, (wl.name, err, t)
    finally:
        for p in plans:
            p.close()


def test_action_state_path_rejects_unbounded_work(ctx):
    # a norm bound that would need more than 16384 sub-steps in one interval ends the
    # job with MG_EUNSUPPORTED from inside the kernel instead of running on
    wl = W.config(0, N=2)
    wl.H0 = wl.H0 * 100.0
    with pytest.raises(RuntimeError, match="sub-steps"):
        M.evolve_workload(ctx, wl, M.MG_PREC_FP64, flags=M.MG_FLAG_STATE_ACTION)


# ----------------------------------------------------------------------------
# stroboscopic trajectory output (MG_OUT_TRAJECTORY)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("prec,flags,tol", [(0, 0, 1e-11), (1, 0, 1e-6), (0, 8, 1e-11)])
def test_trajectory_matches_oracle(ctx, prec, flags, tol):
    wl = W.config(0, N=150)
    out, rep = M.evolve_workload(ctx, wl, prec, 6, flags=flags, trajectory=True)
    U = oracle.evolve_workload(wl, return_parts=True)[1]["U"]
    _, ref = oracle.propagate_state(U, wl.psi0, trajectory=True)
    got = out.cpu().numpy()
    assert got.shape == ref.shape == (wl.N + 1, wl.d)
    assert np.array_equal(got[0], wl.psi0)
    assert np.abs(got - ref).max() <= tol


def test_trajectory_large_d_and_host_buffers(ctx):
    # d > 256 takes the one-launch-per-interval state path; host output buffer
    wl = W.transmon_chain(n_sites=6, levels=3, J=0.01, seed=2, omega0_max=0.05, T=0.5, sigma=0.2, N=5, P=16,
                          unitary=False)
    samples, w = M.node_samples(wl)
    plan = M.Plan(ctx, cuda(wl.H0), cuda(wl.Hk), M.MG_PREC_FP64, 6)
    plan.set_controls(wl.N, wl.P, wl.t0, wl.dt, w, cuda(samples))
    out = torch.empty((wl.N + 1, wl.d), dtype=torch.complex128).pin_memory()
    psi0 = torch.from_numpy(wl.psi0).pin_memory()
    plan.evolve(M.MG_OUT_TRAJECTORY, psi0, out, 0, host=True)
    plan.close()
    U = oracle.evolve_workload(wl, return_parts=True)[1]["U"]
    _, ref = oracle.propagate_state(U, wl.psi0, trajectory=True)
    assert np.abs(out.numpy() - ref).max() <= 1e-11


@pytest.mark.parametrize("flags", [0, M.MG_FLAG_STATE_ACTION])
def test_state_edge_cases_d1_k0_and_time_independent(ctx, flags):
    # d = 1, no controls: psi(T) = e^{-i h T} psi0
    wl = W.Workload("d1_k0", np.array([[2.0 + 0j]]), np.zeros((0, 1, 1), complex), W.ConstantDrive(np.zeros(0)),
                    0.0, 1.3, 3, 4, np.array([1.0 + 0j]))
    out, _ = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, flags=flags)
    assert abs(out.cpu().numpy()[0] - np.exp(-2.6j)) < 1e-14
    # time-independent d = 21 (constant drive): psi(T) = exp(-i H T) psi0 for any N, incl. N = 1
    rng = np.random.default_rng(8)
    d = 21
    H0, H1 = rand_herm(rng, d, 2.0), rand_herm(rng, d)
    psi0 = rand_c(rng, d)
    psi0 /= np.linalg.norm(psi0)
    for N in (1, 7):
        wl = W.Workload("const_state", H0, H1[None], W.ConstantDrive(np.array([0.3])), 0.0, 1.7, N, 4, psi0)
        out, _ = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, flags=flags)
        ref = oracle.expm_minus_i(wl.T * (H0 + 0.3 * H1)) @ psi0
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12, N


def test_trajectory_single_interval(ctx):
    wl = W.config(0, N=1, T=0.5)   # one interval of 0.5 ns (||Hbar|| ~ 100 rad)
    out, _ = M.evolve_workload(ctx, wl, M.MG_PREC_FP64, trajectory=True)
    ref = oracle.evolve_workload(wl)
    got = out.cpu().numpy()
    assert got.shape == (2, wl.d)
    assert np.array_equal(got[0], wl.psi0) and np.abs(got[1] - ref).max() <= 1e-13


@pytest.mark.parametrize("prec,L,tol", [(M.MG_PREC_FP64, 6, 1e-13), (M.MG_PREC_SPLIT, 6, 1e-8)])
def test_expm_nilpotent_is_finite_taylor_sum(ctx, prec, L, tol):
    """A strictly upper-triangular exponent: exp(-i A) is the finite sum of (-i A)^j / j!, j < d.
    The evaluation uses no Hermitian structure beyond the real trace shift, and the trace is 0."""
    rng = np.random.default_rng(41)
    d = 12
    A = np.triu(rng.uniform(-1.0, 1.0, (2, d, d)), 1).astype(np.complex128)
    U = torch.empty_like(cuda(A))
    M.mg_expm(ctx, 2, d, cuda(A), U, prec, L)
    torch.cuda.synchronize()
    for b in range(2):
        X = -1j * A[b]
        ref, term = np.eye(d, dtype=complex), np.eye(d, dtype=complex)
        for j in range(1, d):
            term = term @ X / j
            ref = ref + term
        assert np.abs(U[b].cpu().numpy() - ref).max() <= tol * np.abs(ref).max(), b


@pytest.mark.parametrize("d", [64, 129])
def test_cgemm_split_adversarial_row_and_column_scales(ctx, d):
    """Rows of A and columns of B scaled by powers of two from 2^-12 to 2^12: the per-row and
    per-column exponents keep every element within the unscaled digit bound times its scale."""
    rng = np.random.default_rng(5 * d)
    L = 6
    A0, B0 = rand_c(rng, (1, d, d)), rand_c(rng, (1, d, d))
    r = 2.0 ** rng.integers(-12, 13, d)
    c = 2.0 ** rng.integers(-12, 13, d)
    A, B = A0 * r[None, :, None], B0 * c[None, None, :]
    C = torch.empty((1, d, d), dtype=torch.complex128, device="cuda")
    M.mg_cgemm(ctx, 1, d, cuda(A), cuda(B), C, M.MG_PREC_SPLIT, L)
    torch.cuda.synchronize()
    ref = A[0] @ B[0]
    beta = split_beta(d)
    ma = np.abs(np.stack([A0.real, A0.imag])).max()
    mb = np.abs(np.stack([B0.real, B0.imag])).max()
    bound = (L + 2) * 2 * d * (2 * ma) * (2 * mb) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta)) \
        + 1e-13 * d * ma * mb
    scaled_err = np.abs(C[0].cpu().numpy() - ref) / (r[:, None] * c[None, :])
    assert scaled_err.max() <= bound, (scaled_err.max(), bound)


@pytest.mark.parametrize("d,L", [(30, 6), (129, 5), (300, 6), (729, 6), (700, 3), (64, 2), (200, 4), (97, 8)])
def test_cgemm_split_stage_k_variants_agree_bit_for_bit(d, L):
    """The product's pipeline stage (K = 16, 32 or 64 per stage: 32-, 64- or 128-byte operand
    rows) and the paired digit layout (two digits per row: 64-byte rows of 16-deep stages
    or 128-byte rows of 32-deep ones; even L) do not change its arithmetic: the MMAs run in the same order over K, so the results
    agree bit for bit (K = 64 applies where L <= 3 and each half of K is a multiple of 64,
    else the product takes K = 32; odd L ignores the paired layout).  The same holds for
    the M = 256 products of CTA pairs (d > 128; d = 300 has an odd number of row tiles,
    so its last pair's second CTA lies beyond row d)."""
    rng = np.random.default_rng(50 + d)
    A, B = rand_c(rng, (2, d, d)), rand_c(rng, (2, d, d))
    c = M.Context(0)
    out = {}
    for k in (32, 16, 64, "pairs", "cta32", "cta16", "cta64", "pairs2", "ctapairs", "ctapairs2"):
        c.set_digit_pairs({"pairs": 1, "ctapairs": 1, "pairs2": 2, "ctapairs2": 2}.get(str(k), 0))
        c.set_cta_pairs(str(k).startswith("cta"))
        c.set_stage_k(int(str(k)[3:]) if str(k)[3:].isdigit() and str(k).startswith("cta") else
                      (k if isinstance(k, int) else 32))
        C = torch.empty((2, d, d), dtype=torch.complex128, device="cuda")
        M.mg_cgemm(c, 2, d, cuda(A), cuda(B), C, M.MG_PREC_SPLIT, L)
        torch.cuda.synchronize()
        out[k] = C.cpu().numpy()
    c.close()
    assert np.array_equal(out[16], out[32]) and np.array_equal(out[64], out[32])
    for k in ("pairs", "pairs2", "cta32", "cta16", "cta64", "ctapairs", "ctapairs2"):
        assert np.array_equal(out[k], out[32]), (k, np.abs(out[k] - out[32]).max())
    beta = split_beta(d)
    bound = (L + 2) * 2 * d * (2 * np.abs(A).max()) * (2 * np.abs(B).max()) * (2.0 ** (-beta * L) + L * 2.0 ** (-22 - 3 * beta))
    assert np.abs(out[16] - A @ B).max() <= bound
