"""Pins of the CPU FP64 oracle against closed forms, library routines and invariants.

Each test fixes one part of the oracle to something other than itself:
quadrature exactness, exact exponentials, exactness of the first-order term for
self-commuting H(t), Rabi formulas, unitarity, and convergence to a fine-step
RK4 integration of the Schroedinger equation.  All run on the CPU.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.special

import oracle
import workloads as W

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def rand_herm(rng, d, scale=1.0):
    a = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    return scale * 0.5 * (a + a.conj().T)


def samples_for(wl, N=None):
    x, w = oracle.gauss_legendre(wl.P)
    N = wl.N if N is None else N
    return wl.drive(oracle.node_times(wl.t0, wl.dt, N, x)), w


# ----------------------------------------------------------------------------
# quadrature (Eq. magnus-first-order-coeff)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 3, 8, 16])
def test_gauss_legendre_integrates_polynomials_exactly(P):
    """P-point Gauss-Legendre is exact for degree <= 2P-1; the node map and dt/2 factor must be right."""
    rng = np.random.default_rng(P)
    deg = 2 * P - 1
    coef = rng.normal(size=(2, deg + 1))
    drive = W.PolynomialDrive(coef)
    t0, dt, N = 0.3, 0.17, 9
    x, w = oracle.gauss_legendre(P)
    c = oracle.drive_coefficients(drive(oracle.node_times(t0, dt, N, x)), w, dt)
    for k in range(2):
        anti = np.polynomial.polynomial.polyint(coef[k])
        for n in range(N):
            a, b = t0 + n * dt, t0 + (n + 1) * dt
            exact = np.polynomial.polynomial.polyval(b, anti) - np.polynomial.polynomial.polyval(a, anti)
            assert abs(c[n, k] - exact) <= 1e-13 * max(1.0, abs(exact))


def test_quadrature_matches_adaptive_integral_for_gaussian_cosine():
    """Coefficients of the d = 30 workload's drive agree with scipy.integrate.quad."""
    wl = W.config(0)
    s, w = samples_for(wl, N=wl.N)
    c = oracle.drive_coefficients(s, w, wl.dt)
    f = lambda t: float(wl.drive(np.array([t]))[0, 0])
    for n in [0, 1, 250, 499, 500, 777, 999]:
        a, b = wl.t0 + n * wl.dt, wl.t0 + (n + 1) * wl.dt
        ref, _ = scipy.integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-13, limit=200)
        assert abs(c[n, 0] - ref) <= 1e-14 + 1e-12 * abs(ref)


# ----------------------------------------------------------------------------
# first-order term (Eq. magnus-first-order-term)
# ----------------------------------------------------------------------------
def test_first_order_term_constant_drive():
    """For u_k = a_k constant, Hbar_n = dt (H0 + sum_k a_k H_k), with complex Hermitian operators."""
    rng = np.random.default_rng(5)
    d, K = 7, 3
    H0 = rand_herm(rng, d)
    Hk = np.stack([rand_herm(rng, d) for _ in range(K)])
    amp = rng.normal(size=K)
    dt, N, P = 0.25, 4, 5
    x, w = oracle.gauss_legendre(P)
    s = W.ConstantDrive(amp)(oracle.node_times(0.0, dt, N, x))
    _, Hbar, c = oracle.interval_propagators(H0, Hk, s, w, dt)
    expect = dt * (H0 + np.einsum("k,kij->ij", amp, Hk))
    for n in range(N):
        np.testing.assert_allclose(Hbar[n], expect, atol=1e-14, rtol=0)
        np.testing.assert_allclose(Hbar[n], Hbar[n].conj().T, atol=1e-15, rtol=0)


# ----------------------------------------------------------------------------
# exponential
# ----------------------------------------------------------------------------
def test_expm_diagonal_exact():
    lam = np.array([-7.3, 0.0, 1e-3, 2.5, 40.0])
    U = oracle.expm_minus_i(np.diag(lam).astype(np.complex128))
    # phases of magnitude |lambda| carry a rounding error of order |lambda| * 2^-53
    np.testing.assert_allclose(U, np.diag(np.exp(-1j * lam)), atol=4e-16 * np.max(np.abs(lam)), rtol=0)


@pytest.mark.parametrize("seed", range(6))
def test_expm_su2_closed_form(seed):
    """exp(-i(a0 I + a.sigma)) = e^{-i a0} (cos|a| I - i sin|a| (a/|a|).sigma)."""
    rng = np.random.default_rng(seed)
    a0 = rng.normal() * 3
    a = rng.normal(size=3) * (seed + 1)
    H = a0 * np.eye(2) + a[0] * SX + a[1] * SY + a[2] * SZ
    r = np.linalg.norm(a)
    n = a / r
    expect = np.exp(-1j * a0) * (math.cos(r) * np.eye(2) - 1j * math.sin(r) * (n[0] * SX + n[1] * SY + n[2] * SZ))
    np.testing.assert_allclose(oracle.expm_minus_i(H), expect, atol=2e-15 * (1 + r), rtol=0)


@pytest.mark.parametrize("d,scale", [(3, 0.1), (16, 1.0), (30, 5.0), (64, 2.0)])
def test_expm_matches_scipy_pade(d, scale):
    """Agreement with scipy.linalg.expm (an independent scaling-and-squaring Pade method)."""
    rng = np.random.default_rng(d)
    H = rand_herm(rng, d, scale)
    nrm = np.linalg.norm(H, 1)
    np.testing.assert_allclose(oracle.expm_minus_i(H), scipy.linalg.expm(-1j * H), atol=2e-14 * max(1, nrm), rtol=0)


# ----------------------------------------------------------------------------
# whole evolution: exact cases
# ----------------------------------------------------------------------------
def test_scalar_system_is_exact():
    """d = 1: U(T) = exp(-i (h0 T + h1 int_0^T u)), any N."""
    coef = np.array([[0.4, -1.1, 0.3, 0.05]])
    drive = W.PolynomialDrive(coef)
    h0, h1, T, N, P = 2.3, -0.7, 3.0, 13, 4
    x, w = oracle.gauss_legendre(P)
    dt = T / N
    U = oracle.magnus_evolve(np.array([[h0]], np.complex128), np.array([[[h1]]], np.complex128),
                             drive(oracle.node_times(0.0, dt, N, x)), w, dt)
    anti = np.polynomial.polynomial.polyint(coef[0])
    integral = np.polynomial.polynomial.polyval(T, anti)
    assert abs(U[0, 0] - np.exp(-1j * (h0 * T + h1 * integral))) < 1e-13


@pytest.mark.parametrize("N", [1, 7, 50])
def test_time_independent_hamiltonian_is_exact(N):
    """Constant H: prod_n exp(-i H dt) = exp(-i H T) for every N (independent scipy expm)."""
    rng = np.random.default_rng(N)
    d = 9
    H0, H1 = rand_herm(rng, d), rand_herm(rng, d)
    a = 0.7
    T, P = 2.0, 3
    x, w = oracle.gauss_legendre(P)
    dt = T / N
    s = W.ConstantDrive(np.array([a]))(oracle.node_times(0.0, dt, N, x))
    U = oracle.magnus_evolve(H0, H1[None], s, w, dt)
    ref = scipy.linalg.expm(-1j * T * (H0 + a * H1))
    np.testing.assert_allclose(U, ref, atol=N * 1e-14 * np.linalg.norm(T * (H0 + a * H1), 1), rtol=0)


def test_commuting_diagonal_hamiltonian_is_exact():
    """Diagonal H0 and H_k commute at all times: U = exp(-i (H0 T + sum_k C_k H_k)), C_k = int_0^T u_k."""
    rng = np.random.default_rng(11)
    d = 6
    H0 = np.diag(rng.normal(size=d) * 5).astype(np.complex128)
    Hk = np.stack([np.diag(rng.normal(size=d)).astype(np.complex128) for _ in range(2)])
    drive = W.GaussianTones(amp=np.array([[3.0], [1.5]]), freq=np.array([[9.0], [4.0]]),
                            phase=np.array([[0.3], [1.2]]), t_center=1.0, sigma=0.4)
    T, N, P = 2.0, 40, 16
    x, w = oracle.gauss_legendre(P)
    dt = T / N
    U = oracle.magnus_evolve(H0, Hk, drive(oracle.node_times(0.0, dt, N, x)), w, dt)
    C = [scipy.integrate.quad(lambda t, k=k: float(drive(np.array([t]))[0, k]), 0, T,
                              epsabs=1e-15, epsrel=1e-14, limit=400)[0] for k in range(2)]
    phase = np.diag(H0).real * T + C[0] * np.diag(Hk[0]).real + C[1] * np.diag(Hk[1]).real
    np.testing.assert_allclose(U, np.diag(np.exp(-1j * phase)), atol=1e-12, rtol=0)


def test_control_proportional_to_drift_is_exact():
    """H_1 = beta H0 (non-diagonal): U = exp(-i (T + beta C) H0) with C = int u."""
    rng = np.random.default_rng(12)
    H0 = rand_herm(rng, 5)
    beta = 0.37
    coef = np.array([[1.0, -0.5, 0.25]])
    T, N, P = 1.5, 11, 3
    x, w = oracle.gauss_legendre(P)
    dt = T / N
    U = oracle.magnus_evolve(H0, (beta * H0)[None], W.PolynomialDrive(coef)(oracle.node_times(0.0, dt, N, x)), w, dt)
    C = np.polynomial.polynomial.polyval(T, np.polynomial.polynomial.polyint(coef[0]))
    np.testing.assert_allclose(U, scipy.linalg.expm(-1j * (T + beta * C) * H0), atol=1e-13, rtol=0)


def test_piecewise_constant_drive_fixes_product_order():
    """A drive constant on each interval makes every U_n exact, so U(T) = e^{-iH_B dt} e^{-iH_A dt};
    reversing the product order fails this test for non-commuting H_A, H_B."""
    rng = np.random.default_rng(13)
    H0, H1 = rand_herm(rng, 4), rand_herm(rng, 4)
    dt, P = 0.6, 4

    def drive(t):
        t = np.asarray(t)
        return np.where(t < dt, 1.3, -0.8)[..., None]

    x, w = oracle.gauss_legendre(P)
    U = oracle.magnus_evolve(H0, H1[None], drive(oracle.node_times(0.0, dt, 2, x)), w, dt)
    UA = scipy.linalg.expm(-1j * dt * (H0 + 1.3 * H1))
    UB = scipy.linalg.expm(-1j * dt * (H0 - 0.8 * H1))
    np.testing.assert_allclose(U, UB @ UA, atol=1e-13, rtol=0)
    assert np.max(np.abs(U - UA @ UB)) > 1e-3


# ----------------------------------------------------------------------------
# two-level physics
# ----------------------------------------------------------------------------
def test_resonant_rabi_area_theorem():
    """RWA drive Omega(t)/4 sx (Eq. magnus-rwa-ham) commutes with itself: P1(T) = sin^2(A/2),
    A = int_0^T Omega(t)/2 dt, for any number of intervals."""
    wl = W.driven_qubit_rot(omega_ratio=0.33, T=10.0, N=50, rwa=True)
    s, w = samples_for(wl)
    psi = oracle.magnus_evolve(wl.H0, wl.Hk, s, w, wl.dt, wl.psi0)
    Om0, sig, tc, T = wl.drive.omega0, wl.drive.sigma, wl.drive.t_center, wl.T
    gauss_int = sig * math.sqrt(math.pi / 2) * (scipy.special.erf((T - tc) / (sig * math.sqrt(2)))
                                                - scipy.special.erf(-tc / (sig * math.sqrt(2))))
    A = 0.5 * Om0 * gauss_int
    assert abs(abs(psi[1]) ** 2 - math.sin(A / 2) ** 2) < 1e-13


def test_detuned_rabi_at_every_interval_boundary():
    """Constant detuned drive H = (Delta/2) sz + (Omega/2) sx: stroboscopic populations
    P1(t_n) = Omega^2/(Omega^2+Delta^2) sin^2(sqrt(Omega^2+Delta^2) t_n / 2)."""
    Delta, Om = 1.7, 2.9
    N, T, P = 37, 6.0, 2
    x, w = oracle.gauss_legendre(P)
    dt = T / N
    s = W.ConstantDrive(np.array([Om / 2]))(oracle.node_times(0.0, dt, N, x))
    U, _, _ = oracle.interval_propagators(0.5 * Delta * SZ, SX[None], s, w, dt)
    _, traj = oracle.propagate_state(U, np.array([1, 0], np.complex128), trajectory=True)
    tn = dt * np.arange(N + 1)
    R = math.hypot(Om, Delta)
    expect = Om ** 2 / R ** 2 * np.sin(R * tn / 2) ** 2
    np.testing.assert_allclose(np.abs(traj[:, 1]) ** 2, expect, atol=1e-13, rtol=0)


def test_unitarity_and_norm_on_transmon_resonator():
    wl = W.config(0)
    s, w = samples_for(wl, N=200)
    U, Hbar, _ = oracle.interval_propagators(wl.H0, wl.Hk, s, w, wl.dt)
    assert max(oracle.unitarity_defect(U[n]) for n in range(0, 200, 17)) < 1e-13
    psi = oracle.propagate_state(U, wl.psi0)
    assert oracle.norm_defect(psi) < 1e-13
    Uall = oracle.propagate_unitary(U)
    assert oracle.unitarity_defect(Uall) < 1e-12


# ----------------------------------------------------------------------------
# convergence to a fine-step Runge-Kutta solution
# ----------------------------------------------------------------------------
def rk4_state(Hfun, psi0, T, steps):
    """Classical RK4 for i dpsi/dt = H(t) psi."""
    psi = psi0.astype(np.complex128).copy()
    h = T / steps
    for j in range(steps):
        t = j * h
        k1 = -1j * (Hfun(t) @ psi)
        k2 = -1j * (Hfun(t + h / 2) @ (psi + h / 2 * k1))
        k3 = -1j * (Hfun(t + h / 2) @ (psi + h / 2 * k2))
        k4 = -1j * (Hfun(t + h) @ (psi + h * k3))
        psi = psi + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return psi


@pytest.mark.slow
def test_counter_rotating_qubit_converges_at_second_order():
    """Rotating-frame driven qubit with counter-rotating terms (Eq. magnus-rot-ham), Omega0/w = 0.33.
    No closed form: the first-order Magnus state converges to a fine-step RK4 solution with
    global error O(dt^2), and 50 intervals already track the 5000-interval result."""
    wl = W.driven_qubit_rot(omega_ratio=0.33, w_ghz=1.0, T=4.0, N=50)

    def Hfun(t):
        u = wl.drive(np.array([t]))[0]
        return u[0] * SX + u[1] * SX + u[2] * SY

    ref = rk4_state(Hfun, wl.psi0, wl.T, 40000)
    errs = []
    Ns = [40, 80, 160, 320]
    for N in Ns:
        x, w = oracle.gauss_legendre(wl.P)
        dt = wl.T / N
        psi = oracle.magnus_evolve(wl.H0, wl.Hk, wl.drive(oracle.node_times(0.0, dt, N, x)), w, dt, wl.psi0)
        errs.append(np.linalg.norm(psi - ref))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ns))
    assert np.all(slopes < -1.8) and np.all(slopes > -2.3), (errs, slopes)
    # the paper's protocol: 50 intervals vs 5000 intervals of the same method
    x, w = oracle.gauss_legendre(wl.P)
    fine = oracle.magnus_evolve(wl.H0, wl.Hk, wl.drive(oracle.node_times(0.0, wl.T / 5000, 5000, x)), w,
                                wl.T / 5000, wl.psi0)
    coarse = oracle.magnus_evolve(wl.H0, wl.Hk, wl.drive(oracle.node_times(0.0, wl.T / 50, 50, x)), w,
                                  wl.T / 50, wl.psi0)
    assert 1 - abs(np.vdot(fine, coarse)) ** 2 < 1e-3
    assert np.linalg.norm(fine - ref) < 1e-5


@pytest.mark.slow
def test_transmon_resonator_converges_to_rk4():
    """Small transmon (3) x resonator (2) in the lab frame (d = 6, non-commuting H(t))."""
    wl = W.transmon_resonator(nt=3, nr=2, T=2.0, sigma=0.5, omega0=0.3, N=50, P=8)

    def Hfun(t):
        return wl.H0 + wl.drive(np.array([t]))[0, 0] * wl.Hk[0]

    ref = rk4_state(Hfun, wl.psi0, wl.T, 40000)
    errs = []
    Ns = [100, 200, 400]
    for N in Ns:
        x, w = oracle.gauss_legendre(wl.P)
        dt = wl.T / N
        psi = oracle.magnus_evolve(wl.H0, wl.Hk, wl.drive(oracle.node_times(0.0, dt, N, x)), w, dt, wl.psi0)
        errs.append(np.linalg.norm(psi - ref))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ns))
    assert np.all(slopes < -1.8) and np.all(slopes > -2.3), (errs, slopes)


# ----------------------------------------------------------------------------
# second-order term (Eq. magnus-avg, second line)
# ----------------------------------------------------------------------------
def test_second_order_term_linear_drive_closed_form():
    """H(t) = H0 + t H1 on [0, tau]: [H(t1), H(t2)] = (t2 - t1)[H0, H1], so
    Hbar^(2) = -(i/2) int_0^tau int_0^t1 (t2 - t1) dt2 dt1 [H0, H1] = (i tau^3 / 12) [H0, H1]."""
    rng = np.random.default_rng(3)
    H0, H1 = rand_herm(rng, 4), rand_herm(rng, 4)
    tau = 0.8
    got = oracle.second_order_term(lambda t: H0 + t * H1, 0.0, tau, P=3)
    expect = 1j * tau ** 3 / 12 * (H0 @ H1 - H1 @ H0)
    np.testing.assert_allclose(got, expect, atol=1e-14, rtol=0)
    np.testing.assert_allclose(got, got.conj().T, atol=1e-14, rtol=0)


@pytest.mark.slow
def test_second_order_magnus_converges_at_fourth_order():
    """Hbar^(1) + Hbar^(2) (Eq. magnus-avg) is the fourth-order Magnus integrator: its global error
    against a fine-step RK4 solution falls as dt^4 (first order alone: dt^2)."""
    wl = W.transmon_resonator(nt=3, nr=2, T=2.0, sigma=0.5, omega0=0.3, N=50, P=8)

    def Hfun(t):
        return wl.H0 + wl.drive(np.array([t]))[0, 0] * wl.Hk[0]

    ref = rk4_state(Hfun, wl.psi0, wl.T, 40000)
    errs = []
    Ns = [40, 80, 160]
    for N in Ns:
        U = oracle.interval_propagators_second_order(wl.H0, wl.Hk, wl.drive, 0.0, wl.T / N, N, wl.P)
        errs.append(np.linalg.norm(oracle.propagate_state(U, wl.psi0) - ref))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ns))
    assert np.all(slopes < -3.6) and np.all(slopes > -4.5), (errs, slopes)


def test_workload_generators_give_hermitian_operators():
    """Every synthetic model generator returns exactly Hermitian H0 and H_k (the
    inputs the method assumes), drives of the declared width, and a normalised psi0."""
    rng = np.random.default_rng(3)
    models = [W.config(0, N=10), W.config(1, N=10),
              W.transmon_chain(n_sites=3, levels=4, seed=3, N=5, all_to_all=True, two_tone=True),
              W.transmon_resonator(nt=4, nr=6, N=5, unitary=True), W.spin_chain(n=4, N=5),
              W.driven_qubit_rot(N=5), W.random_instance(rng, N_range=(5, 9), d_range=(16, 40))]
    for wl in models:
        assert np.array_equal(wl.H0, wl.H0.conj().T), wl.name
        for h in wl.Hk:
            assert np.array_equal(h, h.conj().T), wl.name
        t = oracle.node_times(wl.t0, wl.dt, wl.N, oracle.gauss_legendre(wl.P)[0])
        assert wl.drive(t).shape == (wl.N, wl.P, wl.K), wl.name
        if wl.psi0 is not None:
            assert abs(np.linalg.norm(wl.psi0) - 1.0) < 1e-15, wl.name


def test_oracle_self_consistency_on_high_norm_instances():
    """The uneven random instances with long intervals (||Hbar_n||_1 up to ~1e4 rad): the
    oracle (eigendecomposition per interval) and the same evolution through
    scipy.linalg.expm (scaling and squaring with Pade) agree to a few u ||Hbar|| N, the
    oracle's own rounding scale on these jobs."""
    rng = np.random.default_rng(21)
    for i in range(6):
        wl = W.random_instance(rng, name=f"job{i}", N_range=(5, 40), d_range=(16, 110))
        ref, parts = oracle.evolve_workload(wl, return_parts=True)
        U = np.stack([scipy.linalg.expm(-1j * h) for h in parts["Hbar"]])
        alt = oracle.propagate_unitary(U) if wl.psi0 is None else oracle.propagate_state(U, wl.psi0)
        hmax = max(np.abs(h).sum(axis=0).max() for h in parts["Hbar"])
        assert np.abs(alt - ref).max() <= 4 * 2.0 ** -53 * hmax * wl.N, (wl.d, wl.N, hmax)


def test_single_job_workloads_have_the_stated_sizes():
    """d = 30 transmon-resonator: K = 1, N = 1000, P = 16, T = 50 ns, a state from |0,0>.
    d = 729 chain of six three-level transmons: K = 6, N = 2000, P = 16, T = 50 ns, full
    propagator."""
    wl0, wl1 = W.config(0), W.config(1)
    assert (wl0.d, wl0.K, wl0.N, wl0.P, wl0.T) == (30, 1, 1000, 16, 50.0)
    assert wl0.psi0 is not None and wl0.psi0[0] == 1.0 and np.count_nonzero(wl0.psi0) == 1
    assert (wl1.d, wl1.K, wl1.N, wl1.P, wl1.T) == (729, 6, 2000, 16, 50.0) and wl1.psi0 is None
    assert abs(wl1.dt - 0.025) < 1e-15 and abs(wl0.dt - 0.05) < 1e-15


def test_workload_recipes_match_the_stated_configurations():
    """The uneven batch: 512 state jobs, d = nt nr in [16, 256], N in [200, 2000], P = 16,
    one drive.  The served stream: Poisson arrivals at 200/s over 60 s, d the largest
    family member not above a log-uniform draw on [32, 2048], N in [100, 5000], state or
    unitary with probability 1/2 each."""
    jobs = W.uneven_batch()
    assert len(jobs) == 512
    assert all(16 <= j.d <= 256 and 200 <= j.N <= 2000 and j.P == 16 and j.K == 1 for j in jobs)
    assert all(j.psi0 is not None for j in jobs)
    stream = W.serving_stream()
    t = np.array([a for a, _ in stream])
    assert np.all(np.diff(t) > 0) and t[-1] <= 60.0
    assert abs(len(stream) - 12000) < 4 * math.sqrt(12000)
    for _, s in stream:
        assert 100 <= s["N"] <= 5000 and s["dt"] == 0.05 and s["output"] in ("state", "unitary")
        if s["family"] == "chain3":
            n = round(math.log(s["d"]) / math.log(3))
            assert 3 ** n == s["d"] and 27 <= s["d"] <= 729
        else:
            assert s["family"] == "transmon_resonator" and 16 <= s["d"] <= 2048
    frac_state = np.mean([s["output"] == "state" for _, s in stream])
    assert abs(frac_state - 0.5) < 4 * math.sqrt(0.25 / len(stream))


def test_streamed_evolution_equals_stored_evolution():
    """The streamed form (one interval at a time, used for the d = 4096 stored values) takes
    the same steps in the same order as evolve_workload: identical results, bit for bit,
    for propagators and states, and snapshots equal the shorter runs."""
    chain = W.transmon_chain(n_sites=3, levels=3, J=0.02, seed=4, omega0_max=0.2, T=5.0, sigma=1.2, N=5, P=8,
                             unitary=True)
    for wl in (chain, W.config(0, N=6)):
        full = oracle.evolve_workload(wl)
        streamed, snaps = oracle.evolve_workload_streamed(wl, snapshots=(1, 3))
        assert np.array_equal(full, streamed)
        for n, v in snaps.items():
            assert np.array_equal(v, oracle.evolve_workload(wl, n_intervals=n))
