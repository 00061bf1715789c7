"""Seeded synthetic workloads for first-order Magnus time evolution.

This module only *creates inputs*: the drift Hamiltonian H0, the control
Hamiltonians H_k, the control signals u^(k)(t) as vectorised callables, the time
grid and the initial state, in the form H(t) = H0 + sum_k u^(k)(t) H_k
(Eq. magnus-generic-ham, Sec. "Magnus Expansion").  It contains none of the
method's arithmetic (no quadrature, no Magnus term, no exponential, no product)
and imports neither the oracle nor the CUDA package, so both sides can consume
the same inputs.

Units: hbar = 1, energies in rad/ns (GHz values times 2*pi), times in ns.
Basis conventions: tensor products put subsystem 0 in the most significant
position (transmon before resonator, chain site 0 first); the lowering operator
acts as b|n> = sqrt(n)|n-1>; basis index 0 is the all-ground state.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# single-mode operators
# ----------------------------------------------------------------------------
def lowering(n: int) -> np.ndarray:
    """Truncated bosonic lowering operator b with b|m> = sqrt(m)|m-1>."""
    b = np.zeros((n, n), dtype=np.complex128)
    for m in range(1, n):
        b[m - 1, m] = math.sqrt(m)
    return b


def embed(op: np.ndarray, site: int, dims: list[int]) -> np.ndarray:
    """Kronecker-embed a single-site operator into the full space (site 0 major)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for j, dj in enumerate(dims):
        out = np.kron(out, op if j == site else np.eye(dj, dtype=np.complex128))
    return out


def number_diag(site: int, dims: list[int]) -> np.ndarray:
    """Occupation number of one site for every basis index (site 0 most significant)."""
    idx = np.arange(int(np.prod(dims)))
    stride = int(np.prod(dims[site + 1:])) if site + 1 < len(dims) else 1
    return ((idx // stride) % dims[site]).astype(np.float64)


# ----------------------------------------------------------------------------
# control signals
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class GaussianTones:
    """u_k(t) = env(t) * sum_j a_{k,j} cos(w_{k,j} t + phi_{k,j}), env a Gaussian.

    env(t) = exp(-(t - t_c)^2 / (2 sigma^2)).  A drive with a single tone per
    channel is the Gaussian-envelope cosine of the circuit-QED workloads; two
    tones per channel give the two-tone drives.
    """
    amp: np.ndarray      # (K, J)
    freq: np.ndarray     # (K, J) rad/ns
    phase: np.ndarray    # (K, J)
    t_center: float
    sigma: float

    @property
    def K(self) -> int:
        return self.amp.shape[0]

    def __call__(self, t) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        env = np.exp(-((t - self.t_center) ** 2) / (2.0 * self.sigma ** 2))
        tt = t[..., None, None]
        tones = self.amp * np.cos(self.freq * tt + self.phase)
        return env[..., None] * tones.sum(axis=-1)


@dataclasses.dataclass
class ConstantDrive:
    """u_k(t) = a_k for all t."""
    amp: np.ndarray  # (K,)

    @property
    def K(self) -> int:
        return self.amp.shape[0]

    def __call__(self, t) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        return np.broadcast_to(self.amp, t.shape + (self.amp.shape[0],)).copy()


@dataclasses.dataclass
class PolynomialDrive:
    """u_k(t) = sum_j coef[k, j] t^j (used to test quadrature exactness)."""
    coef: np.ndarray  # (K, deg+1)

    @property
    def K(self) -> int:
        return self.coef.shape[0]

    def __call__(self, t) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        out = np.zeros(t.shape + (self.coef.shape[0],))
        for k in range(self.coef.shape[0]):
            out[..., k] = np.polynomial.polynomial.polyval(t, self.coef[k])
        return out


@dataclasses.dataclass
class RotatingFrameQubitDrive:
    """The three control signals of the rotating-frame driven qubit.

    H_rot(t) = Omega(t)/4 (sx + cos(2 w t) sx - sin(2 w t) sy)
    (Eq. magnus-rot-ham) written as u_0 sx + u_1 sx + u_2 sy with
    u_0 = Omega/4, u_1 = Omega/4 cos(2wt), u_2 = -Omega/4 sin(2wt); the RWA
    version (Eq. magnus-rwa-ham) keeps u_0 only.  Omega(t) is a Gaussian
    envelope of peak Omega0.
    """
    omega0: float
    w: float
    t_center: float
    sigma: float
    rwa: bool = False

    @property
    def K(self) -> int:
        return 1 if self.rwa else 3

    def envelope(self, t):
        t = np.asarray(t, dtype=np.float64)
        return self.omega0 * np.exp(-((t - self.t_center) ** 2) / (2.0 * self.sigma ** 2))

    def __call__(self, t) -> np.ndarray:
        t = np.asarray(t, dtype=np.float64)
        q = self.envelope(t) / 4.0
        if self.rwa:
            return q[..., None]
        return np.stack([q, q * np.cos(2 * self.w * t), -q * np.sin(2 * self.w * t)], axis=-1)


# ----------------------------------------------------------------------------
# workload record
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    H0: np.ndarray                  # (d, d) complex128, Hermitian
    Hk: np.ndarray                  # (K, d, d) complex128, Hermitian
    drive: Callable                 # t -> (..., K)
    t0: float
    T: float
    N: int                          # Magnus intervals
    P: int                          # quadrature points per interval
    psi0: Optional[np.ndarray]      # (d,) complex128, or None for the full propagator
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.H0.shape[0]

    @property
    def K(self) -> int:
        return self.Hk.shape[0]

    @property
    def dt(self) -> float:
        return self.T / self.N

    @property
    def output(self) -> str:
        return "unitary" if self.psi0 is None else "state"


def basis_state(d: int, index: int = 0) -> np.ndarray:
    psi = np.zeros(d, dtype=np.complex128)
    psi[index] = 1.0
    return psi


# ----------------------------------------------------------------------------
# model families
# ----------------------------------------------------------------------------
def transmon_resonator(nt=3, nr=10, wq=5.0, alpha=-0.25, wr=7.0, g=0.1,
                       omega0=0.05, wd=None, T=50.0, sigma=10.0, N=1000, P=16,
                       phase=0.0, name="transmon_resonator", unitary=False) -> Workload:
    """Transmon (nt levels) (x) resonator (nr Fock levels), one transmon drive.

    H0 = wq n_q + (alpha/2) n_q (n_q - 1) + wr a^dag a + g (b^dag a + b a^dag),
    H_1 = b + b^dag, u(t) = Omega0 exp(-(t-T/2)^2 / 2 sigma^2) cos(wd t + phase).
    Frequencies are given in GHz and converted to rad/ns; wd defaults to wq.
    """
    dims = [nt, nr]
    b = embed(lowering(nt), 0, dims)
    a = embed(lowering(nr), 1, dims)
    nq = number_diag(0, dims)
    na = number_diag(1, dims)
    H0 = np.diag(TWO_PI * (wq * nq + 0.5 * alpha * nq * (nq - 1) + wr * na)).astype(np.complex128)
    H0 = H0 + TWO_PI * g * (b.conj().T @ a + b @ a.conj().T)
    Hk = (b + b.conj().T)[None]
    wd = wq if wd is None else wd
    drive = GaussianTones(amp=np.array([[TWO_PI * omega0]]), freq=np.array([[TWO_PI * wd]]),
                          phase=np.array([[phase]]), t_center=T / 2, sigma=sigma)
    d = nt * nr
    return Workload(name=name, H0=H0, Hk=Hk, drive=drive, t0=0.0, T=T, N=N, P=P,
                    psi0=None if unitary else basis_state(d, 0),
                    meta=dict(nt=nt, nr=nr, wq=wq, alpha=alpha, wr=wr, g=g, omega0=omega0))


def transmon_chain(n_sites=6, levels=3, J=0.01, seed=1, omega0_max=0.05, T=50.0, sigma=10.0,
                   N=2000, P=16, all_to_all=False, J_max=0.02, two_tone=False, unitary=True,
                   name="transmon_chain") -> Workload:
    """Chain (or all-to-all graph) of transmons with exchange coupling.

    H0 = sum_j [w_j n_j + (alpha_j/2) n_j (n_j - 1)] + sum_{(i,j)} J_ij (b_i^dag b_j + b_i b_j^dag)
    with w_j ~ U[4.8, 5.2] GHz and alpha_j ~ U[-0.3, -0.2] GHz.  The chain is open
    with nearest-neighbour J; the all-to-all graph draws J_ij ~ U[0, J_max] GHz for
    every pair i < j.  One drive per site, H_k = b_k + b_k^dag, with a
    Gaussian-envelope cosine at the site frequency (two-tone: also at w_k + alpha_k),
    amplitudes ~ U(0, omega0_max] GHz and phases ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    dims = [levels] * n_sites
    w = rng.uniform(4.8, 5.2, n_sites)
    al = rng.uniform(-0.3, -0.2, n_sites)
    diag = np.zeros(levels ** n_sites)
    for j in range(n_sites):
        nj = number_diag(j, dims)
        diag += w[j] * nj + 0.5 * al[j] * nj * (nj - 1)
    H0 = np.diag(TWO_PI * diag).astype(np.complex128)
    bs = [embed(lowering(levels), j, dims) for j in range(n_sites)]
    pairs = []
    if all_to_all:
        for i in range(n_sites):
            for j in range(i + 1, n_sites):
                pairs.append((i, j, rng.uniform(0.0, J_max)))
    else:
        for i in range(n_sites - 1):
            pairs.append((i, i + 1, J))
    for i, j, Jij in pairs:
        H0 = H0 + TWO_PI * Jij * (bs[i].conj().T @ bs[j] + bs[i] @ bs[j].conj().T)
    Hk = np.stack([b + b.conj().T for b in bs])
    n_tones = 2 if two_tone else 1
    amp = TWO_PI * (omega0_max * (1.0 - rng.uniform(0.0, 1.0, (n_sites, n_tones))))
    freq = np.empty((n_sites, n_tones))
    freq[:, 0] = TWO_PI * w
    if two_tone:
        freq[:, 1] = TWO_PI * (w + al)
    phase = rng.uniform(0.0, TWO_PI, (n_sites, n_tones))
    drive = GaussianTones(amp=amp, freq=freq, phase=phase, t_center=T / 2, sigma=sigma)
    d = levels ** n_sites
    return Workload(name=name, H0=H0, Hk=Hk, drive=drive, t0=0.0, T=T, N=N, P=P,
                    psi0=None if unitary else basis_state(d, 0),
                    meta=dict(w=w, alpha=al, pairs=pairs, seed=seed))


def driven_qubit_rot(omega_ratio=0.33, w_ghz=5.0, T=10.0, N=50, P=16, rwa=False,
                     name="driven_qubit_rot") -> Workload:
    """Strongly driven qubit in the frame rotating at the drive frequency.

    H_rot(t) = Omega(t)/4 (sx + cos(2wt) sx - sin(2wt) sy)  (Eq. magnus-rot-ham),
    or its RWA form Omega(t)/4 sx (Eq. magnus-rwa-ham).  H0 = 0.  The envelope is
    Gaussian with peak Omega0 = omega_ratio * w, centre T/2 and width T/5.
    """
    w = TWO_PI * w_ghz
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    drive = RotatingFrameQubitDrive(omega0=omega_ratio * w, w=w, t_center=T / 2, sigma=T / 5, rwa=rwa)
    Hk = sx[None] if rwa else np.stack([sx, sx, sy])
    return Workload(name=name, H0=np.zeros((2, 2), np.complex128), Hk=Hk, drive=drive,
                    t0=0.0, T=T, N=N, P=P, psi0=basis_state(2, 0),
                    meta=dict(omega0=omega_ratio * w, w=w))


def spin_chain(n=6, omega=1.0, J=0.5, g=0.1, T=25.0, N=200, P=16, seed=0, name="spin_chain") -> Workload:
    """Periodic Ising spin chain with two global controls (Eqs. magnus_drift_ham, magnus_control_ham).

    H_d = 1/2 sum_j w sz_j - J sum_j sz_j sz_{j+1} - g sum_j sz_j sz_{j+2},
    H_c = u_x(t) sum_j sx_j + u_y(t) sum_j sy_j.  The paper's optimal pulse is not
    given, so the controls are seeded sinusoidally modulated Gaussians.
    """
    rng = np.random.default_rng(seed)
    dims = [2] * n
    sz = np.diag(np.array([1.0, -1.0], dtype=np.complex128))
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    Z = [embed(sz, j, dims) for j in range(n)]
    H0 = sum(0.5 * TWO_PI * omega * Z[j] for j in range(n))
    H0 = H0 - TWO_PI * J * sum(Z[j] @ Z[(j + 1) % n] for j in range(n))
    H0 = H0 - TWO_PI * g * sum(Z[j] @ Z[(j + 2) % n] for j in range(n))
    Hk = np.stack([sum(embed(sx, j, dims) for j in range(n)), sum(embed(sy, j, dims) for j in range(n))])
    drive = GaussianTones(amp=TWO_PI * 0.05 * np.ones((2, 1)), freq=TWO_PI * rng.uniform(0, 10, (2, 1)),
                          phase=rng.uniform(0, TWO_PI, (2, 1)), t_center=T / 2, sigma=T / 5)
    return Workload(name=name, H0=H0, Hk=Hk, drive=drive, t0=0.0, T=T, N=N, P=P,
                    psi0=basis_state(2 ** n, 0))


def random_instance(rng: np.random.Generator, name="instance", N_range=(200, 2000),
                    d_range=(16, 256)) -> Workload:
    """One transmon-resonator instance with random size and parameters.

    Transmon levels nt ~ U{2..8} and resonator levels nr ~ U{8..32}, redrawn
    until nt*nr lies in d_range; wq ~ U[4.8,5.2], alpha ~ U[-0.3,-0.2],
    wr ~ U[6.5,7.5], g ~ U[0.05,0.15], Omega0 ~ U(0,0.05] GHz, T = 50 ns,
    N ~ U{N_range}, 16 points per interval, psi0 = |0,0>.
    """
    while True:
        nt = int(rng.integers(2, 9))
        nr = int(rng.integers(8, 33))
        if d_range[0] <= nt * nr <= d_range[1]:
            break
    return transmon_resonator(nt=nt, nr=nr, wq=rng.uniform(4.8, 5.2), alpha=rng.uniform(-0.3, -0.2),
                              wr=rng.uniform(6.5, 7.5), g=rng.uniform(0.05, 0.15),
                              omega0=0.05 * (1.0 - rng.uniform()), T=50.0, sigma=10.0,
                              N=int(rng.integers(N_range[0], N_range[1] + 1)), P=16,
                              phase=rng.uniform(0, TWO_PI), name=name)


# ----------------------------------------------------------------------------
# the five named workloads
# ----------------------------------------------------------------------------
def config(index: int, seed: Optional[int] = None, **overrides) -> Workload:
    """The named synthetic workloads.

    0: transmon(3) (x) resonator(10), d = 30, 1000 intervals, 16 points, psi0 = |0,0>.
    1: chain of 6 three-level transmons, d = 729, 2000 intervals, 16 points, full U.
    3: 4 transmons x 8 levels, d = 4096, all-to-all, two-tone drives, 500 intervals,
       8 points, full U.
    The batched (512 uneven instances) and serving workloads are built by
    `uneven_batch` and `serving_stream`.
    """
    seed = index if seed is None else seed
    if index == 0:
        return transmon_resonator(name="cfg0_transmon_resonator_d30", **overrides)
    if index == 1:
        kw = dict(n_sites=6, levels=3, J=0.01, seed=seed, N=2000, P=16, name="cfg1_transmon_chain_d729")
        kw.update(overrides)
        return transmon_chain(**kw)
    if index == 3:
        kw = dict(n_sites=4, levels=8, seed=seed, N=500, P=8, all_to_all=True, J_max=0.02,
                  two_tone=True, name="cfg3_all_to_all_d4096")
        kw.update(overrides)
        return transmon_chain(**kw)
    raise ValueError(f"no single-job workload {index}")


def uneven_batch(n_jobs=512, seed=2, **kw) -> list[Workload]:
    """512 independent transmon-resonator instances of uneven size and length."""
    rng = np.random.default_rng(seed)
    return [random_instance(rng, name=f"cfg2_job{i}", **kw) for i in range(n_jobs)]


def serving_stream(rate_hz=200.0, duration_s=60.0, seed=4, d_min=32, d_max=2048):
    """Poisson arrivals of mixed jobs (dimension log-uniform in [d_min, d_max]).

    Returns a list of (arrival_time_s, job_spec) with job_spec a dict naming the
    family, the realised dimension (largest family member not above the draw),
    the interval count N ~ U{100..5000} (dt = 0.05 ns) and the output kind.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        draw = math.exp(rng.uniform(math.log(d_min), math.log(d_max)))
        fam = "chain3" if rng.uniform() < 0.5 else "transmon_resonator"
        if fam == "chain3":
            n = max(1, int(math.floor(math.log(draw) / math.log(3) + 1e-12)))
            dim = 3 ** n
        else:
            nt = int(rng.integers(2, 9))
            nr = max(1, int(draw // nt))
            dim = nt * nr
        N = int(rng.integers(100, 5001))
        out.append((t, dict(family=fam, d=dim, N=N, dt=0.05,
                            output="unitary" if rng.uniform() < 0.5 else "state",
                            seed=int(rng.integers(0, 2**31 - 1)))))
    return out


def serving_job(spec: dict) -> Workload:
    """The Workload of one request of `serving_stream`: a 3-level transmon chain of
    log3(d) sites or a transmon-resonator with nt x nr = d, N intervals of dt, one
    drive per transmon, parameters drawn from the request's seed."""
    rng = np.random.default_rng(spec["seed"])
    N, dt = spec["N"], spec["dt"]
    T = N * dt
    state = spec["output"] == "state"
    if spec["family"] == "chain3":
        n = int(round(math.log(spec["d"]) / math.log(3)))
        return transmon_chain(n_sites=n, levels=3, J=0.01, seed=int(rng.integers(0, 2**31 - 1)), T=T,
                              sigma=T / 5, N=N, P=16, unitary=not state, name=f"chain3_d{spec['d']}")
    d = spec["d"]
    nt = next(k for k in range(8, 1, -1) if d % k == 0) if d > 1 else 1
    nr = d // nt
    return transmon_resonator(nt=nt, nr=nr, wq=rng.uniform(4.8, 5.2), alpha=rng.uniform(-0.3, -0.2),
                              wr=rng.uniform(6.5, 7.5), g=rng.uniform(0.05, 0.15),
                              omega0=0.05 * (1.0 - rng.uniform()), T=T, sigma=T / 5, N=N, P=16,
                              phase=rng.uniform(0, TWO_PI), name=f"tr_d{d}", unitary=not state)
