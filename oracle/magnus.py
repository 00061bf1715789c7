"""Plain CPU FP64 oracle for first-order Magnus time evolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; it is
used by the test-suite, by `__graft_entry__.smoke()` and by the CPU baseline
leg of `bench.py`.  It shares no code with the CUDA path.

What it computes (Sec. "Time Coarse-Graining Hamiltonians", subsection
"Magnus Expansion"):

* H(t) = H0 + sum_k u^(k)(t) H_k                          (Eq. magnus-generic-ham)
* c_{k,n} = integral of u^(k) over [t_n, t_n + dt]        (Eq. magnus-first-order-coeff),
  by P-point Gauss-Legendre quadrature with nodes t_{n,p} = t_n + (1 + x_p) dt / 2.
* Hbar_n = dt H0 + sum_k c_{k,n} H_k                     (Eq. magnus-first-order-term),
  the first-order Magnus term of interval n; it is the *integrated* exponent
  (units of phase), as the first line of Eq. magnus-avg integrates H without
  a 1/t factor.
* U_n = exp(-i Hbar_n) (hbar = 1), evaluated through the Hermitian
  eigendecomposition Hbar_n - tau I = V diag(lambda) V^dagger with
  tau = tr(Hbar_n)/d:  U_n = e^{-i tau} V diag(e^{-i lambda}) V^dagger.
* psi(T) = U_{N-1} ... U_0 psi0  or  U(T) = U_{N-1} ... U_0, later intervals
  multiplying on the left, one plain product per interval.

The second-order term of Eq. magnus-avg is provided separately
(`second_order_term`) for the tests of the commutator extension; the paper's
package uses the first-order term only (Sec. "Magnus Expansion").
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# time grid and quadrature  (Eq. magnus-first-order-coeff)
# ----------------------------------------------------------------------------
def gauss_legendre(P: int):
    """P-point Gauss-Legendre nodes x_p and weights w_p on [-1, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(P)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def interval_starts(t0: float, dt: float, N: int) -> np.ndarray:
    """Uniform Magnus intervals: t_n = t0 + n dt, n = 0..N-1."""
    return t0 + dt * np.arange(N, dtype=np.float64)


def node_times(t0: float, dt: float, N: int, x: np.ndarray) -> np.ndarray:
    """Quadrature nodes of every interval, shape (N, P): t_n + (1 + x_p) dt / 2."""
    tn = interval_starts(t0, dt, N)
    return tn[:, None] + (1.0 + x[None, :]) * (0.5 * dt)


def drive_coefficients(samples: np.ndarray, w: np.ndarray, dt: float) -> np.ndarray:
    """c[n, k] = (dt/2) sum_p w_p u^(k)(t_{n,p})  (Eq. magnus-first-order-coeff).

    samples: (N, P, K) values of the control signals at the nodes.
    """
    samples = np.asarray(samples, dtype=np.float64)
    N, P, K = samples.shape
    c = np.zeros((N, K), dtype=np.float64)
    for n in range(N):
        for k in range(K):
            acc = 0.0
            for p in range(P):
                acc += w[p] * samples[n, p, k]
            c[n, k] = 0.5 * dt * acc
    return c


# ----------------------------------------------------------------------------
# Magnus terms  (Eqs. magnus-first-order-term, magnus-avg)
# ----------------------------------------------------------------------------
def first_order_term(H0: np.ndarray, Hk: np.ndarray, c_n: np.ndarray, dt: float) -> np.ndarray:
    """Hbar_n = dt H0 + sum_k c_{k,n} H_k for one interval (Eq. magnus-first-order-term)."""
    out = dt * np.asarray(H0, dtype=np.complex128)
    for k in range(Hk.shape[0]):
        out = out + c_n[k] * Hk[k]
    return out


def second_order_term(Hfun, t_a: float, t_b: float, P: int) -> np.ndarray:
    """Second-order Magnus term of Eq. magnus-avg over [t_a, t_b]:

        Hbar^(2) = -(i/2) int_{t_a}^{t_b} dt1 int_{t_a}^{t1} dt2 [H(t1), H(t2)],

    by nested P-point Gauss-Legendre quadrature (outer over [t_a, t_b], inner
    over [t_a, t1]).  Hfun(t) returns the d x d matrix H(t).
    """
    x, w = gauss_legendre(P)
    half = 0.5 * (t_b - t_a)
    acc = None
    for p in range(P):
        t1 = t_a + (1.0 + x[p]) * half
        H1 = Hfun(t1)
        inner_half = 0.5 * (t1 - t_a)
        inner = np.zeros_like(H1)
        for q in range(P):
            t2 = t_a + (1.0 + x[q]) * inner_half
            inner = inner + w[q] * inner_half * Hfun(t2)
        term = w[p] * half * (H1 @ inner - inner @ H1)
        acc = term if acc is None else acc + term
    return -0.5j * acc


# ----------------------------------------------------------------------------
# exponential
# ----------------------------------------------------------------------------
def expm_minus_i(Hbar: np.ndarray) -> np.ndarray:
    """exp(-i Hbar) for Hermitian Hbar via eigendecomposition with an exact trace shift."""
    Hbar = np.asarray(Hbar, dtype=np.complex128)
    d = Hbar.shape[0]
    tau = float(np.real(np.trace(Hbar))) / d
    Hs = Hbar - tau * np.eye(d)
    Hs = 0.5 * (Hs + Hs.conj().T)          # exact Hermitian part (input is Hermitian)
    lam, V = np.linalg.eigh(Hs)
    return np.exp(-1j * tau) * ((V * np.exp(-1j * lam)[None, :]) @ V.conj().T)


# ----------------------------------------------------------------------------
# full evolution
# ----------------------------------------------------------------------------
def interval_propagators(H0, Hk, samples, w, dt):
    """U_n = exp(-i Hbar_n) for n = 0..N-1; returns (U (N,d,d), Hbar (N,d,d), c (N,K))."""
    c = drive_coefficients(samples, w, dt)
    N = c.shape[0]
    d = H0.shape[0]
    Hbar = np.empty((N, d, d), dtype=np.complex128)
    U = np.empty((N, d, d), dtype=np.complex128)
    for n in range(N):
        Hbar[n] = first_order_term(H0, Hk, c[n], dt)
        U[n] = expm_minus_i(Hbar[n])
    return U, Hbar, c


def propagate_state(U: np.ndarray, psi0: np.ndarray, trajectory: bool = False):
    """psi_{n+1} = U_n psi_n, n = 0..N-1 (stroboscopic states at interval ends)."""
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    traj = [psi.copy()] if trajectory else None
    for n in range(U.shape[0]):
        psi = U[n] @ psi
        if trajectory:
            traj.append(psi.copy())
    return (psi, np.array(traj)) if trajectory else psi


def propagate_unitary(U: np.ndarray) -> np.ndarray:
    """U(T) = U_{N-1} ... U_1 U_0 (later intervals on the left)."""
    d = U.shape[1]
    acc = np.eye(d, dtype=np.complex128)
    for n in range(U.shape[0]):
        acc = U[n] @ acc
    return acc


def magnus_evolve(H0, Hk, samples, w, dt, psi0=None):
    """First-order Magnus evolution: psi(T) if psi0 is given, else the full U(T)."""
    U, _, _ = interval_propagators(H0, Hk, samples, w, dt)
    if psi0 is None:
        return propagate_unitary(U)
    return propagate_state(U, psi0)


def evolve_workload(wl, n_intervals=None, return_parts=False):
    """Run the oracle on a `workloads.Workload` (optionally only its first intervals)."""
    x, w = gauss_legendre(wl.P)
    N = wl.N if n_intervals is None else int(n_intervals)
    t = node_times(wl.t0, wl.dt, N, x)
    samples = wl.drive(t)
    U, Hbar, c = interval_propagators(wl.H0, wl.Hk, samples, w, wl.dt)
    out = propagate_unitary(U) if wl.psi0 is None else propagate_state(U, wl.psi0)
    if return_parts:
        return out, dict(U=U, Hbar=Hbar, c=c, samples=samples, x=x, w=w)
    return out


def evolve_workload_streamed(wl, n_intervals=None, snapshots=()):
    """The result of `evolve_workload`, formed one interval at a time.

    For every n: c_{k,n} (Eq. magnus-first-order-coeff), Hbar_n
    (Eq. magnus-first-order-term), U_n = exp(-i Hbar_n), and the running
    product (U_n @ U or U_n @ psi) -- the same steps in the same order as
    `evolve_workload`, but no interval's matrices are kept, so memory stays at a
    few d x d matrices for the large workloads (d = 4096).  Returns the final
    psi or U, and a dict {n: value after n intervals} for every n in `snapshots`.
    """
    x, w = gauss_legendre(wl.P)
    N = wl.N if n_intervals is None else int(n_intervals)
    d = wl.H0.shape[0]
    acc = np.eye(d, dtype=np.complex128) if wl.psi0 is None else np.asarray(wl.psi0, np.complex128).copy()
    snaps = {}
    for n in range(N):
        t = node_times(wl.t0 + n * wl.dt, wl.dt, 1, x)
        c = drive_coefficients(wl.drive(t), w, wl.dt)[0]
        Un = expm_minus_i(first_order_term(wl.H0, wl.Hk, c, wl.dt))
        acc = Un @ acc
        if n + 1 in snapshots:
            snaps[n + 1] = acc.copy()
    return acc, snaps


def interval_propagators_second_order(H0, Hk, drive, t0, dt, N, P):
    """U_n = exp(-i (Hbar^(1)_n + Hbar^(2)_n)) with both Magnus terms of Eq. magnus-avg over
    every interval: Hbar^(1) by P-point Gauss-Legendre quadrature of the drive, Hbar^(2) by
    nested P-point quadrature of [H(t1), H(t2)] (`second_order_term`).  `drive(t)` -> (..., K)."""
    x, w = gauss_legendre(P)
    d = H0.shape[0]
    U = np.empty((N, d, d), dtype=np.complex128)

    def Hfun(t):
        u = drive(np.array([t]))[0]
        out = np.asarray(H0, dtype=np.complex128).copy()
        for k in range(Hk.shape[0]):
            out = out + u[k] * Hk[k]
        return out

    c = drive_coefficients(drive(node_times(t0, dt, N, x)), w, dt)
    for n in range(N):
        a = t0 + n * dt
        H1 = first_order_term(H0, Hk, c[n], dt)
        H2 = second_order_term(Hfun, a, a + dt, P)
        U[n] = expm_minus_i(H1 + 0.5 * (H2 + H2.conj().T))
    return U


def evolve_workload_second_order(wl, n_intervals=None):
    """Second-order Magnus evolution of a `workloads.Workload`."""
    N = wl.N if n_intervals is None else int(n_intervals)
    U = interval_propagators_second_order(wl.H0, wl.Hk, wl.drive, wl.t0, wl.dt, N, wl.P)
    return propagate_unitary(U) if wl.psi0 is None else propagate_state(U, wl.psi0)


# ----------------------------------------------------------------------------
# invariants reported next to a result
# ----------------------------------------------------------------------------
def unitarity_defect(U: np.ndarray) -> float:
    """max |U^dagger U - I| (elementwise)."""
    d = U.shape[-1]
    return float(np.max(np.abs(U.conj().T @ U - np.eye(d))))


def norm_defect(psi: np.ndarray) -> float:
    return float(abs(np.linalg.norm(psi) - 1.0))
