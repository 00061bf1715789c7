"""A NumPy model of the split-precision arithmetic, for predicting errors on the CPU.

TEST INFRASTRUCTURE ONLY: it imports nothing from the library and the library
imports nothing from it.  It restates, in float64/float32 NumPy, the arithmetic
the split-precision mode is designed to perform, so that the error of each mode
on each workload can be predicted without a GPU and set beside what the GPU
measures.  It models, it does not reproduce bit for bit:

* operands: a complex d x d matrix A is cut row by row (B column by column).
  With every |Re|, |Im| of row i below 2^E_i, an entry a becomes the integer
  X = round(a 2^(beta L - E_i - 1)) (half away from zero), written in balanced
  base 2^beta, X = sum_{s<L} q_s 2^(beta (L - 1 - s)), so that
  a ~ 2^(E_i + 1 - beta) sum_s q_s 2^(-beta s); every q_s 2^(-beta s) is exact
  in BF16.  A double-float input (hi + lo FP32) is cut as
  round(hi 2^sh) + round(lo 2^sh), with E_i taken from the hi parts.
* beta: the largest beta <= 8 with 2^(2 beta - 1) 2d <= 2^24.
* product: the 4M real embedding [Cr | Ci] = [Ar | Ai] [[Br, Bi], [-Bi, Br]]
  with K = 2 roundup(d, 32).  Digit pairs (s, t) with s + t <= L - 1 are summed
  into four FP32 accumulators by level s + t = 0, 1, 2, >= 3; each pair's
  16-deep block of K is summed exactly and added to its accumulator with one
  FP32 rounding, toward zero by default (published studies of NVIDIA tensor
  cores, e.g. Fasi, Higham, Mikaitis and Pranesh, PeerJ Comput. Sci. 7 (2021)
  e330, report truncating accumulation), or to nearest.  The order of the
  updates inside the tensor core is not modelled.
* epilogue: C = 2^(E_i + F_j + 2 - 2 beta) (g0 + g1 + g2 + g3) plus addends
  coef * S (coef rounded to double-float) and a diagonal, stored as
  double-float.
* the exponential: X = -i 2^-s W stored as double-float, Paterson-Stockmeyer
  Taylor evaluation (degree m, block p) with the products above, s squarings,
  then the exact phase e^(-i tau).  The degree and squaring count minimise
  products + s under the remainder bound sum_{j>m} theta^j / j! <= u theta with
  u = max(2^-53, 2^(-beta L)); as on the library's split path, degree 18 in
  five products (A2, A3, A6, A9 = B1 B5 + B4, T = B2 + (B3 + A9) A9, with the
  coefficients of csrc/taylor18.h) is offered beside Paterson-Stockmeyer.
* propagation of a state: each U_n read back to FP64, psi carried in FP64.
"""
from __future__ import annotations

import math

import numpy as np

KBLOCK = 16        # depth of one tensor-core step along K


# ----------------------------------------------------------------------------
# double-float storage: a complex matrix as hi + lo, both complex64
# ----------------------------------------------------------------------------
def df_round(x):
    """Store a complex128 array as double-float: (hi, lo) complex64 with hi + lo ~ x."""
    x = np.asarray(x, dtype=np.complex128)
    hi = x.astype(np.complex64)
    lo = (x - hi.astype(np.complex128)).astype(np.complex64)
    return hi, lo


def df_value(m):
    """The complex128 value of a double-float (hi, lo), or of a plain complex128 array."""
    if isinstance(m, tuple):
        return m[0].astype(np.complex128) + m[1].astype(np.complex128)
    return np.asarray(m, dtype=np.complex128)


def split_beta(d):
    """Digit width: the largest beta <= 8 with 2^(2 beta - 1) 2d <= 2^24."""
    return max(b for b in range(2, 9) if 2.0 ** (2 * b - 1) * 2 * d <= 2.0 ** 24)


# ----------------------------------------------------------------------------
# digits
# ----------------------------------------------------------------------------
def _exp_bound(x):
    """E with |x| < 2^E for every nonzero x (the frexp exponent); zeros give a large negative."""
    _, e = np.frexp(x)
    return np.where(x == 0, -(1 << 29), e).astype(np.int64)


def _fixed_point(x, sh):
    """round(x 2^sh), half away from zero, as int64 (x float32 or float64, sh broadcastable)."""
    y = np.abs(x.astype(np.float64)) * np.exp2(sh.astype(np.float64))
    f = np.floor(y)
    X = f + (y - f >= 0.5)
    return (np.sign(x).astype(np.int64) * X.astype(np.int64))


def _balanced_digits(X, L, beta):
    """q[0..L-1] with X = sum_s q_s 2^(beta (L - 1 - s)), |q_s| <= 2^(beta - 1)."""
    half, mask = 1 << (beta - 1), (1 << beta) - 1
    q = np.empty((L,) + X.shape, dtype=np.int64)
    for s in range(L - 1, 0, -1):
        r = ((X + half) & mask) - half
        q[s] = r
        X = (X - r) >> beta
    q[0] = X
    return q


def digits(M, L, beta, axis):
    """Digits of the operand M (complex128 or double-float) with one exponent per row
    (axis = 1, the A operand) or per column (axis = 0, the B operand).

    Returns (vr, vi, E): vr/vi of shape (L,) + M.shape hold q_s 2^(-beta s) of the real
    and imaginary parts, E the exponent of every row (or column)."""
    assert beta * L <= 62, "the model keeps X in int64"
    if isinstance(M, tuple):
        parts = [(M[0].real, M[1].real), (M[0].imag, M[1].imag)]
        lead = M[0]
    else:
        M = np.asarray(M, dtype=np.complex128)
        parts = [(M.real, None), (M.imag, None)]
        lead = M
    E = np.maximum(_exp_bound(lead.real), _exp_bound(lead.imag)).max(axis=axis + lead.ndim - 2,
                                                                     keepdims=True)
    E = np.where(E < -(1 << 28), 0, E)
    sh = beta * L - E - 1
    out = []
    for hi, lo in parts:
        X = _fixed_point(hi, sh)
        if lo is not None:
            X = X + _fixed_point(lo, sh)
        q = _balanced_digits(X, L, beta)
        scale = np.exp2(-beta * np.arange(L, dtype=np.float64)).reshape((L,) + (1,) * X.ndim)
        out.append(q.astype(np.float64) * scale)
    return out[0], out[1], np.squeeze(E, axis=axis + lead.ndim - 2)


# ----------------------------------------------------------------------------
# the split product
# ----------------------------------------------------------------------------
def _level(s, t, groups=4):
    return min(s + t, groups - 1)


def _to_f32(x, mode):
    """x (float64) to float32, to nearest or toward zero."""
    f = x.astype(np.float32)
    if mode == "nearest":
        return f
    # where rounding to nearest went past x (away from zero), step one unit back: in
    # sign-magnitude bits that is the integer minus one, for either sign
    over = (f.astype(np.float64) - x) * x > 0
    bits = f.view(np.int32)
    bits -= over
    return f


def split_product(A, B, L, beta=None, addends=(), diag=0.0, accumulate="zero", groups=4):
    """C = A B (+ sum coef S + diag I) through L-digit split arithmetic, stored as double-float.

    A, B: (..., d, d) complex128 or double-float; addends: (coef, S) pairs with S of
    the same kind; accumulate: rounding of each FP32 accumulator update, "nearest"
    or "zero" (truncation); groups: number of level accumulators (the last one takes
    every level from groups - 1 up).  Returns (hi, lo)."""
    Av, Bv = (A[0] if isinstance(A, tuple) else A), (B[0] if isinstance(B, tuple) else B)
    d = Av.shape[-1]
    beta = split_beta(d) if beta is None else beta
    ar, ai, Ea = digits(A, L, beta, axis=1)
    br, bi, Fb = digits(B, L, beta, axis=0)
    Kh = -(-d // 32) * 32
    batch = Av.shape[:-2]
    # real embedding, K padded to 2 Kh: A_s = [Ar | 0 | Ai | 0], B_s = [[Br, Bi]; 0; [-Bi, Br]; 0]
    Ae = np.zeros((L,) + batch + (d, 2 * Kh))
    Ae[..., :d] = ar
    Ae[..., Kh:Kh + d] = ai
    Be = np.zeros((L,) + batch + (2 * Kh, 2 * d))
    Be[..., :d, :d] = br
    Be[..., :d, d:] = bi
    Be[..., Kh:Kh + d, :d] = -bi
    Be[..., Kh:Kh + d, d:] = br
    nblk = 2 * Kh // KBLOCK
    # blocks of K as a stack dimension: (L, ..., nblk, d, KBLOCK) and (L, ..., nblk, KBLOCK, 2d)
    Ab = np.moveaxis(Ae.reshape((L,) + batch + (d, nblk, KBLOCK)), -2, -3)
    Bb = Be.reshape((L,) + batch + (nblk, KBLOCK, 2 * d))
    g = np.zeros((groups,) + batch + (d, 2 * d), dtype=np.float32)
    # bound the partial products held at once to about 2^25 doubles
    step = max(1, (1 << 25) // max(1, int(np.prod(batch, dtype=np.int64)) * d * 2 * d))
    for b0 in range(0, nblk, step):
        sl = slice(b0, min(nblk, b0 + step))
        for s in range(L):
            for t in range(L - s):
                part = np.matmul(Ab[s][..., sl, :, :], Bb[t][..., sl, :, :])   # exact 16-deep sums
                lv = _level(s, t, groups)
                for k in range(part.shape[-3]):
                    g[lv] = _to_f32(g[lv].astype(np.float64) + part[..., k, :, :], accumulate)
    tot = g.astype(np.float64).sum(axis=0)
    scale = np.exp2((Ea[..., :, None] + Fb[..., None, :] + 2 - 2 * beta).astype(np.float64))
    C = (tot[..., :d] + 1j * tot[..., d:]) * scale
    for coef, S in addends:
        c_hi = np.float32(coef)
        c_df = float(c_hi) + float(np.float32(coef - float(c_hi)))
        C = C + c_df * df_value(S)
    if diag != 0.0:
        d_hi = np.float32(diag)
        C = C + (float(d_hi) + float(np.float32(diag - float(d_hi)))) * np.eye(d)
    return df_round(C)


# ----------------------------------------------------------------------------
# the alternative the design rejects: three-pass TF32 products ("3xTF32")
# ----------------------------------------------------------------------------
TF32_KBLOCK = 8    # depth of one TF32 tensor-core step along K


def tf32_round(x):
    """float32 values rounded to TF32 (10 explicit mantissa bits), to nearest even."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0xFFF + ((b >> 13) & 1)) & ~np.uint64(0x1FFF)
    return b.astype(np.uint32).view(np.float32)


def tf32x3_product(A, B, accumulate="zero"):
    """C = A B as three TF32 passes, hi hi + hi lo + lo hi, with a = hi + lo, hi = tf32(a),
    lo = tf32(a - hi) (both from the FP32 value of a), in the 4M real embedding; each
    8-deep block of K of each pass is summed exactly and added to ONE FP32 accumulator
    with one rounding.  Returns complex128 (the FP32 accumulator's value)."""
    A, B = df_value(A), df_value(B)
    d = A.shape[-1]
    Ae = np.concatenate([A.real, A.imag], axis=-1).astype(np.float32)                  # (d, 2d)
    Be = np.block([[B.real, B.imag], [-B.imag, B.real]]).astype(np.float32)            # (2d, 2d)
    ah = tf32_round(Ae)
    al = tf32_round(Ae - ah)
    bh = tf32_round(Be)
    bl = tf32_round(Be - bh)
    K = 2 * d
    acc = np.zeros((d, 2 * d), dtype=np.float32)
    for k0 in range(0, K, TF32_KBLOCK):
        k1 = min(K, k0 + TF32_KBLOCK)
        for a_, b_ in ((ah, bh), (ah, bl), (al, bh)):
            part = a_[:, k0:k1].astype(np.float64) @ b_[k0:k1, :].astype(np.float64)
            acc = _to_f32(acc.astype(np.float64) + part, accumulate)
    acc = acc.astype(np.float64)
    return acc[:, :d] + 1j * acc[:, d:]


def expm_tf32x3(W, tau=None):
    """exp(-i W) for one Hermitian W with every product a 3xTF32 product: Paterson-Stockmeyer
    at the (m, s) of unit roundoff 2^-22 (what three TF32 passes carry), s squarings."""
    W = np.asarray(W, dtype=np.complex128)
    d = W.shape[-1]
    m, p, s = taylor_choice(float(np.abs(W).sum(axis=-2).max()), 2.0 ** -22, False)
    X = (-1j * W * 2.0 ** -s).astype(np.complex64).astype(np.complex128)
    a = [1.0 / math.factorial(j) if j <= m else 0.0 for j in range(m + p + 1)]
    Pw = {1: X}
    for j in range(2, p + 1):
        Pw[j] = tf32x3_product(Pw[j - 1], X)
    q, r = divmod(m, p)
    top = q - 1 if r == 0 else q
    R = a[top * p] * np.eye(d) + sum(a[top * p + j] * Pw[j] for j in range(1, p))
    if r == 0:
        R = R + a[m] * Pw[p]
    for i in range(top - 1, -1, -1):
        R = tf32x3_product(R, Pw[p]) + sum(a[i * p + j] * Pw[j] for j in range(1, p)) + a[i * p] * np.eye(d)
        R = R.astype(np.complex64).astype(np.complex128)
    for _ in range(s):
        R = tf32x3_product(R, R)
    if tau is not None:
        R = np.exp(-1j * tau) * R
    return R


# ----------------------------------------------------------------------------
# the exponential
# ----------------------------------------------------------------------------
PS_DEGREES = [(2, 2), (4, 2), (6, 3), (9, 3), (12, 4), (16, 4)]   # (m, block p)


def _ps_products(m, p):
    """Matrix products of Paterson-Stockmeyer at degree m with block p: p - 1 powers and
    one per Horner step."""
    q, r = divmod(m, p)
    top = q - 1 if r == 0 else q
    return (p - 1) + top


def theta(m, u):
    """Largest theta with sum_{j>m} theta^j / j! <= u theta (bisection)."""
    def ratio(th):
        return math.fsum(math.exp(j * math.log(th) - math.lgamma(j + 1)) for j in range(m + 1, m + 81)) / th
    lo, hi = 1e-9, 40.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ratio(mid) <= u else (lo, mid)
    return lo


def taylor18_coefficients():
    """The 24 coefficients of the degree-18 five-product scheme as the library stores them
    (csrc/taylor18.h): B1 on I, A, A2, A3, then B5, B4, B3, B2 on I, A, A2, A3, A6."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2411_09982_gb300", "csrc", "taylor18.h")
    text = open(path).read()
    body = text[text.index("{", text.index("kTaylor18")) + 1:text.index("};")]
    vals = [float(v) for v in re.findall(r"(-?[0-9][0-9.eE+-]*)\s*,", body)]
    assert len(vals) == 24
    return vals


def taylor_choice(norm1, u, allow18=False):
    """(m, p, s) minimising products + s with norm1 / 2^s <= theta_m over the
    Paterson-Stockmeyer degrees and, when allowed, degree 18 in five products (p = 0);
    ties go to fewer squarings, then to the lower degree."""
    best = None
    for m, p in PS_DEGREES + ([(18, 0)] if allow18 else []):
        th = theta(m, u)
        s = 0 if norm1 <= th else math.ceil(math.log2(norm1 / th))
        while norm1 * 2.0 ** -s > th:
            s += 1
        while s > 0 and norm1 * 2.0 ** -(s - 1) <= th:
            s -= 1
        cost = (5 if p == 0 else _ps_products(m, p)) + s
        if best is None or cost < best[0] or (cost == best[0] and s < best[3]):
            best = (cost, m, p, s)
    return best[1:]


def _taylor18(X, L, beta):
    """sum_{k<=18} X^k / k! in five modelled products: A2, A3, A6, A9 = B1 B5 + B4 and
    T = B2 + (B3 + A9) A9, the B's combined in FP64 from double-float inputs."""
    k = taylor18_coefficients()
    d = X[0].shape[-1]
    eye = np.eye(d)
    A2 = split_product(X, X, L, beta)
    A3 = split_product(A2, X, L, beta)
    A6 = split_product(A3, A3, L, beta)
    P = [df_value(M) for M in (X, A2, A3, A6)]
    B1 = df_round(k[0] * eye + k[1] * P[0] + k[2] * P[1] + k[3] * P[2])
    B5, B4, B3, B2 = (df_round(k[q] * eye + sum(k[q + 1 + j] * P[j] for j in range(4))) for q in (4, 9, 14, 19))
    A9 = split_product(B1, B5, L, beta, addends=[(1.0, B4)])
    Q = df_round(df_value(B3) + df_value(A9))
    return split_product(Q, A9, L, beta, addends=[(1.0, B2)])


def expm_split(W, L, tau=None, allow18=True):
    """exp(-i W) (times e^(-i tau) if tau is given) for a batch of Hermitian W (b, d, d),
    through the modelled split arithmetic; one (m, s) for the batch from its largest
    FP64 1-norm, with the degree-18 scheme offered as on the library's split path.
    Returns the double-float result and (m, s)."""
    W = np.asarray(W, dtype=np.complex128)
    d = W.shape[-1]
    beta = split_beta(d)
    u = max(2.0 ** -53, 2.0 ** (-beta * L))
    norm1 = float(np.abs(W).sum(axis=-2).max())
    m, p, s = taylor_choice(norm1, u, allow18)
    X = df_round(-1j * W * 2.0 ** -s)
    if p == 0:
        R = _taylor18(X, L, beta)
        for _ in range(s):
            R = split_product(R, R, L, beta)
        if tau is not None:
            R = df_round(np.exp(-1j * np.asarray(tau))[..., None, None] * df_value(R))
        return R, (m, s)
    a = [1.0 / math.factorial(j) if j <= m else 0.0 for j in range(m + p + 1)]
    Pw = {1: X}
    for j in range(2, p + 1):
        Pw[j] = split_product(Pw[j - 1], X, L, beta)
    q, r = divmod(m, p)
    top = q - 1 if r == 0 else q
    eye = np.eye(d)
    R = a[top * p] * eye + sum(a[top * p + j] * df_value(Pw[j]) for j in range(1, p))
    if r == 0:
        R = R + a[m] * df_value(Pw[p])
    R = df_round(R)
    for i in range(top - 1, -1, -1):
        R = split_product(R, Pw[p], L, beta, addends=[(a[i * p + j], Pw[j]) for j in range(1, p)],
                          diag=a[i * p])
    for _ in range(s):
        R = split_product(R, R, L, beta)
    if tau is not None:
        R = df_round(np.exp(-1j * np.asarray(tau))[..., None, None] * df_value(R))
    return R, (m, s)


# ----------------------------------------------------------------------------
# a whole evolution of a state
# ----------------------------------------------------------------------------
def evolve_state_split(Hbar, psi0, L, chunk=256, allow18=True):
    """psi(T) = U_{N-1} ... U_0 psi0 with U_n = e^(-i tau_n) exp(-i (Hbar_n - tau_n I))
    from the modelled split exponential, in batches of `chunk` intervals (one (m, s)
    per batch), U_n read back to FP64 and psi carried in FP64.  Returns psi and the
    (m, s) of every batch."""
    Hbar = np.asarray(Hbar, dtype=np.complex128)
    d = Hbar.shape[-1]
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    choices = []
    for n0 in range(0, Hbar.shape[0], chunk):
        H = Hbar[n0:n0 + chunk]
        tau = np.real(np.trace(H, axis1=-2, axis2=-1)) / d
        U, ms = expm_split(H - tau[:, None, None] * np.eye(d), L, tau, allow18)
        choices.append(ms)
        U = df_value(U)
        for n in range(U.shape[0]):
            psi = U[n] @ psi
    return psi, choices


# ----------------------------------------------------------------------------
# command line: predicted error of a state workload against the FP64 oracle
# ----------------------------------------------------------------------------
def main(argv=None):
    """python tests/precision_model.py [--config 0 | --batch-job I] [--slices L]
    [--intervals N] [--no-taylor18]: the modelled split-precision psi(T) against the
    oracle's, max-abs error printed with the (m, s) choices."""
    import argparse
    import os
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import workloads as W
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--config", type=int, default=0, help="single-job state workload (0)")
    ap.add_argument("--batch-job", type=int, default=None, help="job I of the 512-instance uneven batch instead")
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--intervals", type=int, default=None, help="first N intervals only")
    ap.add_argument("--chunk", type=int, default=64, help="intervals per modelled batch (one (m, s) each)")
    ap.add_argument("--no-taylor18", action="store_true", help="Paterson-Stockmeyer only")
    a = ap.parse_args(argv)
    wl = W.uneven_batch()[a.batch_job] if a.batch_job is not None else W.config(a.config)
    if wl.psi0 is None:
        raise SystemExit(f"{wl.name} has no initial state: the model evolves states only")
    t = time.time()
    ref, parts = oracle.evolve_workload(wl, n_intervals=a.intervals, return_parts=True)
    psi, ms = evolve_state_split(parts["Hbar"], wl.psi0, a.slices, chunk=a.chunk, allow18=not a.no_taylor18)
    print(f"{wl.name}: d = {wl.d}, {parts['Hbar'].shape[0]} intervals, L = {a.slices}, "
          f"(m, s) = {sorted(set(ms))}: max |psi_model - psi_oracle| = {np.abs(psi - ref).max():.3e} "
          f"({time.time() - t:.1f} s)")


if __name__ == "__main__":
    main()
