// Action-based state propagation with sparse operators.
//
// For state outputs the product U_{N-1} ... U_0 psi0 never needs the matrices
// U_n = exp(-i Hbar_n), Hbar_n = dt H0 + sum_k c_{k,n} H_k (Eq.
// magnus-first-order-term): each interval applies the exponential to the state.
//
// Spectral interval.  Gershgorin's discs of Hbar_n put its (real) spectrum in
// [c_n - rho_n, c_n + rho_n].  With X = (Hbar_n - c_n I) / rho_n, whose
// spectrum lies in [-1, 1], and s_n sub-steps of z = rho_n / s_n <= 20,
//
//   exp(-i Hbar_n) = e^{-i c_n} [ J_0(z) I + 2 sum_{k>=1} (-i)^k J_k(z) T_k(X) ]^{s_n}
//
// (the Jacobi-Anger expansion of e^{-i z x} in Chebyshev polynomials: the
// Chebyshev propagator of Tal-Ezer and Kosloff, J. Chem. Phys. 81, 3967
// (1984)), with T_k(X) v from the three-term recurrence
// T_{k+1}(X) v = 2 X T_k(X) v - T_{k-1}(X) v.  The phase e^{-i c_n} is applied
// exactly in FP64.  The Bessel values J_k(z) come from Miller's downward
// recurrence J_{k-1} = (2k/z) J_k - J_{k+1}, normalised by
// J_0 + 2 sum_{k>=1} J_{2k} = 1; the series stops at the first degree k_t past
// which the bound |J_k(z)| <= (z/2)^k / k! leaves a tail below 2^-56.
//
// Sparse operators.  H0 and the H_k are held in one CSR pattern (the union of
// their nonzeros plus the diagonal) with one value array per operator, so an
// interval first forms X's values (sum over operators, shift, scale) and then
// runs plain CSR products.  In the circuit-QED models (b + b^dag, n, a^dag a)
// an interval costs about (degree) x (nonzeros) complex multiply-adds instead
// of the d^3 products that forming U_n takes.
//
// Kernels: a bounds kernel (one warp per interval, all intervals of all jobs
// in parallel) computes c_n, rho_n, s_n, k_t and the J_k(z); a chain kernel
// carries each job's state through its intervals with one thread per row and
// one barrier per operator application, the vectors and, where they fit, the
// interval matrix and its pattern in shared memory.  The chain runs either as
// one CTA per job (batches: every SM busy with its own jobs) or as one thread
// block cluster of up to 16 CTAs per job (a few large jobs): each CTA owns a
// contiguous block of rows and keeps copies of the two recurrence vectors,
// writes each new row through distributed shared memory into the CTAs whose
// nonzeros read it (a per-row mask built on the host: for banded operators only
// the neighbouring blocks) after each operator application, and the cluster
// barrier that follows orders them before the next application reads.
#include "common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>

namespace mg {

constexpr int ACTION_THREADS = 256;   // chain kernels: up to 3 CTAs per SM (80 registers)
constexpr int ACTION_MAX_OPS = 256;
constexpr double ACTION_ZMAX = 20.0;          // largest z = rho / s of one sub-step
constexpr int ACTION_MAX_SUBSTEPS = 1 << 14;  // per interval
// z <= 20 needs degrees below 64: 2 (10^{k+1} / (k+1)!) <= 2^-56 from k = 53
constexpr int ACTION_KMAX = 64;
static_assert(5 + ACTION_KMAX + 1 + 2 <= ACTION_REC, "interval record too small");

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {   // acc + a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

// J_k(z), k = 0..k_t, into J; returns k_t (see the file comment).  0 <= z <= 20.
__device__ int bessel_series(double z, double* J) {
  if (!(z > 1e-100)) {   // J_0 = 1 and J_1 ~ z/2 below any rounding of the state
    J[0] = 1.0;
    return 0;
  }
  // degree: smallest k >= z - 2 with 2 (z/2)^{k+1} / (k+1)! <= 2^-56; past it
  // the bound's ratio (z/2)/(k+2) is at most 1/2, so the tail is at most twice that
  const double h = 0.5 * z;
  double b = 1.0;   // (z/2)^k / k!
  int kt = ACTION_KMAX;
  for (int k = 0; k < ACTION_KMAX; ++k) {
    const double next = b * h / (k + 1);
    if (k + 2 >= z && 2.0 * next <= 0x1p-56) {
      kt = k;
      break;
    }
    b = next;
  }
  // Miller: downward from m0 well past k_t, rescaling to stay in range
  const int m0 = kt + 32;
  const double two_over_z = 2.0 / z;
  double jp1 = 0.0, j = 0x1p-200, norm = 0.0;
  for (int k = m0; k >= 1; --k) {
    if (k <= kt) J[k] = j;
    if ((k & 1) == 0) norm += 2.0 * j;
    const double jm1 = fma(k * two_over_z, j, -jp1);
    jp1 = j;
    j = jm1;
    if (fabs(j) > 0x1p+600) {   // rescale everything held so far
      j *= 0x1p-600;
      jp1 *= 0x1p-600;
      norm *= 0x1p-600;
      for (int q = k; q <= kt; ++q) J[q] *= 0x1p-600;
    }
  }
  norm += j;   // J_0
  J[0] = j;
  const double inv = 1.0 / norm;
  for (int q = 0; q <= kt; ++q) J[q] *= inv;
  return kt;
}

// One warp per (job, interval): Gershgorin bounds of Hbar_n, the sub-step
// count and the Chebyshev coefficients.  Record layout (ACTION_REC doubles):
// [c_n, 1/rho_n, s_n, k_t, rho_n, J_0 .. J_{k_t}, ..., cos c_n, sin c_n]; s_n = -1 marks a
// non-finite bound, -2 one that needs more than ACTION_MAX_SUBSTEPS sub-steps.
__global__ void __launch_bounds__(256) action_bounds_kernel(const ActionJob* __restrict__ jobs) {
  const ActionJob& J = jobs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (n >= J.N) return;   // whole warps leave together
  const double* crow = J.c + (long long)(J.first + n) * J.K;
  double lo = 1e300, hi = -1e300;
  bool bad = false;
  for (int i = lane; i < J.d; i += 32) {
    double dv = 0.0, r = 0.0;
    const int di = J.diag[i];
    for (int e = J.rowptr[i]; e < J.rowptr[i + 1]; ++e) {
      double ar = 0.0, ai = 0.0;
      for (int op = 0; op <= J.K; ++op) {
        const double coef = op == 0 ? J.dt : crow[op - 1];
        const double2 v = reinterpret_cast<const double2*>(J.val)[(long long)op * J.nnz + e];
        ar = fma(coef, v.x, ar);
        ai = fma(coef, v.y, ai);
      }
      if (e == di) {
        dv = ar;
        r += fabs(ai);   // zero for Hermitian input; kept so the disc stays an upper bound
      } else {
        r += hypot(ar, ai);
      }
    }
    if (!isfinite(dv) || !isfinite(r)) bad = true;
    lo = fmin(lo, dv - r);
    hi = fmax(hi, dv + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane != 0) return;
  double* rec = J.cheb + (long long)n * ACTION_REC;
  const double center = 0.5 * (lo + hi);
  // half-width, widened by 2^-40 of the largest endpoint to cover the rounding of the disc sums
  const double rho = 0.5 * (hi - lo) + 0x1p-40 * fmax(fabs(lo), fabs(hi));
  if (bad || !isfinite(center) || !isfinite(rho)) {
    rec[2] = -1.0;
    return;
  }
  if (rho > ACTION_ZMAX * ACTION_MAX_SUBSTEPS) {
    rec[2] = -2.0;
    return;
  }
  const int s = rho > ACTION_ZMAX ? (int)ceil(rho / ACTION_ZMAX) : 1;
  const double z = rho / s;
  const int kt = bessel_series(z, rec + 5);
  rec[0] = center;
  rec[1] = rho > 0.0 ? 1.0 / rho : 0.0;
  rec[2] = (double)s;
  rec[3] = (double)kt;
  rec[4] = rho;
  sincos(center, &rec[ACTION_REC - 1], &rec[ACTION_REC - 2]);   // the phase e^{-i c_n}: cos, sin
}


// acc + 2 (-i)^k J_k t without a branch on k: (a, b) = (t.y, -t.x) for odd k,
// (t.x, t.y) for even k, times +2 J_k for k mod 4 < 2 and -2 J_k otherwise
__device__ __forceinline__ double2 add_term_sel(double2 acc, double2 t, double f, bool odd) {
  const double a = odd ? t.y : t.x, b = odd ? -t.x : t.y;
  return make_double2(fma(f, a, acc.x), fma(f, b, acc.y));
}

// One sub-step on rows threadIdx.x, threadIdx.x + blockDim.x, ... of d:
// acc <- J_0 acc + 2 sum_{k=1..kt} (-i)^k J_k T_k(X) acc, vx / vy the recurrence
// vectors.  Inlined at two call sites, one with the interval matrix and pattern
// in shared memory and one with them in global memory, so that each copy
// addresses its operands directly rather than through generic pointers.
__device__ __forceinline__ void cheb_substep(int d, int kt, const double* Jk, const double2* A, const int* col,
                                             const int* rp, double2* acc, double2* vx, double2* vy) {
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double2 v = acc[i];
    vx[i] = v;
    acc[i] = make_double2(Jk[0] * v.x, Jk[0] * v.y);
  }
  __syncthreads();
  for (int k = 1; k <= kt; ++k) {
    // k odd: vy <- 2 X vx - vy (k = 1: X vx); k even: vx <- 2 X vy - vx
    const double2* cur = (k & 1) ? vx : vy;
    double2* old = (k & 1) ? vy : vx;
    const double two = k == 1 ? 1.0 : 2.0;
    const double f = ((k & 3) < 2 ? 2.0 : -2.0) * Jk[k];
    const bool odd = k & 1;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      double2 y0 = make_double2(0.0, 0.0), y1 = make_double2(0.0, 0.0);
      const int e1 = rp[i + 1];
      int e = rp[i];
      for (; e + 1 < e1; e += 2) {   // two independent accumulators
        y0 = cfma(A[e], cur[col[e]], y0);
        y1 = cfma(A[e + 1], cur[col[e + 1]], y1);
      }
      if (e < e1) y0 = cfma(A[e], cur[col[e]], y0);
      const double2 o = k > 1 ? old[i] : make_double2(0.0, 0.0);
      const double2 t = make_double2(fma(two, y0.x + y1.x, -o.x), fma(two, y0.y + y1.y, -o.y));
      old[i] = t;
      acc[i] = add_term_sel(acc[i], t, f, odd);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(ACTION_THREADS, 3)
action_chain_kernel(ActionJob* __restrict__ jobs, int dmax, int nnz_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double cn[ACTION_MAX_OPS];
  __shared__ double Jk[ACTION_KMAX + 1];
  ActionJob& R = jobs[blockIdx.x];
  const ActionJob J = R;
  const int d = J.d;
  double2* acc = reinterpret_cast<double2*>(smem_raw);   // the state
  double2* vx = acc + dmax;
  double2* vy = acc + 2 * dmax;
  const bool in_smem = J.nnz <= nnz_cap;
  double2* A = in_smem ? acc + 3 * dmax : reinterpret_cast<double2*>(J.abuf);
  int* col_s = reinterpret_cast<int*>(acc + 3 * dmax + nnz_cap);
  int* rp_s = col_s + nnz_cap;
  const int* rp = in_smem ? rp_s : J.rowptr;
  if (in_smem) {
    for (int e = threadIdx.x; e < J.nnz; e += blockDim.x) col_s[e] = J.col[e];
    for (int i = threadIdx.x; i <= d; i += blockDim.x) rp_s[i] = J.rowptr[i];
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) acc[i] = reinterpret_cast<const double2*>(J.psi)[i];
  long long matvecs = 0;
  int max_sub = 0, min_sub = 1 << 30, max_deg = 0, done = 0;
  double max_rho = 0.0;
  __syncthreads();
  for (int n = 0; n < J.N; ++n) {
    const double* rec = J.cheb + (long long)n * ACTION_REC;
    const int s = (int)rec[2];
    if (s <= 0) {   // uniform: every thread reads the same record
      if (threadIdx.x == 0) R.status = s == -1 ? MG_ENONFINITE : MG_EUNSUPPORTED;
      return;
    }
    const double center = rec[0], inv_rho = rec[1];
    const int kt = (int)rec[3];
    max_sub = max(max_sub, s);
    min_sub = min(min_sub, s);
    max_deg = max(max_deg, kt);
    max_rho = fmax(max_rho, rec[4]);
    const double* crow = J.c + (long long)(J.first + n) * J.K;
    for (int k = threadIdx.x; k < J.K; k += blockDim.x) cn[k] = crow[k];
    for (int k = threadIdx.x; k <= kt; k += blockDim.x) Jk[k] = rec[5 + k];
    __syncthreads();
    // X = (Hbar_n - c_n I) / rho_n on the union pattern, own rows
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      const int di = J.diag[i];
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        double ar = 0.0, ai = 0.0;
        for (int op = 0; op <= J.K; ++op) {
          const double coef = op == 0 ? J.dt : cn[op - 1];
          const double2 v = reinterpret_cast<const double2*>(J.val)[(long long)op * J.nnz + e];
          ar = fma(coef, v.x, ar);
          ai = fma(coef, v.y, ai);
        }
        if (e == di) ar -= center;
        A[e] = make_double2(ar * inv_rho, ai * inv_rho);
      }
    }
    __syncthreads();
    for (int sub = 0; sub < s; ++sub) {
      if (in_smem)
        cheb_substep(d, kt, Jk, acc + 3 * dmax, col_s, rp_s, acc, vx, vy);
      else
        cheb_substep(d, kt, Jk, reinterpret_cast<const double2*>(J.abuf), J.col, J.rowptr, acc, vx, vy);
      matvecs += kt;
    }
    // exact phase of the spectral centre (cos, sin from the bounds kernel)
    const double cs = rec[ACTION_REC - 2], sn = rec[ACTION_REC - 1];
    double2* trow = J.traj ? reinterpret_cast<double2*>(J.traj) + (long long)(J.first + n + 1) * d : nullptr;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      const double2 v = acc[i];
      acc[i] = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
      if (trow) trow[i] = acc[i];
    }
    __syncthreads();
    done = n + 1;
    if (J.max_steps > 0 && matvecs >= J.max_steps) break;   // uniform: the same count in every thread
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) reinterpret_cast<double2*>(J.psi)[i] = acc[i];
  if (threadIdx.x == 0) {
    R.done = done;
    R.matvecs = matvecs;
    R.max_sub = max_sub;
    R.min_sub = J.N > 0 ? min_sub : 0;
    R.max_terms = max_deg;
    R.max_nu = max_rho;
  }
}

// The recurrence of one sub-step in the cluster variant (own rows r0 .. r0 + nr,
// local pattern offsets rp); inlined once for on-chip and once for global
// operands, as cheb_substep.
__device__ __forceinline__ void cluster_recurrence(cooperative_groups::cluster_group& cl, int kt, const double* Jk,
                                                   int r0, int nr, const double2* A, const int* col, const int* rp,
                                                   const uint16_t* sendmask, double2* acc, double2* vx,
                                                   double2* vy) {
  for (int k = 1; k <= kt; ++k) {
    const double2* cur = (k & 1) ? vx : vy;
    double2* old = (k & 1) ? vy : vx;
    const double two = k == 1 ? 1.0 : 2.0;
    const double f = ((k & 3) < 2 ? 2.0 : -2.0) * Jk[k];
    const bool odd = k & 1;
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
      const int i = r0 + li;
      double2 y0 = make_double2(0.0, 0.0), y1 = make_double2(0.0, 0.0);
      const int e1 = rp[li + 1];
      int e = rp[li];
      for (; e + 1 < e1; e += 2) {
        y0 = cfma(A[e], cur[col[e]], y0);
        y1 = cfma(A[e + 1], cur[col[e + 1]], y1);
      }
      if (e < e1) y0 = cfma(A[e], cur[col[e]], y0);
      const double2 o = k > 1 ? old[i] : make_double2(0.0, 0.0);
      const double2 t = make_double2(fma(two, y0.x + y1.x, -o.x), fma(two, y0.y + y1.y, -o.y));
      acc[li] = add_term_sel(acc[li], t, f, odd);
      for (unsigned m = sendmask[i]; m; m &= m - 1) cl.map_shared_rank(old, __ffs(m) - 1)[i] = t;
    }
    cl.sync();
  }
}

// One cluster of C CTAs per job (blockIdx.x / C); CTA r of the cluster owns
// rows [r * ceil(d / C), ...).  Shared memory: full copies of the two
// recurrence vectors (dmax each), the state of the own rows (rows_max), then,
// where cap_loc > 0 and the job's own-row nonzeros fit, the own rows' interval
// matrix and column indices; the own rows' local row offsets always.
__global__ void __launch_bounds__(ACTION_THREADS, 3)
action_chain_cluster_kernel(ActionJob* __restrict__ jobs, int dmax, int cap_loc) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double cn[ACTION_MAX_OPS];
  __shared__ double Jk[ACTION_KMAX + 1];
  const int job = blockIdx.x / C;
  ActionJob& R = jobs[job];
  const ActionJob J = R;
  const int d = J.d;
  const int rows_max = (dmax + C - 1) / C;
  const int rows_per = (d + C - 1) / C;
  const int r0 = min(d, rank * rows_per), r1 = min(d, r0 + rows_per);
  const int nr = r1 - r0;
  double2* vx = reinterpret_cast<double2*>(smem_raw);
  double2* vy = vx + dmax;
  double2* acc = vy + dmax;   // own rows
  const int e_base = J.rowptr[r0];
  const int nnz_loc = J.rowptr[r1] - e_base;
  const bool in_smem = nnz_loc <= cap_loc;
  double2* A_s = acc + rows_max;
  int* col_s = reinterpret_cast<int*>(A_s + cap_loc);
  int* rp = col_s + cap_loc;   // rows_max + 1 local offsets
  double2* A = in_smem ? A_s : reinterpret_cast<double2*>(J.abuf) + e_base;
  for (int li = threadIdx.x; li <= nr; li += blockDim.x) rp[li] = J.rowptr[r0 + li] - e_base;
  if (in_smem)
    for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) col_s[e] = J.col[e_base + e];
  for (int li = threadIdx.x; li < nr; li += blockDim.x)
    acc[li] = reinterpret_cast<const double2*>(J.psi)[r0 + li];
  long long matvecs = 0;
  int max_sub = 0, min_sub = 1 << 30, max_deg = 0, done = 0;
  double max_rho = 0.0;
  cl.sync();   // every CTA of the cluster runs before any remote write
  for (int n = 0; n < J.N; ++n) {
    const double* rec = J.cheb + (long long)n * ACTION_REC;
    const int s = (int)rec[2];
    if (s <= 0) {   // uniform over the cluster: every CTA reads the same record
      if (rank == 0 && threadIdx.x == 0) R.status = s == -1 ? MG_ENONFINITE : MG_EUNSUPPORTED;
      cl.sync();
      return;
    }
    const double center = rec[0], inv_rho = rec[1];
    const int kt = (int)rec[3];
    max_sub = max(max_sub, s);
    min_sub = min(min_sub, s);
    max_deg = max(max_deg, kt);
    max_rho = fmax(max_rho, rec[4]);
    const double* crow = J.c + (long long)(J.first + n) * J.K;
    for (int k = threadIdx.x; k < J.K; k += blockDim.x) cn[k] = crow[k];
    for (int k = threadIdx.x; k <= kt; k += blockDim.x) Jk[k] = rec[5 + k];
    __syncthreads();
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
      const int i = r0 + li;
      const int di = J.diag[i] - e_base;
      for (int e = rp[li]; e < rp[li + 1]; ++e) {
        double ar = 0.0, ai = 0.0;
        for (int op = 0; op <= J.K; ++op) {
          const double coef = op == 0 ? J.dt : cn[op - 1];
          const double2 v = reinterpret_cast<const double2*>(J.val)[(long long)op * J.nnz + e_base + e];
          ar = fma(coef, v.x, ar);
          ai = fma(coef, v.y, ai);
        }
        if (e == di) ar -= center;
        A[e] = make_double2(ar * inv_rho, ai * inv_rho);
      }
    }
    for (int sub = 0; sub < s; ++sub) {
      // T_0 v = v into every CTA's vx; acc = J_0 v
      for (int li = threadIdx.x; li < nr; li += blockDim.x) {
        const double2 v = acc[li];
        acc[li] = make_double2(Jk[0] * v.x, Jk[0] * v.y);
        for (unsigned m = J.sendmask[r0 + li]; m; m &= m - 1) cl.map_shared_rank(vx, __ffs(m) - 1)[r0 + li] = v;
      }
      cl.sync();
      if (in_smem)
        cluster_recurrence(cl, kt, Jk, r0, nr, A_s, col_s, rp, J.sendmask, acc, vx, vy);
      else
        cluster_recurrence(cl, kt, Jk, r0, nr, reinterpret_cast<const double2*>(J.abuf) + e_base, J.col + e_base, rp,
                           J.sendmask, acc, vx, vy);
      matvecs += kt;
    }
    const double cs = rec[ACTION_REC - 2], sn = rec[ACTION_REC - 1];
    double2* trow = J.traj ? reinterpret_cast<double2*>(J.traj) + (long long)(J.first + n + 1) * d + r0 : nullptr;
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
      const double2 v = acc[li];
      acc[li] = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
      if (trow) trow[li] = acc[li];
    }
    __syncthreads();
    done = n + 1;
    if (J.max_steps > 0 && matvecs >= J.max_steps) break;   // uniform over the cluster
  }
  for (int li = threadIdx.x; li < nr; li += blockDim.x) reinterpret_cast<double2*>(J.psi)[r0 + li] = acc[li];
  if (rank == 0 && threadIdx.x == 0) {
    R.done = done;
    R.matvecs = matvecs;
    R.max_sub = max_sub;
    R.min_sub = J.N > 0 ? min_sub : 0;
    R.max_terms = max_deg;
    R.max_nu = max_rho;
  }
  cl.sync();   // no CTA leaves while another may still address its shared memory
}

size_t action_cluster_smem_bytes(int dmax, int C, int cap_loc) {
  const size_t rows_max = (size_t)(dmax + C - 1) / C;
  return sizeof(double2) * (2 * (size_t)dmax + rows_max) + (sizeof(double2) + sizeof(int)) * (size_t)cap_loc +
         sizeof(int) * (rows_max + 1);
}

// Both chain kernels get the largest dynamic shared memory any launch uses
// (and the cluster kernel non-portable cluster sizes) once, up front.
int action_attrs() {
  MG_TRY(ensure_smem_limit(reinterpret_cast<const void*>(action_chain_kernel), ACTION_SMEM_LIMIT));
  MG_TRY(ensure_smem_limit(reinterpret_cast<const void*>(action_chain_cluster_kernel), ACTION_SMEM_LIMIT));
  return ensure_func_attr(reinterpret_cast<const void*>(action_chain_cluster_kernel),
                          cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// Largest cluster size <= want (a power of two) that the device can co-schedule
// with this shared memory, or 1; answers are cached per (size, shared memory).
int action_cluster_size(int want, int dmax, int cap_loc) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, bool> fits;
  if (action_attrs() != MG_OK) {
    cudaGetLastError();
    return 1;
  }
  for (int C = want; C >= 2; C >>= 1) {
    const size_t smem = action_cluster_smem_bytes(dmax, C, cap_loc);
    if (smem > (size_t)ACTION_SMEM_LIMIT) continue;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = fits.find({C, smem});
      if (it != fits.end()) {
        if (it->second) return C;
        continue;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(ACTION_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&active, action_chain_cluster_kernel, &cfg) == cudaSuccess &&
                    active >= 1;
    if (!ok) cudaGetLastError();
    std::lock_guard<std::mutex> lock(mu);
    fits[{C, smem}] = ok;
    if (ok) return C;
  }
  return 1;
}

int launch_action_cluster(int njobs, ActionJob* jobs_dev, int dmax, int C, int cap_loc, cudaStream_t s) {
  const size_t smem = action_cluster_smem_bytes(dmax, C, cap_loc);
  MG_TRY(action_attrs());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * C, 1, 1);
  cfg.blockDim = dim3(ACTION_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, action_chain_cluster_kernel, jobs_dev, dmax, cap_loc);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "cudaLaunchKernelEx(action_chain_cluster_kernel)", __FILE__, __LINE__);
    return MG_ECUDA;
  }
  return check_launch("action_chain_cluster_kernel");
}

size_t action_smem_bytes(int dmax, int nnz_cap) {
  size_t b = sizeof(double2) * 3 * (size_t)dmax;
  if (nnz_cap > 0) b += (sizeof(double2) + sizeof(int)) * (size_t)nnz_cap + sizeof(int) * ((size_t)dmax + 1);
  return b;
}

int launch_action_chain(int njobs, ActionJob* jobs_dev, int dmax, int nmax, int nnz_cap, int cluster,
                        cudaStream_t s) {
  if (njobs <= 0) return MG_OK;
  if (nmax > 0) {
    dim3 grid((nmax + 7) / 8, njobs);
    action_bounds_kernel<<<grid, 256, 0, s>>>(jobs_dev);
    MG_TRY(check_launch("action_bounds_kernel"));
  }
  if (cluster > 1) return launch_action_cluster(njobs, jobs_dev, dmax, cluster, nnz_cap, s);
  const size_t smem = action_smem_bytes(dmax, nnz_cap);
  MG_TRY(action_attrs());
  // one thread per row up to ACTION_THREADS; small jobs take fewer warps
  const int threads = std::min(ACTION_THREADS, (dmax + 31) / 32 * 32);
  action_chain_kernel<<<njobs, threads, smem, s>>>(jobs_dev, dmax, nnz_cap);
  return check_launch("action_chain_kernel");
}

}  // namespace mg
