// Action-based state propagation with sparse operators.
//
// For state outputs the product U_{N-1} ... U_0 psi0 never needs the matrices
// U_n = exp(-i Hbar_n): each interval applies the exponential to the state,
//
//   psi <- e^{-i tau_n} exp(-i (Hbar_n - tau_n I)) psi,
//   (Hbar_n - tau_n I) v = dt (H0 - t0 I) v + sum_k c_{k,n} (H_k - t_k I) v,
//
// (t0, t_k the operators' trace means, tau_n = dt t0 + sum_k c_{k,n} t_k), with
// a scaled Taylor series: s_n = ceil(nu_n / 2) sub-steps of at most 40 terms,
//   v <- sum_{j<=m} (-i A / s_n)^j v / j!,
// stopped early once two consecutive terms fall below the FP64 unit roundoff
// relative to the partial sum.  The operators are held in CSR (they are
// sparse in the circuit-QED models: b + b^dag, n, a^dag a), so an interval
// costs about (terms) x (nonzeros) complex multiply-adds instead of the d^3
// products that forming U_n takes.  s_n comes from an FP64 upper bound of
// ||Hbar_n - tau_n I||_1 built from the operators' shifted 1-norms.
//
// One CTA carries one job's state through a range of intervals (grid = jobs),
// vectors in shared memory, one thread per row.
#include "common.cuh"

namespace mg {

constexpr int ACTION_THREADS = 256;
// Sub-step norm theta = 2: the rounding of one sub-step grows like e^theta
// (the sum of the terms' magnitudes) while the sub-step count falls like
// 1/theta; theta = 2 keeps the summed rounding of a long run within a few
// times that of theta = 1 at 65% of its matvecs.  2^40/40! is far below the
// FP64 unit roundoff, so 40 terms always suffice.
constexpr int ACTION_MAX_TERMS = 40;
constexpr double ACTION_THETA = 2.0;
constexpr int ACTION_MAX_OPS = 256;
constexpr int ACTION_MAX_SUBSTEPS = 1 << 14;

__device__ __forceinline__ double2 cmul_i(double2 a, double s) {  // (-i s) a
  return make_double2(s * a.y, -s * a.x);
}

// y = (Hbar - tau I) x for one interval (x, y in shared memory)
__device__ void apply_shifted(const ActionJob& J, const double* cn, double tau, const double2* x, double2* y) {
  for (int i = threadIdx.x; i < J.d; i += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int op = 0; op <= J.K; ++op) {
      const double coef = op == 0 ? J.dt : cn[op - 1];
      if (coef == 0.0) continue;
      const int* rp = J.rowptr + op * (J.d + 1);
      const int base = J.opoff[op];
      double sr = 0.0, si = 0.0;
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int j = J.col[base + e];
        const double2 h = reinterpret_cast<const double2*>(J.val)[base + e];
        const double2 v = x[j];
        sr = fma(h.x, v.x, sr);
        sr = fma(-h.y, v.y, sr);
        si = fma(h.x, v.y, si);
        si = fma(h.y, v.x, si);
      }
      re = fma(coef, sr, re);
      im = fma(coef, si, im);
    }
    re -= tau * x[i].x;
    im -= tau * x[i].y;
    y[i] = make_double2(re, im);
  }
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
  return m;
}

__global__ void __launch_bounds__(ACTION_THREADS)
action_chain_kernel(ActionJob* __restrict__ jobs, double theta) {
  extern __shared__ double2 vec[];
  __shared__ double red[ACTION_THREADS / 32];
  __shared__ double cn[ACTION_MAX_OPS];
  const ActionJob J = jobs[blockIdx.x];
  const int d = J.d;
  double2* psi = vec;
  double2* term = vec + d;
  double2* nxt = vec + 2 * d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) psi[i] = reinterpret_cast<double2*>(J.psi)[i];
  long long matvecs = 0;
  int max_sub = 0, min_sub = 1 << 30, max_terms = 0;
  double max_nu = 0.0;
  __syncthreads();
  for (int n = 0; n < J.N; ++n) {
    const double* crow = J.c + (long long)(J.first + n) * J.K;
    for (int k = threadIdx.x; k < J.K; k += blockDim.x) cn[k] = crow[k];
    __syncthreads();
    double tau = J.dt * J.trace_mean[0];
    double nu = J.dt * J.shifted_norm[0];
    for (int k = 0; k < J.K; ++k) {
      tau = fma(cn[k], J.trace_mean[1 + k], tau);
      nu = fma(fabs(cn[k]), J.shifted_norm[1 + k], nu);
    }
    // bounded work: a non-finite bound or more than ACTION_MAX_SUBSTEPS sub-steps
    // ends the job with an error status instead of an arbitrarily long loop
    if (!(nu <= theta * ACTION_MAX_SUBSTEPS)) {
      if (threadIdx.x == 0) jobs[blockIdx.x].status = isfinite(nu) ? MG_EUNSUPPORTED : MG_ENONFINITE;
      return;
    }
    const int s = nu > theta ? (int)ceil(nu / theta) : 1;
    max_sub = max(max_sub, s);
    min_sub = min(min_sub, s);
    max_nu = fmax(max_nu, nu);
    const double inv_s = 1.0 / s;
    for (int sub = 0; sub < s; ++sub) {
      // term = psi; acc (psi) accumulates terms
      for (int i = threadIdx.x; i < d; i += blockDim.x) term[i] = psi[i];
      __syncthreads();
      double prev = 1e300;
      for (int j = 1; j <= ACTION_MAX_TERMS; ++j) {
        apply_shifted(J, cn, tau, term, nxt);
        ++matvecs;
        max_terms = max(max_terms, j);
        __syncthreads();
        const double f = inv_s / j;
        double tmax = 0.0, amax = 0.0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
          const double2 t = cmul_i(nxt[i], f);
          term[i] = t;
          double2 a = psi[i];
          a.x += t.x;
          a.y += t.y;
          psi[i] = a;
          tmax = fmax(tmax, fmax(fabs(t.x), fabs(t.y)));
          amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
        }
        tmax = block_max(tmax, red);
        amax = block_max(amax, red);
        if (tmax + prev <= 1.1102230246251565e-16 * amax) break;   // two negligible terms in a row
        prev = tmax;
      }
      __syncthreads();
    }
    // exact phase of the trace shift
    double sn, cs;
    sincos(tau, &sn, &cs);
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      const double2 v = psi[i];
      psi[i] = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) reinterpret_cast<double2*>(J.psi)[i] = psi[i];
  if (threadIdx.x == 0) {
    ActionJob& R = jobs[blockIdx.x];
    R.matvecs = matvecs;
    R.max_sub = max_sub;
    R.min_sub = J.N > 0 ? min_sub : 0;
    R.max_terms = max_terms;
    R.max_nu = max_nu;
  }
}

int launch_action_chain(int njobs, ActionJob* jobs_dev, int dmax, cudaStream_t s) {
  if (njobs <= 0) return MG_OK;
  const size_t smem = sizeof(double2) * 3 * dmax;
  if (smem > 48 * 1024)
    MG_CUDA_TRY(cudaFuncSetAttribute(action_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // one thread per row up to ACTION_THREADS; small jobs take fewer warps
  const int threads = std::min(ACTION_THREADS, (dmax + 31) / 32 * 32);
  action_chain_kernel<<<njobs, threads, smem, s>>>(jobs_dev, ACTION_THETA);
  return check_launch("action_chain_kernel");
}

}  // namespace mg
