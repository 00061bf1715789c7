// Device-side decisions of the batched path, so that a whole batch can be issued
// without reading anything back to the host between its launches (and captured
// in one CUDA graph):
//
//   * op_norm1_kernel      ||A - tau I||_1 (tau = Re tr(A)/d) of each resident
//                          operator: with the per-job largest |c_{k,n}| it bounds
//                          ||Hbar_n - tau_n I||_1 of every interval before any
//                          Hbar_n is formed (triangle inequality over
//                          Eq. magnus-first-order-term; tau_n is linear in c).
//   * coef_absmax_kernel   max_n |c_{k,n}| per job and control.
//   * fail_segments_kernel a job whose Hbar_n has a non-finite norm fails alone:
//                          its flag is set and its segment's norms and phases
//                          are zeroed (its exponents are zeroed by zero_bad_kernel).
//   * squarings_kernel     the squaring count of every interval,
//                          s_n = min{s >= 0 : 2^-s ||Hbar_n - tau_n I||_1 <= theta_m},
//                          capped at the batch's launch count S (the cap raises a flag).
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace mg {

__global__ void __launch_bounds__(256) op_norm1_kernel(int d, const double* __restrict__ ops, double* __restrict__ out) {
  const double* A = ops + (long long)blockIdx.x * 2 * d * d;
  __shared__ double red[256];
  // tau = Re tr(A) / d
  double t = 0.0;
  for (int i = threadIdx.x; i < d; i += 256) t += A[2 * ((long long)i * d + i)];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double tau = red[0] / d;
  __syncthreads();
  // largest absolute column sum of A - tau I (one thread per column, rows in order)
  double best = 0.0;
  for (int j = threadIdx.x; j < d; j += 256) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
      const long long e = 2 * ((long long)i * d + j);
      const double re = A[e] - (i == j ? tau : 0.0), im = A[e + 1];
      s += hypot(re, im);
    }
    best = fmax(best, s);
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

int launch_op_norm1(int count, int d, const double* ops, double* out, cudaStream_t s) {
  if (count <= 0) return MG_OK;
  op_norm1_kernel<<<count, 256, 0, s>>>(d, ops, out);
  return check_launch("op_norm1_kernel");
}

// one block per job: out[off + k] = max_n |c[n][k]| (NaN propagates: fmax ignores it, so
// a non-finite coefficient is recorded through isfinite instead)
__global__ void __launch_bounds__(128) coef_absmax_kernel(const CoefRef* __restrict__ refs, double* __restrict__ out) {
  const CoefRef r = refs[blockIdx.x];
  for (int k = threadIdx.x; k < r.K; k += 128) {
    double m = 0.0;
    bool finite = true;
    for (int n = 0; n < r.N; ++n) {
      const double v = r.c[(long long)n * r.K + k];
      finite &= isfinite(v);
      m = fmax(m, fabs(v));
    }
    out[r.off + k] = finite ? m : __longlong_as_double(0x7ff8000000000000LL);
  }
}

int launch_coef_absmax(int njobs, const CoefRef* refs_dev, double* out, cudaStream_t s) {
  if (njobs <= 0) return MG_OK;
  coef_absmax_kernel<<<njobs, 128, 0, s>>>(refs_dev, out);
  return check_launch("coef_absmax_kernel");
}

// one block per segment: seg_tab[3 q] = job, [3 q + 1] = first item, [3 q + 2] = items
__global__ void __launch_bounds__(256) fail_segments_kernel(const int* __restrict__ seg_tab, double* __restrict__ norm,
                                                            double* __restrict__ tau, int* __restrict__ job_fail,
                                                            int* __restrict__ seg_bad) {
  const int q = blockIdx.x;
  const int job = seg_tab[3 * q], off = seg_tab[3 * q + 1], n = seg_tab[3 * q + 2];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < n; i += 256) mine |= !isfinite(norm[off + i]) || !isfinite(tau[off + i]);
  if (mine) atomicOr(&bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    seg_bad[q] = bad;
    if (bad) job_fail[job] = 1;
  }
  if (bad)
    for (int i = threadIdx.x; i < n; i += 256) {
      norm[off + i] = 0.0;
      tau[off + i] = 0.0;
    }
}

// one block per item: zero the exponent of items of failed segments
__global__ void __launch_bounds__(256) zero_bad_kernel(long long md, const int* __restrict__ seg_of_item,
                                                       const int* __restrict__ seg_bad, double* __restrict__ W) {
  const int b = blockIdx.x;
  if (!seg_bad[seg_of_item[b]]) return;
  double* w = W + (long long)b * md;
  for (long long e = threadIdx.x; e < md; e += 256) w[e] = 0.0;
}

int launch_fail_segments(int nseg, int fill, long long md, const int* seg_tab, const int* seg_of_item, double* norm,
                         double* tau, int* job_fail, int* seg_bad, double* W, cudaStream_t s) {
  if (nseg <= 0) return MG_OK;
  fail_segments_kernel<<<nseg, 256, 0, s>>>(seg_tab, norm, tau, job_fail, seg_bad);
  MG_TRY(check_launch("fail_segments_kernel"));
  zero_bad_kernel<<<fill, 256, 0, s>>>(md, seg_of_item, seg_bad, W);
  return check_launch("zero_bad_kernel");
}

__global__ void copy_active_kernel(long long md2, const double2* __restrict__ src, double2* __restrict__ dst,
                                   const int* __restrict__ item_sq, int sq_step) {
  const int b = blockIdx.y;
  if (item_sq[b] <= sq_step) return;
  const double2* s = src + (long long)b * md2;
  double2* t = dst + (long long)b * md2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < md2; e += (long long)gridDim.x * blockDim.x)
    t[e] = s[e];
}

int launch_copy_active(int batch, long long md, const double* src, double* dst, const int* item_sq, int sq_step,
                       cudaStream_t s) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  const long long md2 = md / 2;
  const int gx = (int)std::min<long long>((md2 + 255) / 256, 64);
  copy_active_kernel<<<dim3(gx, batch), 256, 0, s>>>(md2, reinterpret_cast<const double2*>(src),
                                                      reinterpret_cast<double2*>(dst), item_sq, sq_step);
  return check_launch("copy_active_kernel");
}

// *out = max |a_e - b_e| over n doubles (out preset to 0; non-negative doubles order as integers)
__global__ void max_abs_diff_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                    unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = fabs(a[e] - b[e]);
    m = v > m || v != v ? v : m;   // a NaN difference wins (it marks a failed candidate)
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, m, o);
    m = w > m || w != w ? w : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int launch_max_abs_diff(long long n, const double* a, const double* b, double* out, cudaStream_t s) {
  MG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n <= 0) return MG_OK;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  max_abs_diff_kernel<<<grid, 256, 0, s>>>(n, a, b, reinterpret_cast<unsigned long long*>(out));
  return check_launch("max_abs_diff_kernel");
}

__global__ void squarings_kernel(int n, const double* __restrict__ norm, double theta, int S, int uniform,
                                 int* __restrict__ sq, int* __restrict__ overflow, double* __restrict__ flops_acc,
                                 double flops_per_square) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = norm[i];
  int s = 0;
  while (s < 1022 && ldexp(v, -s) > theta) ++s;
  if (s > S) {
    atomicExch(overflow, 1);
    s = S;
  }
  const int q = uniform ? S : s;
  sq[i] = q;
  if (flops_acc && !uniform && q > 0) atomicAdd(flops_acc, flops_per_square * q);
}

int launch_squarings(int n, const double* norm, double theta, int S, int uniform, int* sq, int* overflow,
                     double* flops_acc, double flops_per_square, cudaStream_t s) {
  if (n <= 0) return MG_OK;
  squarings_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, norm, theta, S, uniform, sq, overflow, flops_acc,
                                                   flops_per_square);
  return check_launch("squarings_kernel");
}

}  // namespace mg
