// Quadrature coefficients and the first-order Magnus term of every interval.
//
//   c_{k,n}  = (dt/2) sum_p w_p u^(k)(t_{n,p})        (Eq. magnus-first-order-coeff)
//   Hbar_n   = dt H0 + sum_k c_{k,n} H_k              (Eq. magnus-first-order-term)
//
// The Hbar builder is HBM-bound: it streams the operators once per block of
// NB intervals (register blocking over intervals) and writes every Hbar_n once.
// In the same pass it forms the exact trace shift tau_n = Re tr(Hbar_n)/d (from
// the precomputed operator traces) and the FP64 1-norm ||Hbar_n - tau_n I||_1
// that selects the squaring count of the exponential.
#include "common.cuh"
#include "df32.cuh"

namespace mg {

// ---------------------------------------------------------------------------
__global__ void coefficients_kernel(int N, int P, int K, double half_dt, const double* __restrict__ w,
                                    const double* __restrict__ samples, double* __restrict__ c) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)N * K) return;
  int n = (int)(idx / K), k = (int)(idx % K);
  const double* s = samples + (long long)n * P * K + k;
  double acc = 0.0;
  for (int p = 0; p < P; ++p) acc = fma(w[p], s[(long long)p * K], acc);
  c[idx] = half_dt * acc;
}

int launch_coefficients(int N, int P, int K, double dt, const double* w_dev, const double* samples,
                        double* c, cudaStream_t s) {
  if (N <= 0 || K <= 0) return MG_OK;
  long long total = (long long)N * K;
  int threads = 256;
  coefficients_kernel<<<ceil_div(total, threads), threads, 0, s>>>(N, P, K, 0.5 * dt, w_dev, samples, c);
  return check_launch("coefficients_kernel");
}

// ---------------------------------------------------------------------------
// Second-order Magnus coefficients (Eq. magnus-avg, second line).  With
// H(t) = H0 + sum_k u_k(t) H_k the commutator splits as
//   [H(t1), H(t2)] = sum_k (u_k(t2) - u_k(t1)) [H0, H_k]
//                  + sum_{k<l} (u_k(t1) u_l(t2) - u_l(t1) u_k(t2)) [H_k, H_l],
// so Hbar^(2)_n = sum_k alpha_k (-i/2)[H0, H_k] + sum_{k<l} beta_kl (-i/2)[H_k, H_l]
// with scalar double integrals over t_n <= t2 <= t1 <= t_n + dt.  The drive is
// represented by its interpolating polynomial through the P samples, for which
//   int int f(t2) g(t1) = dt^2 sum_{p,q} g_p f_q M_pq
// with M_pq = int_0^1 l_p(s1) int_0^s1 l_q(s2) (Lagrange basis on the nodes).
// mrc holds M (P x P, row p = t1 node), then its column sums C_q and row sums R_p.
// Output row n of c (length K + K + K(K-1)/2): first-order c_k, then alpha_k, then
// beta_kl in the order (0,1), (0,2), ..., (K-2,K-1).
__global__ void second_order_coefficients_kernel(int N, int P, int K, double dt, const double* __restrict__ w,
                                                 const double* __restrict__ mrc,
                                                 const double* __restrict__ samples, double* __restrict__ c) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int Kx = 2 * K + K * (K - 1) / 2;
  const double* u = samples + (long long)n * P * K;   // u[p*K + k]
  double* out = c + (long long)n * Kx;
  const double* Mm = mrc;
  const double* Cq = mrc + P * P;
  const double* Rp = Cq + P;
  const double dt2 = dt * dt;
  for (int k = 0; k < K; ++k) {
    double first = 0.0, a = 0.0;
    for (int p = 0; p < P; ++p) {
      const double v = u[p * K + k];
      first = fma(w[p], v, first);
      a = fma(Cq[p] - Rp[p], v, a);
    }
    out[k] = 0.5 * dt * first;
    out[K + k] = dt2 * a;
  }
  int m = 2 * K;
  for (int k = 0; k < K; ++k)
    for (int l = k + 1; l < K; ++l, ++m) {
      double b = 0.0;
      for (int p = 0; p < P; ++p) {
        double inner_kl = 0.0, inner_lk = 0.0;
        for (int q = 0; q < P; ++q) {
          const double mpq = Mm[p * P + q];
          inner_kl = fma(mpq, u[q * K + l], inner_kl);
          inner_lk = fma(mpq, u[q * K + k], inner_lk);
        }
        b = fma(u[p * K + k], inner_kl, b);
        b = fma(-u[p * K + l], inner_lk, b);
      }
      out[m] = dt2 * b;
    }
}

int launch_second_order_coefficients(int N, int P, int K, double dt, const double* w_dev, const double* mrc_dev,
                                     const double* samples, double* c, cudaStream_t s) {
  if (N <= 0 || K <= 0) return MG_OK;
  second_order_coefficients_kernel<<<ceil_div(N, 128), 128, 0, s>>>(N, P, K, dt, w_dev, mrc_dev, samples, c);
  return check_launch("second_order_coefficients_kernel");
}

// ---------------------------------------------------------------------------
// traces: tr[0] = Re tr H0, tr[1 + k] = Re tr H_k
__global__ void operator_traces_kernel(int d, int K, const double* __restrict__ H0,
                                       const double* __restrict__ Hk, double* __restrict__ tr) {
  int k = blockIdx.x;  // 0..K
  const double* H = (k == 0) ? H0 : Hk + (long long)(k - 1) * d * d * 2;
  double acc = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) acc += H[2 * ((long long)i * d + i)];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) tr[k] = red[0];
}

// Ordered encoding of a non-negative double so that unsigned max = double max.
__device__ __forceinline__ unsigned long long nonneg_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// |x + i y| rounded up: an FP32 magnitude widened by 2^-20 relative, so that the
// FP64-accumulated column sums bound ||.||_1 from above (the norm only selects
// the squaring count, for which any upper bound is valid) without a long chain
// of FP64 instructions per element on GB300's narrow FP64 pipe.
__device__ __forceinline__ double magnitude_upper(double x, double y) {
  const float xf = (float)x, yf = (float)y;
  const float m = sqrtf(fmaf(xf, xf, yf * yf));
  return (double)(m * (1.0f + 9.5367431640625e-07f)) + 1e-300;
}

constexpr int OMEGA_NB = 8;      // intervals per CTA (register blocking)
constexpr int OMEGA_COLS = 32;   // columns per CTA (one per lane)
constexpr int OMEGA_WARPS = 8;   // row phases per CTA

// grid: (ceil(d/32), ceil(N/NB)); block 256 = 8 warps x 32 lanes.
// lane -> column j, warp -> rows i = warp, warp + 8, ...
__global__ void __launch_bounds__(256)
build_omega_kernel(int N, int d, int K, double dt, const double* __restrict__ H0,
                   const double* __restrict__ Hk, const double* __restrict__ c,
                   const double* __restrict__ tr, double* __restrict__ omega,
                   double* __restrict__ tau_out, unsigned long long* __restrict__ norm_bits,
                   int shift, int write_shifted) {
  extern __shared__ double sm[];
  double* cs = sm;                              // [NB][K]
  double* taus = cs + OMEGA_NB * (K > 0 ? K : 1);   // [NB]
  double* colpart = taus + OMEGA_NB;            // [WARPS][NB][32]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * OMEGA_COLS + lane;
  const int n0 = blockIdx.y * OMEGA_NB;
  const int nb = min(OMEGA_NB, N - n0);

  for (int t = threadIdx.x; t < OMEGA_NB * K; t += blockDim.x) {
    int b = t / K, k = t % K;
    cs[t] = (b < nb) ? c[(long long)(n0 + b) * K + k] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < OMEGA_NB) {
    int b = threadIdx.x;
    double t = 0.0;
    if (shift && b < nb) {
      t = dt * tr[0];
      for (int k = 0; k < K; ++k) t += cs[b * K + k] * tr[1 + k];
      t /= d;
    }
    taus[b] = t;
    if (b < nb && blockIdx.x == 0 && tau_out) tau_out[n0 + b] = t;
  }
  __syncthreads();

  double colsum[OMEGA_NB];
#pragma unroll
  for (int b = 0; b < OMEGA_NB; ++b) colsum[b] = 0.0;

  if (j < d) {
    const long long dd2 = (long long)d * d * 2;
    for (int i = warp; i < d; i += OMEGA_WARPS) {
      const long long off = 2 * ((long long)i * d + j);
      const double2 h0 = *reinterpret_cast<const double2*>(H0 + off);
      double re[OMEGA_NB], im[OMEGA_NB];
#pragma unroll
      for (int b = 0; b < OMEGA_NB; ++b) { re[b] = dt * h0.x; im[b] = dt * h0.y; }
      for (int k = 0; k < K; ++k) {
        const double2 hk = *reinterpret_cast<const double2*>(Hk + k * dd2 + off);
        // control operators are sparse (b + b^dag): skip the 2 NB FP64 FMAs of a zero
        // entry (integer test, uniform over the interval block)
        if (((__double_as_longlong(hk.x) | __double_as_longlong(hk.y)) << 1) == 0) continue;
#pragma unroll
        for (int b = 0; b < OMEGA_NB; ++b) {
          const double ck = cs[b * K + k];
          re[b] = fma(ck, hk.x, re[b]);
          im[b] = fma(ck, hk.y, im[b]);
        }
      }
#pragma unroll
      for (int b = 0; b < OMEGA_NB; ++b) {
        if (b < nb) {
          double r = re[b];
          if (i == j) r -= taus[b];
          colsum[b] += magnitude_upper(r, im[b]);
          double2 o;
          o.x = write_shifted ? r : re[b];
          o.y = im[b];
          *reinterpret_cast<double2*>(omega + (long long)(n0 + b) * dd2 + off) = o;
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < OMEGA_NB; ++b) colpart[(warp * OMEGA_NB + b) * 32 + lane] = colsum[b];
  __syncthreads();
  // reduce over warps (rows) then max over lanes (columns)
  if (warp < OMEGA_NB && warp < nb) {
    const int b = warp;
    double s = 0.0;
    for (int w = 0; w < OMEGA_WARPS; ++w) s += colpart[(w * OMEGA_NB + b) * 32 + lane];
    if (j >= d) s = 0.0;
    // NaN/Inf -> +Inf before the max (fmax would drop a NaN)
    if (!(s <= 1.0e300)) s = __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) atomicMax(norm_bits + n0 + b, nonneg_bits(s));
  }
}

// The same first-order term for the split-precision path, written as double-float
// (float4 {re.hi, re.lo, im.hi, im.lo} per element, minus tau_n I) so that the
// exponential's inputs never pass through the FP64 pipe: each operator entry is split
// into two FP32 numbers once per block of NB intervals, and every interval's sum
// dt H0 + sum_k c_{k,n} H_k is formed with error-free FP32 transformations
// (about 2^-46 relative); only the phases tau_n (K + 1 FP64 FMAs per interval) and
// the column sums of the norm bound stay in FP64.
__device__ __forceinline__ float magnitude_upper_f(float x, float y) {
  // |x + i y| of the hi parts, widened by 2^-20: also covers the lo parts (< 2^-23 relative)
  return sqrtf(fmaf(x, x, y * y)) * (1.0f + 9.5367431640625e-07f) + 1e-30f;
}
__device__ __forceinline__ df32 dfx_add(df32 x, df32 y) {   // double-float sum, one error-free step fewer
  const df32 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__global__ void __launch_bounds__(256)
build_omega_df_kernel(int N, int d, int K, double dt, const double* __restrict__ H0,
                      const double* __restrict__ Hk, const double* __restrict__ c,
                      const double* __restrict__ tr, float4* __restrict__ omega,
                      double* __restrict__ tau_out, unsigned long long* __restrict__ norm_bits, int shift) {
  extern __shared__ double sm[];
  double* taus = sm;                                  // [NB]
  double* colpart = taus + OMEGA_NB;                  // [WARPS][NB][32]
  df32* cs = reinterpret_cast<df32*>(colpart + OMEGA_WARPS * OMEGA_NB * 32);   // [NB][K]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * OMEGA_COLS + lane;
  const int n0 = blockIdx.y * OMEGA_NB;
  const int nb = min(OMEGA_NB, N - n0);

  for (int t = threadIdx.x; t < OMEGA_NB * K; t += blockDim.x) {
    int b = t / K, k = t % K;
    cs[t] = df_from_double((b < nb) ? c[(long long)(n0 + b) * K + k] : 0.0);
  }
  if (threadIdx.x < OMEGA_NB) {
    int b = threadIdx.x;
    double t = 0.0;
    if (shift && b < nb) {
      t = dt * tr[0];
      for (int k = 0; k < K; ++k) t += c[(long long)(n0 + b) * K + k] * tr[1 + k];
      t /= d;
    }
    taus[b] = t;
    if (b < nb && blockIdx.x == 0 && tau_out) tau_out[n0 + b] = t;
  }
  __syncthreads();
  const df32 dtd = df_from_double(dt);

  double colsum[OMEGA_NB];
#pragma unroll
  for (int b = 0; b < OMEGA_NB; ++b) colsum[b] = 0.0;

  if (j < d) {
    const long long dd2 = (long long)d * d * 2;
    const long long ddc = (long long)d * d;   // complex elements per matrix
    for (int i = warp; i < d; i += OMEGA_WARPS) {
      const long long off = 2 * ((long long)i * d + j);
      const double2 h0 = *reinterpret_cast<const double2*>(H0 + off);
      const df32 r0 = df_mul(df_from_double(h0.x), dtd), i0 = df_mul(df_from_double(h0.y), dtd);
      df32 re[OMEGA_NB], im[OMEGA_NB];
#pragma unroll
      for (int b = 0; b < OMEGA_NB; ++b) { re[b] = r0; im[b] = i0; }
      for (int k = 0; k < K; ++k) {
        const double2 hk = *reinterpret_cast<const double2*>(Hk + k * dd2 + off);
        if (((__double_as_longlong(hk.x) | __double_as_longlong(hk.y)) << 1) == 0) continue;   // sparse H_k
        const df32 hx = df_from_double(hk.x), hy = df_from_double(hk.y);
#pragma unroll
        for (int b = 0; b < OMEGA_NB; ++b) {
          const df32 ck = cs[b * K + k];
          re[b] = dfx_add(re[b], df_mul(hx, ck));
          im[b] = dfx_add(im[b], df_mul(hy, ck));
        }
      }
#pragma unroll
      for (int b = 0; b < OMEGA_NB; ++b) {
        if (b < nb) {
          df32 r = re[b];
          if (i == j) r = df_add(r, df_from_double(-taus[b]));
          colsum[b] += (double)magnitude_upper_f(r.hi, im[b].hi);
          omega[(long long)(n0 + b) * ddc + off / 2] = make_float4(r.hi, r.lo, im[b].hi, im[b].lo);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < OMEGA_NB; ++b) colpart[(warp * OMEGA_NB + b) * 32 + lane] = colsum[b];
  __syncthreads();
  if (warp < OMEGA_NB && warp < nb) {
    const int b = warp;
    double s = 0.0;
    for (int w = 0; w < OMEGA_WARPS; ++w) s += colpart[(w * OMEGA_NB + b) * 32 + lane];
    if (j >= d) s = 0.0;
    if (!(s <= 1.0e300)) s = __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) atomicMax(norm_bits + n0 + b, nonneg_bits(s));
  }
}

// The split path's builder for up to 8 operators (K <= 7), in two kernels with the
// arithmetic of build_omega_df_kernel (bit-identical Hbar_n and norms):
//
// omega_tile_df_kernel: one CTA per 8 x 32 tile of elements (one per thread) and tz
// intervals.  The thread's operator entries are split into FP32 pairs once and kept in
// registers, so an entry passes GB300's FP64 pipe once per tz intervals (up to 128)
// instead of once per 8; every interval's element is then formed on the FP32 pipe and
// stored in coalesced 16-byte rows.  tz is chosen per launch so that the grid has about
// eight CTAs per SM at every dimension (the single-kernel form had one CTA per 32
// columns and 8 intervals: a quarter of a wave at small d).
//
// omega_norm_df_kernel: the norm bound from the stored values, in the single-kernel
// form's order (per column, rows i = w mod 8 summed in double, then the eight partial
// sums in order, then the max over columns as an integer atomic).
constexpr int OT_ROWS = 8, OT_COLS = 32, OT_TZ = 128, OT_KMAX = 8;

template <int KP1>
__global__ void __launch_bounds__(256)
omega_tile_df_kernel(int N, int d, double dt, const double* __restrict__ H0, const double* __restrict__ Hk,
                     const double* __restrict__ c, const double* __restrict__ tr, float4* __restrict__ omega,
                     double* __restrict__ tau_out, int shift, int tz) {
  constexpr int K = KP1 - 1;
  __shared__ df32 cs[OT_TZ][K > 0 ? K : 1];
  __shared__ df32 mtau[OT_TZ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * OT_COLS + lane;
  const int row = blockIdx.y * OT_ROWS + warp;
  const int n0 = blockIdx.z * tz;
  const int nb = min(tz, N - n0);
  for (int t = threadIdx.x; t < tz * K; t += blockDim.x) {
    const int b = t / K, k = t % K;
    cs[b][k] = df_from_double(b < nb ? c[(long long)(n0 + b) * K + k] : 0.0);
  }
  if (threadIdx.x < tz) {
    const int b = threadIdx.x;
    double t = 0.0;
    if (shift && b < nb) {
      t = dt * tr[0];
      for (int k = 0; k < K; ++k) t += c[(long long)(n0 + b) * K + k] * tr[1 + k];
      t /= d;
    }
    mtau[b] = df_from_double(-t);
    if (b < nb && blockIdx.x == 0 && blockIdx.y == 0 && tau_out) tau_out[n0 + b] = t;
  }
  // the thread's element (row, j): its operator entries as FP32 pairs
  const df32 dtd = df_from_double(dt);
  const long long dd = (long long)d * d;
  const bool in = row < d && j < d;
  df32 r0{0.f, 0.f}, q0{0.f, 0.f}, hr[K > 0 ? K : 1], hq[K > 0 ? K : 1];
  unsigned nz = 0u;
  if (in) {
    const long long off = 2 * ((long long)row * d + j);
    const double2 h0 = *reinterpret_cast<const double2*>(H0 + off);
    r0 = df_mul(df_from_double(h0.x), dtd);
    q0 = df_mul(df_from_double(h0.y), dtd);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double2 hk = *reinterpret_cast<const double2*>(Hk + 2 * dd * k + off);
      hr[k] = df_from_double(hk.x);
      hq[k] = df_from_double(hk.y);
      if (((__double_as_longlong(hk.x) | __double_as_longlong(hk.y)) << 1) != 0) nz |= 1u << k;   // sparse H_k
    }
  }
  __syncthreads();
  if (!in) return;
  float4* o = omega + (long long)n0 * dd + (long long)row * d + j;
  for (int b = 0; b < nb; ++b) {
    df32 re = r0, im = q0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (nz & (1u << k)) {
        const df32 ck = cs[b][k];
        re = dfx_add(re, df_mul(hr[k], ck));
        im = dfx_add(im, df_mul(hq[k], ck));
      }
    }
    if (row == j) re = df_add(re, mtau[b]);
    o[b * dd] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// grid (ceil(d / 32), N), block 256; norm_bits zeroed before
__global__ void __launch_bounds__(256)
omega_norm_df_kernel(int d, const float4* __restrict__ omega, unsigned long long* __restrict__ norm_bits) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int n = blockIdx.y;
  const float4* ob = omega + (long long)n * d * d;
  double s = 0.0;
  if (j < d) {
    for (int i = warp; i < d; i += 8) {
      const float4 v = ob[(long long)i * d + j];
      s += (double)magnitude_upper_f(v.x, v.z);
    }
  }
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += part[w][lane];
    if (j >= d) v = 0.0;
    if (!(v <= 1.0e300)) v = __longlong_as_double(0x7ff0000000000000LL);   // NaN/Inf -> +Inf before the max
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomicMax(norm_bits + n, nonneg_bits(v));
  }
}

template <int KP1>
static int launch_omega_tiles(int N, int d, double dt, const double* H0, const double* Hk, const double* c,
                              const double* tr, float4* omega, double* tau, unsigned long long* bits, int shift,
                              cudaStream_t s) {
  // intervals per CTA: about eight CTAs per SM (152 SMs), at most OT_TZ
  const long long tiles = (long long)ceil_div(d, OT_COLS) * ceil_div(d, OT_ROWS);
  const long long want = 8LL * 152;
  int tz = (int)std::min<long long>(OT_TZ, std::max<long long>(1, (tiles * N + want - 1) / want));
  dim3 grid(ceil_div(d, OT_COLS), ceil_div(d, OT_ROWS), ceil_div(N, tz));
  omega_tile_df_kernel<KP1><<<grid, 256, 0, s>>>(N, d, dt, H0, Hk, c, tr, omega, tau, shift, tz);
  MG_TRY(check_launch("omega_tile_df_kernel"));
  omega_norm_df_kernel<<<dim3(ceil_div(d, 32), N), 256, 0, s>>>(d, omega, bits);
  return check_launch("omega_norm_df_kernel");
}

__global__ void bits_to_double_kernel(int n, const unsigned long long* bits, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __longlong_as_double((long long)bits[i]);
}

int launch_build_omega(int N, int d, int K, double dt, const double* H0, const double* Hk,
                       const double* c, double* omega, double* tau, double* norm1, int shift,
                       int write_shifted, double* scratch, cudaStream_t s, int out_df32) {
  // scratch: (K+1) traces + N norm words
  if (N <= 0) return MG_OK;
  double* tr = scratch;
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(scratch + (K + 1));
  operator_traces_kernel<<<K + 1, 256, 0, s>>>(d, K, H0, Hk, tr);
  MG_TRY(check_launch("operator_traces_kernel"));
  MG_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * N, s));
  dim3 grid(ceil_div(d, OMEGA_COLS), ceil_div(N, OMEGA_NB));
  size_t smem = sizeof(double) * (OMEGA_NB * (K > 0 ? K : 1) + OMEGA_NB + OMEGA_WARPS * OMEGA_NB * 32);
  if (out_df32 && K + 1 <= OT_KMAX && N <= 65535) {   // N: grid y of the norm kernel
    if (!write_shifted) return MG_EINVAL;
    float4* o4 = reinterpret_cast<float4*>(omega);
    switch (K + 1) {
      case 1: MG_TRY(launch_omega_tiles<1>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 2: MG_TRY(launch_omega_tiles<2>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 3: MG_TRY(launch_omega_tiles<3>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 4: MG_TRY(launch_omega_tiles<4>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 5: MG_TRY(launch_omega_tiles<5>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 6: MG_TRY(launch_omega_tiles<6>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      case 7: MG_TRY(launch_omega_tiles<7>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
      default: MG_TRY(launch_omega_tiles<8>(N, d, dt, H0, Hk, c, tr, o4, tau, bits, shift, s)); break;
    }
  } else if (out_df32) {
    if (!write_shifted) return MG_EINVAL;
    MG_TRY(ensure_smem_limit(reinterpret_cast<const void*>(build_omega_df_kernel), (int)smem));
    build_omega_df_kernel<<<grid, 256, smem, s>>>(N, d, K, dt, H0, Hk, c, tr, reinterpret_cast<float4*>(omega), tau,
                                                 bits, shift);
    MG_TRY(check_launch("build_omega_df_kernel"));
  } else {
    MG_TRY(ensure_smem_limit(reinterpret_cast<const void*>(build_omega_kernel), (int)smem));
    build_omega_kernel<<<grid, 256, smem, s>>>(N, d, K, dt, H0, Hk, c, tr, omega, tau, bits, shift,
                                              write_shifted);
    MG_TRY(check_launch("build_omega_kernel"));
  }
  if (norm1) {
    bits_to_double_kernel<<<ceil_div(N, 256), 256, 0, s>>>(N, bits, norm1);
    MG_TRY(check_launch("bits_to_double_kernel"));
  }
  return MG_OK;
}

// ---------------------------------------------------------------------------
// General Hermitian input (mg_expm): tau_b = Re tr(A_b)/d, dst = A_b - tau_b I,
// norm1_b = ||dst||_1.  grid (ceil(d/32), batch), block 256.
__global__ void __launch_bounds__(256)
shift_norm_kernel(int d, const double* __restrict__ A, double* __restrict__ dst,
                  const double* __restrict__ tau, unsigned long long* __restrict__ norm_bits) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const long long base = (long long)blockIdx.y * d * d * 2;
  const double t = tau[blockIdx.y];
  double s = 0.0;
  if (j < d) {
    for (int i = warp; i < d; i += 8) {
      long long off = base + 2 * ((long long)i * d + j);
      double2 v = *reinterpret_cast<const double2*>(A + off);
      if (i == j) v.x -= t;
      s += hypot(v.x, v.y);
      *reinterpret_cast<double2*>(dst + off) = v;
    }
  }
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += part[w][lane];
    if (!(v <= 1.0e300)) v = __longlong_as_double(0x7ff0000000000000LL);   // before fmax drops a NaN
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomicMax(norm_bits + blockIdx.y, nonneg_bits(v));
  }
}

__global__ void batch_trace_kernel(int d, const double* __restrict__ A, double* __restrict__ tau) {
  const long long base = (long long)blockIdx.x * d * d * 2;
  double acc = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) acc += A[base + 2 * ((long long)i * d + i)];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) tau[blockIdx.x] = red[0] / d;
}

int launch_shift_norm(int batch, int d, const double* A, double* dst, double* tau, double* norm1,
                      unsigned long long* bits, int shift, cudaStream_t s) {
  if (shift) {
    batch_trace_kernel<<<batch, 256, 0, s>>>(d, A, tau);
    MG_TRY(check_launch("batch_trace_kernel"));
  } else {
    MG_CUDA_TRY(cudaMemsetAsync(tau, 0, sizeof(double) * batch, s));
  }
  MG_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * batch, s));
  shift_norm_kernel<<<dim3(ceil_div(d, 32), batch), 256, 0, s>>>(d, A, dst, tau, bits);
  MG_TRY(check_launch("shift_norm_kernel"));
  bits_to_double_kernel<<<ceil_div(batch, 256), 256, 0, s>>>(batch, bits, norm1);
  return check_launch("bits_to_double_kernel");
}

// ---------------------------------------------------------------------------
// Hermiticity check of a stack of operators: out[0] = max |H - H^dag|, out[1] = max |H|
__global__ void hermitian_defect_kernel(int d, int count, const double* __restrict__ H,
                                        unsigned long long* __restrict__ out) {
  long long total = (long long)count * d * d;
  double dmax = 0.0, hmax = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long m = e / ((long long)d * d);
    long long r = e % ((long long)d * d);
    int i = (int)(r / d), j = (int)(r % d);
    const double* M = H + m * d * d * 2;
    double ar = M[2 * ((long long)i * d + j)], ai = M[2 * ((long long)i * d + j) + 1];
    double br = M[2 * ((long long)j * d + i)], bi = -M[2 * ((long long)j * d + i) + 1];
    dmax = fmax(dmax, hypot(ar - br, ai - bi));
    hmax = fmax(hmax, hypot(ar, ai));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    hmax = fmax(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, nonneg_bits(dmax));
    atomicMax(out + 1, nonneg_bits(hmax));
  }
}

int launch_hermitian_defect(int d, int count, const double* H, unsigned long long* out, cudaStream_t s) {
  MG_CUDA_TRY(cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s));
  if (count <= 0) return MG_OK;
  hermitian_defect_kernel<<<304, 256, 0, s>>>(d, count, H, out);
  return check_launch("hermitian_defect_kernel");
}

// Structure of a stack of `count` d x d complex operators: *out |= 1 if an entry has a
// nonzero imaginary part, |= 2 if a real part differs from its transpose's (out preset to
// 0).  Real operators keep every Hbar_n of the first-order term real; real symmetric ones
// make every polynomial in X_n = -i 2^-s (Hbar_n - tau_n I) complex symmetric.
__global__ void operator_structure_kernel(int d, long long count, const double* __restrict__ M,
                                          int* __restrict__ out) {
  const long long dd = (long long)d * d, n = count * dd;
  int bits = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long m = e / dd, r = e % dd;
    const long long i = r / d, j = r % d;
    if (M[2 * e + 1] != 0.0) bits |= 1;
    if (M[2 * e] != M[2 * (m * dd + j * d + i)]) bits |= 2;
  }
  for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(out, bits);
}

int launch_operator_structure(int d, long long count, const double* M, int* out, cudaStream_t s) {
  if (count <= 0) return MG_OK;
  operator_structure_kernel<<<304, 256, 0, s>>>(d, count, M, out);
  return check_launch("operator_structure_kernel");
}

}  // namespace mg
