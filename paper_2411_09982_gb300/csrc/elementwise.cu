// Elementwise and reduction kernels of the exponential and propagation steps
// (FP64, HBM-bound): scaling X = -i 2^{-s} Hbar, linear combinations of matrix
// powers for the Taylor polynomial, the exact trace-shift phase e^{-i tau},
// identities and strided copies, and the FP64 unitarity/norm diagnostics.
#include "common.cuh"
#include "df32.cuh"

#include <algorithm>
#include <cmath>

namespace mg {

// ---------------------------------------------------------------------------
__global__ void scale_minus_i_kernel(long long per_item, int batch, const double* __restrict__ src,
                                     double* __restrict__ dst, const int* __restrict__ sq_dev, int sq) {
  long long total = per_item * batch;  // complex elements
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / per_item);
    int s = sq_dev ? sq_dev[b] : sq;
    const double f = __longlong_as_double((long long)(1023 - s) << 52);   // 2^{-s}, 0 <= s < 1023
    double2 v = reinterpret_cast<const double2*>(src)[e];
    // (-i)(a + i b) = b - i a
    reinterpret_cast<double2*>(dst)[e] = make_double2(f * v.y, -f * v.x);
  }
}

static int grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

int launch_scale_minus_i(int batch, int d, const double* src, double* dst, const int* sq_dev, int sq,
                         cudaStream_t s) {
  long long per = (long long)d * d;
  scale_minus_i_kernel<<<grid_for(per * batch), 256, 0, s>>>(per, batch, src, dst, sq_dev, sq);
  return check_launch("scale_minus_i_kernel");
}

// ---------------------------------------------------------------------------
struct LincombArgs {
  const double* src[4];
  double coef[4];
};

__global__ void lincomb_kernel(int d, int batch, int nsrc, LincombArgs a, double diag,
                               double* __restrict__ dst) {
  const long long per = (long long)d * d;
  const long long total = per * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int m = 0; m < nsrc; ++m) {
      double2 v = reinterpret_cast<const double2*>(a.src[m])[e];
      re = fma(a.coef[m], v.x, re);
      im = fma(a.coef[m], v.y, im);
    }
    long long r = e % per;
    if (r / d == r % d) re += diag;
    reinterpret_cast<double2*>(dst)[e] = make_double2(re, im);
  }
}

int launch_lincomb(int batch, int d, double* dst, int nsrc, const double* const* src, const double* coef,
                   double diag, cudaStream_t s) {
  if (nsrc < 0 || nsrc > 4) return MG_EINVAL;
  LincombArgs a{};
  for (int m = 0; m < nsrc; ++m) { a.src[m] = src[m]; a.coef[m] = coef[m]; }
  lincomb_kernel<<<grid_for((long long)d * d * batch), 256, 0, s>>>(d, batch, nsrc, a, diag, dst);
  return check_launch("lincomb_kernel");
}

// Several linear combinations of the same sources in one pass: dst_o =
// sum_m coef[o][m] src_m + diag[o] I for o < nout (nout <= 5, nsrc <= 4).  Every
// thread reads all sources of its element before writing, so a destination may
// alias a source.
struct LincombMultiArgs {
  const double* src[4];
  double* dst[5];
  double coef[5][4];
  double diag[5];
};

__global__ void lincomb_multi_kernel(int d, long long total, int nsrc, int nout, LincombMultiArgs a) {
  const long long per = (long long)d * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double2 v[4];
    for (int m = 0; m < nsrc; ++m) v[m] = reinterpret_cast<const double2*>(a.src[m])[e];
    const long long r = e % per;
    const bool on_diag = r / d == r % d;
    for (int o = 0; o < nout; ++o) {
      double re = on_diag ? a.diag[o] : 0.0, im = 0.0;
      for (int m = 0; m < nsrc; ++m) {
        re = fma(a.coef[o][m], v[m].x, re);
        im = fma(a.coef[o][m], v[m].y, im);
      }
      reinterpret_cast<double2*>(a.dst[o])[e] = make_double2(re, im);
    }
  }
}

int launch_lincomb_multi(int batch, int d, int nout, double* const* dst, int nsrc, const double* const* src,
                         const double* coef, const double* diag, cudaStream_t s) {
  if (nsrc < 1 || nsrc > 4 || nout < 1 || nout > 5) return MG_EINVAL;
  LincombMultiArgs a{};
  for (int m = 0; m < nsrc; ++m) a.src[m] = src[m];
  for (int o = 0; o < nout; ++o) {
    a.dst[o] = dst[o];
    a.diag[o] = diag[o];
    for (int m = 0; m < nsrc; ++m) a.coef[o][m] = coef[o * nsrc + m];
  }
  const long long total = (long long)d * d * batch;
  lincomb_multi_kernel<<<grid_for(total), 256, 0, s>>>(d, total, nsrc, nout, a);
  return check_launch("lincomb_multi_kernel");
}

// dst[p] = src[idx[p]] for p < n matrices of md doubles (gathering the operand
// pairs of a segmented tree product into contiguous batches)
__global__ void gather_mats_kernel(int n, long long md2, const double2* __restrict__ src, const int* __restrict__ idx,
                                   double2* __restrict__ dst) {
  const long long total = md2 * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / md2, r = e - p * md2;
    dst[e] = src[(long long)idx[p] * md2 + r];
  }
}

int launch_gather_mats(int n, long long md, const double* src, const int* idx_dev, double* dst, cudaStream_t s) {
  if (n <= 0) return MG_OK;
  const long long md2 = md / 2;
  gather_mats_kernel<<<grid_for(md2 * n), 256, 0, s>>>(n, md2, reinterpret_cast<const double2*>(src), idx_dev,
                                                        reinterpret_cast<double2*>(dst));
  return check_launch("gather_mats_kernel");
}

// ---------------------------------------------------------------------------
// grid (chunks, batch): the phase factor is formed once per block, not per element.
__global__ void apply_phase_kernel(long long per_item, const double* __restrict__ phase,
                                   const double* __restrict__ src, double* __restrict__ dst) {
  __shared__ double cs_sn[2];
  const int b = blockIdx.y;
  if (threadIdx.x == 0) sincos(phase[b], &cs_sn[1], &cs_sn[0]);
  __syncthreads();
  const double cs = cs_sn[0], sn = cs_sn[1];
  const double2* sb = reinterpret_cast<const double2*>(src) + (long long)b * per_item;
  double2* db = reinterpret_cast<double2*>(dst) + (long long)b * per_item;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per_item;
       e += (long long)gridDim.x * blockDim.x) {
    // e^{-i p} (x + i y) = (c - i s)(x + i y)
    const double2 v = sb[e];
    db[e] = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);
  }
}

int launch_apply_phase(int batch, int d, long long count_per_item, const double* phase, const double* src,
                       double* dst, cudaStream_t s) {
  (void)d;
  if (batch > 65535) return MG_EUNSUPPORTED;
  long long bx = (count_per_item + 1023) / 1024;
  if (bx > 64) bx = 64;
  apply_phase_kernel<<<dim3((unsigned)bx, batch), 256, 0, s>>>(count_per_item, phase, src, dst);
  return check_launch("apply_phase_kernel");
}

// ---------------------------------------------------------------------------
__global__ void identity_kernel(int d, int batch, double* __restrict__ dst) {
  const long long per = (long long)d * d;
  const long long total = per * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e % per;
    reinterpret_cast<double2*>(dst)[e] = make_double2((r / d == r % d) ? 1.0 : 0.0, 0.0);
  }
}

int launch_identity(int batch, int d, double* dst, cudaStream_t s) {
  identity_kernel<<<grid_for((long long)d * d * batch), 256, 0, s>>>(d, batch, dst);
  return check_launch("identity_kernel");
}

__global__ void copy_strided_kernel(int batch, long long elems, const double* __restrict__ src,
                                    long long ss, double* __restrict__ dst, long long ds) {
  const long long total = elems * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long b = e / elems, r = e % elems;
    dst[b * ds + r] = src[b * ss + r];
  }
}

int launch_copy_strided(int batch, long long elems, const double* src, long long src_stride, double* dst,
                        long long dst_stride, cudaStream_t s) {
  copy_strided_kernel<<<grid_for(elems * batch), 256, 0, s>>>(batch, elems, src, src_stride, dst, dst_stride);
  return check_launch("copy_strided_kernel");
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void identity_defect_kernel(int d, int batch, const double* __restrict__ G, double* out) {
  const long long per = (long long)d * d;
  const long long total = per * batch;
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e % per;
    double2 v = reinterpret_cast<const double2*>(G)[e];
    if (r / d == r % d) v.x -= 1.0;
    m = fmax(m, hypot(v.x, v.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

int launch_max_identity_defect(int batch, int d, const double* G, double* out_dev, cudaStream_t s) {
  MG_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(double), s));
  identity_defect_kernel<<<grid_for((long long)d * d * batch), 256, 0, s>>>(d, batch, G, out_dev);
  return check_launch("identity_defect_kernel");
}

// ---------------------------------------------------------------------------
// double-float (DF32) versions used by the split-precision path
// ---------------------------------------------------------------------------
// X = (-i) 2^{-sq} src: FP64 in, DF32 out
// Grid of the per-item double-float kernels: y = batch item, x strides over the
// item's d^2 elements, so that the element index and the diagonal test (r is on the
// diagonal iff r % (d + 1) == 0) stay 32-bit: no 64-bit division per element.
static dim3 item_grid(int batch, long long per) {
  long long gx = (per + 255) / 256;
  const long long cap = std::max<long long>(1, (152LL * 32) / std::max(1, batch));
  if (gx > cap) gx = cap;
  return dim3((unsigned)std::max<long long>(gx, 1), (unsigned)batch);
}

// lower-block storage of a symmetric matrix (see split_gemm.cu): with `lower`, the
// per-element kernels below touch only the 32 x 32 blocks on and below the diagonal
__device__ __forceinline__ bool outside_lower(int lower, int r, int d) {
  if (!lower) return false;
  const int i = r / d, j = r - i * d;
  return (j >> 5) > (i >> 5);
}

__global__ void scale_minus_i_df_kernel(int per, const double* __restrict__ src, float4* __restrict__ dst, double f,
                                        const int* __restrict__ sq_dev) {
  const long long base = (long long)blockIdx.y * per;
  // 2^{-s} exactly (0 <= s < 1023)
  const double g = sq_dev ? __longlong_as_double((long long)(1023 - sq_dev[blockIdx.y]) << 52) : f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < per; r += gridDim.x * blockDim.x) {
    const double2 v = reinterpret_cast<const double2*>(src)[base + r];
    const df32 re = df_from_double(g * v.y), im = df_from_double(-g * v.x);
    dst[base + r] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// the same from a double-float W: (-i)(a + i b) 2^{-s} = (b - i a) 2^{-s}, exact on the FP32 pipe
__global__ void scale_minus_i_dfdf_kernel(int per, const float4* __restrict__ src, float4* __restrict__ dst, int sq,
                                          const int* __restrict__ sq_dev, int d, int lower) {
  const long long base = (long long)blockIdx.y * per;
  const int s = sq_dev ? sq_dev[blockIdx.y] : sq;
  const int s1 = s / 2, s2 = s - s1;   // two factors keep each in range
  const float f1 = __int_as_float((127 - s1) << 23), f2 = __int_as_float((127 - s2) << 23);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < per; r += gridDim.x * blockDim.x) {
    if (outside_lower(lower, r, d)) continue;
    const float4 v = src[base + r];
    dst[base + r] = make_float4((v.z * f1) * f2, (v.w * f1) * f2, -(v.x * f1) * f2, -(v.y * f1) * f2);
  }
}

int launch_scale_minus_i_df(int batch, int d, const double* src, double* dst_df, int sq, cudaStream_t s,
                            const int* sq_dev, int in_df32, int lower) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  const dim3 grid = item_grid(batch, (long long)d * d);
  if (in_df32) {
    scale_minus_i_dfdf_kernel<<<grid, 256, 0, s>>>(d * d, reinterpret_cast<const float4*>(src),
                                                   reinterpret_cast<float4*>(dst_df), sq, sq_dev, d, lower);
    return check_launch("scale_minus_i_dfdf_kernel");
  }
  const double f = std::ldexp(1.0, -sq);
  scale_minus_i_df_kernel<<<grid, 256, 0, s>>>(d * d, src, reinterpret_cast<float4*>(dst_df), f, sq_dev);
  return check_launch("scale_minus_i_df_kernel");
}

// x + y in double-float with one fewer error-free step than df_add (error below
// ~2^-46 of |x| + |y|; the combinations below add terms of like size)
__device__ __forceinline__ df32 df_add_fast(df32 x, df32 y) {
  const df32 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

struct LincombDfArgs {
  const float4* src[4];
  df32 coef[4];
};

__global__ void lincomb_df_kernel(int d, int nsrc, LincombDfArgs a, df32 diag, float4* __restrict__ dst, int lower) {
  const int per = d * d;
  const long long base = (long long)blockIdx.y * per;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < per; r += gridDim.x * blockDim.x) {
    if (outside_lower(lower, r, d)) continue;
    const long long e = base + r;
    df32 re{0.f, 0.f}, im{0.f, 0.f};
    for (int m = 0; m < nsrc; ++m) {
      const float4 v = a.src[m][e];
      re = df_add(re, df_mul(df32{v.x, v.y}, a.coef[m]));
      im = df_add(im, df_mul(df32{v.z, v.w}, a.coef[m]));
    }
    if (r % (d + 1) == 0) re = df_add(re, diag);
    dst[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

int launch_lincomb_df(int batch, int d, double* dst, int nsrc, const double* const* src, const double* coef,
                      double diag, cudaStream_t s, int lower) {
  if (nsrc < 0 || nsrc > 4) return MG_EINVAL;
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  LincombDfArgs a{};
  for (int m = 0; m < nsrc; ++m) {
    a.src[m] = reinterpret_cast<const float4*>(src[m]);
    a.coef[m] = df_from_double(coef[m]);
  }
  lincomb_df_kernel<<<item_grid(batch, (long long)d * d), 256, 0, s>>>(d, nsrc, a, df_from_double(diag),
                                                                       reinterpret_cast<float4*>(dst), lower);
  return check_launch("lincomb_df_kernel");
}

// the multi-output combination in double-float (see lincomb_multi_kernel)
struct LincombMultiDfArgs {
  const float4* src[4];
  float4* dst[5];
  df32 coef[5][4];
  df32 diag[5];
};

template <int NSRC>
__global__ void lincomb_multi_df_kernel(int d, int nout, LincombMultiDfArgs a, int lower) {
  const int per = d * d;
  const long long base = (long long)blockIdx.y * per;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < per; r += gridDim.x * blockDim.x) {
    if (outside_lower(lower, r, d)) continue;
    const long long e = base + r;
    float4 v[NSRC];
#pragma unroll
    for (int m = 0; m < NSRC; ++m) v[m] = a.src[m][e];
    const bool on_diag = r % (d + 1) == 0;
    for (int o = 0; o < nout; ++o) {
      df32 re = df_mul(df32{v[0].x, v[0].y}, a.coef[o][0]), im = df_mul(df32{v[0].z, v[0].w}, a.coef[o][0]);
#pragma unroll
      for (int m = 1; m < NSRC; ++m) {
        re = df_add_fast(re, df_mul(df32{v[m].x, v[m].y}, a.coef[o][m]));
        im = df_add_fast(im, df_mul(df32{v[m].z, v[m].w}, a.coef[o][m]));
      }
      if (on_diag) re = df_add(re, a.diag[o]);
      a.dst[o][e] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  }
}

int launch_lincomb_multi_df(int batch, int d, int nout, double* const* dst, int nsrc, const double* const* src,
                            const double* coef, const double* diag, cudaStream_t s, int lower) {
  if (nsrc < 1 || nsrc > 4 || nout < 1 || nout > 5) return MG_EINVAL;
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  LincombMultiDfArgs a{};
  for (int m = 0; m < nsrc; ++m) a.src[m] = reinterpret_cast<const float4*>(src[m]);
  for (int o = 0; o < nout; ++o) {
    a.dst[o] = reinterpret_cast<float4*>(dst[o]);
    a.diag[o] = df_from_double(diag[o]);
    for (int m = 0; m < nsrc; ++m) a.coef[o][m] = df_from_double(coef[o * nsrc + m]);
  }
  const dim3 grid = item_grid(batch, (long long)d * d);
  switch (nsrc) {
    case 1: lincomb_multi_df_kernel<1><<<grid, 256, 0, s>>>(d, nout, a, lower); break;
    case 2: lincomb_multi_df_kernel<2><<<grid, 256, 0, s>>>(d, nout, a, lower); break;
    case 3: lincomb_multi_df_kernel<3><<<grid, 256, 0, s>>>(d, nout, a, lower); break;
    default: lincomb_multi_df_kernel<4><<<grid, 256, 0, s>>>(d, nout, a, lower); break;
  }
  return check_launch("lincomb_multi_df_kernel");
}

// dst_b = e^{-i phase_b} src_b in DF32; the phase factor is formed once per block in FP64
__global__ void apply_phase_df_kernel(long long per_item, const double* __restrict__ phase,
                                      const float4* __restrict__ src, float4* __restrict__ dst) {
  __shared__ df32 cs_sn[2];
  const int b = blockIdx.y;
  if (threadIdx.x == 0) {
    double sn, cs;
    sincos(phase[b], &sn, &cs);
    cs_sn[0] = df_from_double(cs);
    cs_sn[1] = df_from_double(sn);
  }
  __syncthreads();
  const df32 c = cs_sn[0], sn = cs_sn[1], msn = df_neg(cs_sn[1]);
  const float4* sb = src + (long long)b * per_item;
  float4* db = dst + (long long)b * per_item;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per_item;
       e += (long long)gridDim.x * blockDim.x) {
    const float4 v = sb[e];
    const df32 x{v.x, v.y}, y{v.z, v.w};
    // (c - i s)(x + i y) = (c x + s y) + i (c y - s x)
    const df32 re = df_add(df_mul(x, c), df_mul(y, sn));
    const df32 im = df_add(df_mul(y, c), df_mul(x, msn));
    db[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// The same from a symmetric src in lower-block storage into a full dst: entry (i, j) with
// j > i is taken from (j, i), also inside the diagonal blocks, so dst is exactly
// symmetric.  One 32 x 32 block per CTA (its own, or its transposed partner, staged in
// shared memory): grid (ceil(d/32), ceil(d/32), batch), 256 threads.
__global__ void apply_phase_sym_df_kernel(int d, const double* __restrict__ phase, const float4* __restrict__ src,
                                          float4* __restrict__ dst) {
  __shared__ float4 t[32][33];
  __shared__ df32 cs_sn[2];
  const int bj = blockIdx.x, bi = blockIdx.y, b = blockIdx.z;
  const long long per = (long long)d * d;
  const float4* sb = src + b * per;
  float4* db = dst + b * per;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = bi * 32, j0 = bj * 32;
  if (threadIdx.x == 0) {
    double sn, cs;
    sincos(phase[b], &sn, &cs);
    cs_sn[0] = df_from_double(cs);
    cs_sn[1] = df_from_double(sn);
  }
  for (int r = ty; r < 32; r += 8) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (bj <= bi) {   // t[r][tx] = src[i0 + r][j0 + tx]
      if (i0 + r < d && j0 + tx < d) v = sb[(long long)(i0 + r) * d + j0 + tx];
      t[r][tx] = v;
    } else {          // t[tx][r] = src[j0 + r][i0 + tx]
      if (j0 + r < d && i0 + tx < d) v = sb[(long long)(j0 + r) * d + i0 + tx];
      t[tx][r] = v;
    }
  }
  __syncthreads();
  const df32 c = cs_sn[0], sn = cs_sn[1], msn = df_neg(cs_sn[1]);
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    if (i >= d || j >= d) continue;
    const float4 v = (bi == bj && tx > r) ? t[tx][r] : t[r][tx];
    const df32 x{v.x, v.y}, y{v.z, v.w};
    // (c - i s)(x + i y) = (c x + s y) + i (c y - s x)
    const df32 re = df_add(df_mul(x, c), df_mul(y, sn));
    const df32 im = df_add(df_mul(y, c), df_mul(x, msn));
    db[(long long)i * d + j] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

int launch_apply_phase_sym_df(int batch, int d, const double* phase, const double* src, double* dst, cudaStream_t s) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  const int nb = (d + 31) / 32;
  apply_phase_sym_df_kernel<<<dim3(nb, nb, batch), 256, 0, s>>>(d, phase, reinterpret_cast<const float4*>(src),
                                                                reinterpret_cast<float4*>(dst));
  return check_launch("apply_phase_sym_df_kernel");
}

int launch_apply_phase_df(int batch, int d, const double* phase, const double* src, double* dst, cudaStream_t s) {
  if (batch > 65535) return MG_EUNSUPPORTED;
  const long long per = (long long)d * d;
  long long bx = (per + 1023) / 1024;
  if (bx > 64) bx = 64;
  apply_phase_df_kernel<<<dim3((unsigned)bx, batch), 256, 0, s>>>(per, phase, reinterpret_cast<const float4*>(src),
                                                                  reinterpret_cast<float4*>(dst));
  return check_launch("apply_phase_df_kernel");
}

__global__ void identity_df_kernel(int d, long long total, float4* __restrict__ dst) {
  const long long per = (long long)d * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % per;
    dst[e] = make_float4((r / d == r % d) ? 1.f : 0.f, 0.f, 0.f, 0.f);
  }
}

int launch_identity_df(int batch, int d, double* dst, cudaStream_t s) {
  const long long total = (long long)d * d * batch;
  identity_df_kernel<<<grid_for(total), 256, 0, s>>>(d, total, reinterpret_cast<float4*>(dst));
  return check_launch("identity_df_kernel");
}

__global__ void df_to_fp64_kernel(long long per, long long total, const float4* __restrict__ src, long long ss,
                                  double2* __restrict__ dst, long long ds) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per, r = e % per;
    const float4 v = src[b * ss + r];
    dst[b * ds + r] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

__global__ void fp64_to_df_kernel(long long per, long long total, const double2* __restrict__ src, long long ss,
                                  float4* __restrict__ dst, long long ds) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per, r = e % per;
    const double2 v = src[b * ss + r];
    const df32 re = df_from_double(v.x), im = df_from_double(v.y);
    dst[b * ds + r] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// strides in doubles (two per complex element in either format)
int launch_df_to_fp64(int batch, int d, const double* src, long long ss, double* dst, long long ds, cudaStream_t s) {
  const long long per = (long long)d * d, total = per * batch;
  df_to_fp64_kernel<<<grid_for(total), 256, 0, s>>>(per, total, reinterpret_cast<const float4*>(src), ss / 2,
                                                    reinterpret_cast<double2*>(dst), ds / 2);
  return check_launch("df_to_fp64_kernel");
}

int launch_fp64_to_df(int batch, int d, const double* src, long long ss, double* dst, long long ds, cudaStream_t s) {
  const long long per = (long long)d * d, total = per * batch;
  fp64_to_df_kernel<<<grid_for(total), 256, 0, s>>>(per, total, reinterpret_cast<const double2*>(src), ss / 2,
                                                    reinterpret_cast<float4*>(dst), ds / 2);
  return check_launch("fp64_to_df_kernel");
}

// ---------------------------------------------------------------------------
// zero padding of operators to a bucket dimension (exact: exp of a block-diagonal
// matrix with a zero block is the identity on that block)
__global__ void pad_copy_kernel(long long total, int d, int dp, const double2* __restrict__ src,
                                double2* __restrict__ dst) {
  const long long per = (long long)dp * dp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long m = e / per, r = e % per;
    const int i = (int)(r / dp), j = (int)(r % dp);
    dst[e] = (i < d && j < d) ? src[m * (long long)d * d + (long long)i * d + j] : make_double2(0.0, 0.0);
  }
}

int launch_pad_copy(int count, int d, int dp, const double* src, double* dst, cudaStream_t s) {
  const long long total = (long long)count * dp * dp;
  if (total == 0) return MG_OK;
  pad_copy_kernel<<<grid_for(total), 256, 0, s>>>(total, d, dp, reinterpret_cast<const double2*>(src),
                                                 reinterpret_cast<double2*>(dst));
  return check_launch("pad_copy_kernel");
}

__global__ void unpad_copy_kernel(int d, int dp, const double2* __restrict__ src, double2* __restrict__ dst) {
  const long long total = (long long)d * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    dst[e] = src[(long long)i * dp + j];
  }
}

int launch_unpad_copy(int d, int dp, const double* src, double* dst, cudaStream_t s) {
  unpad_copy_kernel<<<grid_for((long long)d * d), 256, 0, s>>>(d, dp, reinterpret_cast<const double2*>(src),
                                                                reinterpret_cast<double2*>(dst));
  return check_launch("unpad_copy_kernel");
}

__global__ void pad_into_kernel(int d, int dp, const double2* __restrict__ src, double2* __restrict__ dst) {
  const long long total = (long long)d * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    dst[(long long)i * dp + j] = src[e];
  }
}

int launch_pad_into(int d, int dp, const double* src, double* dst, cudaStream_t s) {
  pad_into_kernel<<<grid_for((long long)d * d), 256, 0, s>>>(d, dp, reinterpret_cast<const double2*>(src),
                                                              reinterpret_cast<double2*>(dst));
  return check_launch("pad_into_kernel");
}

}  // namespace mg
