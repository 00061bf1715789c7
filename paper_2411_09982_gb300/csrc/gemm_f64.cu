// Native-FP64 batched complex matrix product (the MG_PREC_FP64 path and the
// FP64 re-orthonormalisation).
//
//   C[b] = scale * opA(A[b]) * B[b] + sum_m coef_m P_m[b] + diag * I
//
// with opA = identity or conjugate transpose.  GB300's FP64 throughput is a
// small fraction of its tensor-core throughput, so this kernel is ALU-bound on
// the FP64 pipe: TM x TM complex output tiles per CTA (TM = 64, or 32 / 16 for
// small d, so that padding does not multiply the FP64 work), (TM/16)^2 complex
// outputs per thread, operands staged through shared memory in K-slabs of 8.
#include "common.cuh"

namespace mg {

constexpr int FBK = 8;

struct AddDev {
  const double* src[3];
  double coef[3];
  long long stride;
  int n;
  double diag;
  double scale;
  const int* item_sq;   // null, or per-item squaring counts: item b is skipped when item_sq[b] <= sq_step
  int sq_step;
};

template <int TM>
__global__ void __launch_bounds__(256)
cgemm_f64_kernel(int d, const double* __restrict__ A, long long sA, int opA,
                 const double* __restrict__ B, long long sB, double* __restrict__ C, long long sC,
                 AddDev add) {
  constexpr int RT = TM / 16;                   // outputs per thread along each dimension
  constexpr int STAGE = (TM * FBK + 255) / 256; // staged elements per thread per operand
  __shared__ double2 As[FBK][TM];   // As[k][i] = opA(A)[i][k]
  __shared__ double2 Bs[FBK][TM];   // Bs[k][j] = B[k][j]

  const int b = blockIdx.z;
  if (add.item_sq && add.item_sq[b] <= add.sq_step) return;   // uniform over the CTA
  const double2* Ab = reinterpret_cast<const double2*>(A + b * sA);
  const double2* Bb = reinterpret_cast<const double2*>(B + b * sB);
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TM;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  double accr[RT][RT], acci[RT][RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) { accr[r][c] = 0.0; acci[r][c] = 0.0; }

  for (int k0 = 0; k0 < d; k0 += FBK) {
#pragma unroll
    for (int t = 0; t < STAGE; ++t) {
      const int e = tid + t * 256;
      if (e >= TM * FBK) break;
      double2 v = make_double2(0.0, 0.0);
      int i, k;
      if (opA == 0) {  // A[i][k]: contiguous along k
        i = e / FBK; k = e % FBK;
        if (i0 + i < d && k0 + k < d) v = Ab[(long long)(i0 + i) * d + (k0 + k)];
      } else {         // conj(A[k][i]): contiguous along i
        k = e / TM; i = e % TM;
        if (i0 + i < d && k0 + k < d) {
          v = Ab[(long long)(k0 + k) * d + (i0 + i)];
          v.y = -v.y;
        }
      }
      As[k][i] = v;
    }
#pragma unroll
    for (int t = 0; t < STAGE; ++t) {
      const int e = tid + t * 256;
      if (e >= TM * FBK) break;
      const int k = e / TM, j = e % TM;
      double2 v = make_double2(0.0, 0.0);
      if (k0 + k < d && j0 + j < d) v = Bb[(long long)(k0 + k) * d + (j0 + j)];
      Bs[k][j] = v;
    }
    __syncthreads();
    const int kmax = min(FBK, d - k0);
#pragma unroll
    for (int k = 0; k < FBK; ++k) {
      if (k >= kmax) break;   // zero padding beyond d adds nothing
      double2 a[RT], bb[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) a[r] = As[k][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < RT; ++c) bb[c] = Bs[k][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < RT; ++c) {
          accr[r][c] = fma(a[r].x, bb[c].x, accr[r][c]);
          accr[r][c] = fma(-a[r].y, bb[c].y, accr[r][c]);
          acci[r][c] = fma(a[r].x, bb[c].y, acci[r][c]);
          acci[r][c] = fma(a[r].y, bb[c].x, acci[r][c]);
        }
    }
    __syncthreads();
  }

  double2* Cb = reinterpret_cast<double2*>(C + b * sC);
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= d) continue;
#pragma unroll
    for (int c = 0; c < RT; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= d) continue;
      const long long off = (long long)i * d + j;
      double re = add.scale * accr[r][c], im = add.scale * acci[r][c];
      for (int m = 0; m < add.n; ++m) {
        double2 p = reinterpret_cast<const double2*>(add.src[m] + b * add.stride)[off];
        re = fma(add.coef[m], p.x, re);
        im = fma(add.coef[m], p.y, im);
      }
      if (i == j) re += add.diag;
      Cb[off] = make_double2(re, im);
    }
  }
}

int launch_cgemm_f64(int batch, int d, const double* A, long long strideA, int opA, const double* B,
                     long long strideB, double* C, long long strideC, const AddTerms& add,
                     cudaStream_t s) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  AddDev a{};
  a.n = add.n;
  for (int m = 0; m < 3; ++m) { a.src[m] = add.src[m]; a.coef[m] = add.coef[m]; }
  a.stride = add.stride;
  a.diag = add.diag;
  a.scale = add.scale;
  a.item_sq = add.item_sq;
  a.sq_step = add.sq_step;
  // tile edge: the smallest of 16, 32, 64 that covers d (64 beyond)
  if (d <= 16) {
    cgemm_f64_kernel<16><<<dim3(1, 1, batch), 256, 0, s>>>(d, A, strideA, opA, B, strideB, C, strideC, a);
  } else if (d <= 32) {
    cgemm_f64_kernel<32><<<dim3(1, 1, batch), 256, 0, s>>>(d, A, strideA, opA, B, strideB, C, strideC, a);
  } else {
    dim3 grid(ceil_div(d, 64), ceil_div(d, 64), batch);
    cgemm_f64_kernel<64><<<grid, 256, 0, s>>>(d, A, strideA, opA, B, strideB, C, strideC, a);
  }
  return check_launch("cgemm_f64_kernel");
}

}  // namespace mg
