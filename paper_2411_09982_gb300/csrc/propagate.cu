// Sequential state propagation psi_{n+1} = U_n psi_n (the state form of the
// product U_{N-1} ... U_0 psi0), with the optional FP64 renormalisation
// psi <- psi / |psi| every R intervals.
//
// Small d (<= 256): one CTA carries the state through all intervals of a
// chunk: psi lives in shared memory, each warp forms whole rows of U_n psi_n
// (coalesced row reads of U_n), one barrier per interval.  The chain is
// latency-bound; its traffic is one read of every U_n.
// Large d: one multi-CTA matrix-vector launch per interval (HBM-bound).
#include "common.cuh"

namespace mg {

constexpr int CHAIN_THREADS = 1024;

// One CTA carries psi (d complex, global) through n_steps propagators.
// traj (may be null): psi after every step is also written to traj + (step_offset + n + 1) d.
__device__ void chain_body(int n_steps, int d, const double* __restrict__ U, long long sU,
                           double* __restrict__ psi, int reorth_every, int step_offset, double2* sh,
                           double* red, double* __restrict__ traj) {
  double2* cur = sh;
  double2* nxt = sh + d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < d; i += blockDim.x) cur[i] = reinterpret_cast<double2*>(psi)[i];
  __syncthreads();
  for (int n = 0; n < n_steps; ++n) {
    const double2* Un = reinterpret_cast<const double2*>(U + n * sU);
    for (int i = warp; i < d; i += nw) {
      const double2* row = Un + (long long)i * d;
      double re = 0.0, im = 0.0;
      for (int j = lane; j < d; j += 32) {
        double2 u = row[j], v = cur[j];
        re = fma(u.x, v.x, re);
        re = fma(-u.y, v.y, re);
        im = fma(u.x, v.y, im);
        im = fma(u.y, v.x, im);
      }
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) nxt[i] = make_double2(re, im);
    }
    __syncthreads();
    double2* t = cur; cur = nxt; nxt = t;
    const int done = step_offset + n + 1;
    if (reorth_every > 0 && done % reorth_every == 0) {
      double s = 0.0;
      for (int i = threadIdx.x; i < d; i += blockDim.x) s += cur[i].x * cur[i].x + cur[i].y * cur[i].y;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp] = s;
      __syncthreads();
      if (warp == 0) {
        double v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[0] = v;
      }
      __syncthreads();
      const double inv = 1.0 / sqrt(red[0]);
      for (int i = threadIdx.x; i < d; i += blockDim.x) { cur[i].x *= inv; cur[i].y *= inv; }
      __syncthreads();
    }
    if (traj) {
      double2* t_out = reinterpret_cast<double2*>(traj) + (long long)done * d;
      for (int i = threadIdx.x; i < d; i += blockDim.x) t_out[i] = cur[i];
    }
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) reinterpret_cast<double2*>(psi)[i] = cur[i];
}

__global__ void __launch_bounds__(CHAIN_THREADS)
state_chain_kernel(int n_steps, int d, const double* __restrict__ U, long long sU,
                   double* __restrict__ psi, int reorth_every, int step_offset, double* __restrict__ traj) {
  extern __shared__ double2 sh[];
  __shared__ double red[CHAIN_THREADS / 32];
  chain_body(n_steps, d, U, sU, psi, reorth_every, step_offset, sh, red, traj);
}

// Many jobs at once: CTA b carries job segs[b].job through its segment of the chunk.
__global__ void __launch_bounds__(CHAIN_THREADS)
multi_chain_kernel(int d, const ChainSeg* __restrict__ segs, const double* __restrict__ U, long long sU,
                   double* const* __restrict__ psi, int reorth_every) {
  extern __shared__ double2 sh[];
  __shared__ double red[CHAIN_THREADS / 32];
  const ChainSeg g = segs[blockIdx.x];
  chain_body(g.count, d, U + g.first * sU, sU, psi[g.job], reorth_every, g.done_before, sh, red, nullptr);
}

// out = U psi (one interval), rows split over CTAs: 8 warps per CTA, one row per warp.
__global__ void __launch_bounds__(256)
matvec_kernel(int d, const double* __restrict__ U, const double* __restrict__ in, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 8 + warp;
  if (i >= d) return;
  const double2* row = reinterpret_cast<const double2*>(U) + (long long)i * d;
  const double2* v = reinterpret_cast<const double2*>(in);
  double re = 0.0, im = 0.0;
  for (int j = lane; j < d; j += 32) {
    double2 u = row[j], x = v[j];
    re = fma(u.x, x.x, re);
    re = fma(-u.y, x.y, re);
    im = fma(u.x, x.y, im);
    im = fma(u.y, x.x, im);
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) reinterpret_cast<double2*>(out)[i] = make_double2(re, im);
}

__global__ void normalize_kernel(int d, double* __restrict__ psi) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(red[0]);
  for (int i = threadIdx.x; i < 2 * d; i += blockDim.x) psi[i] *= inv;
}

__global__ void norm_defect_kernel(int d, const double* __restrict__ psi, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    *out = fabs(sqrt(v) - 1.0);
  }
}

// psi (device, d complex) is carried through n_steps propagators U (stride sU doubles).
// tmp: d complex of scratch for the large-d path.  traj (may be null): the state
// after step n is also written to traj + (step_offset + n + 1) d complex.
int launch_state_chain(int n_steps, int d, const double* U, long long sU, double* psi, double* tmp,
                       int reorth_every, int step_offset, cudaStream_t s, double* traj) {
  if (n_steps <= 0) return MG_OK;
  if (d <= 256) {
    int threads = d <= 32 ? ((d + 31) / 32) * 32 * 8 : CHAIN_THREADS;
    if (threads > CHAIN_THREADS) threads = CHAIN_THREADS;
    size_t smem = sizeof(double2) * 2 * d;
    state_chain_kernel<<<1, threads, smem, s>>>(n_steps, d, U, sU, psi, reorth_every, step_offset, traj);
    return check_launch("state_chain_kernel");
  }
  double* a = psi;
  double* b = tmp;
  for (int n = 0; n < n_steps; ++n) {
    matvec_kernel<<<ceil_div(d, 8), 256, 0, s>>>(d, U + n * sU, a, b);
    MG_TRY(check_launch("matvec_kernel"));
    double* t = a; a = b; b = t;
    const int done = step_offset + n + 1;
    if (reorth_every > 0 && done % reorth_every == 0) {
      normalize_kernel<<<1, 1024, 0, s>>>(d, a);
      MG_TRY(check_launch("normalize_kernel"));
    }
    if (traj)
      MG_CUDA_TRY(cudaMemcpyAsync(traj + (long long)done * 2 * d, a, sizeof(double) * 2 * d,
                                  cudaMemcpyDeviceToDevice, s));
  }
  if (a != psi) MG_CUDA_TRY(cudaMemcpyAsync(psi, a, sizeof(double) * 2 * d, cudaMemcpyDeviceToDevice, s));
  return MG_OK;
}

int launch_multi_chain(int nseg, int d, const ChainSeg* segs_dev, const double* U, long long sU,
                       double* const* psi_dev, int reorth_every, cudaStream_t s) {
  if (nseg <= 0) return MG_OK;
  if (d > 256) return MG_EUNSUPPORTED;
  const int threads = d <= 32 ? 256 : CHAIN_THREADS;
  multi_chain_kernel<<<nseg, threads, sizeof(double2) * 2 * d, s>>>(d, segs_dev, U, sU, psi_dev, reorth_every);
  return check_launch("multi_chain_kernel");
}

int launch_norm_defect(int d, const double* psi, double* out, cudaStream_t s) {
  norm_defect_kernel<<<1, 1024, 0, s>>>(d, psi, out);
  return check_launch("norm_defect_kernel");
}

}  // namespace mg
