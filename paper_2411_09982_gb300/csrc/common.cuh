// Shared definitions of the Magnus library's CUDA translation units.
//
// Complex matrices are stored row-major with interleaved (re, im) FP64 pairs:
// element (i, j) of a d x d matrix lives at doubles [2 (i d + j), 2 (i d + j) + 1].
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "../../include/magnus.h"

namespace mg {

// ---------------------------------------------------------------------------
// error plumbing (no C++ exception crosses the C ABI)
// ---------------------------------------------------------------------------
#define MG_CUDA_TRY(expr)                                                       \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      mg::set_last_cuda_error(_e, #expr, __FILE__, __LINE__);                   \
      return MG_ECUDA;                                                          \
    }                                                                           \
  } while (0)

#define MG_TRY(expr)                                                            \
  do {                                                                          \
    int _r = (expr);                                                            \
    if (_r != MG_OK) return _r;                                                 \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void set_last_message(const char* fmt, ...);

// Device-side status word.  Kernels that wait on an mbarrier give up after a
// bounded number of polls, record MG_DEV_TIMEOUT here and return; the host maps
// it to MG_ETIMEOUT.  Non-finite norms set MG_DEV_NONFINITE.
enum : int { MG_DEV_OK = 0, MG_DEV_TIMEOUT = 1, MG_DEV_NONFINITE = 2 };

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
struct cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Every kernel launch goes through check_launch(): it counts the launch and
// converts a launch error into MG_ECUDA with a message.
int check_launch(const char* name);
void count_launch();
// Raises a kernel's dynamic shared-memory limit to at least `bytes` and sets
// its other launch attributes, calling cudaFuncSetAttribute only the first
// time a value is needed on the current device (a kernel whose attributes
// change while launches of it are in flight on other streams can stall them).
int ensure_smem_limit(const void* func, int bytes);
int ensure_func_attr(const void* func, cudaFuncAttribute attr, int value);

// ---------------------------------------------------------------------------
// kernels shared between translation units (launch wrappers)
// ---------------------------------------------------------------------------
// c[n][k] = (dt/2) sum_p w[p] samples[n][p][k]
int launch_coefficients(int N, int P, int K, double dt, const double* w_dev,
                        const double* samples, double* c, cudaStream_t s);

// first-order c_k, alpha_k and beta_kl of the second-order Magnus term per interval
// (row length 2K + K(K-1)/2); mrc = [M (P x P) | column sums | row sums] on the device
int launch_second_order_coefficients(int N, int P, int K, double dt, const double* w_dev, const double* mrc_dev,
                                     const double* samples, double* c, cudaStream_t s);

// omega[n] = dt H0 + sum_k c[n][k] H_k (minus tau_n I when write_shifted), with
// tau[n] = Re tr/d (0 unless shift) and norm1[n] = ||omega_n - tau_n I||_1.
// scratch: K + 1 + N doubles of device memory.
// out_df32: omega is written as double-float (float4 per element; write_shifted required)
int launch_build_omega(int N, int d, int K, double dt, const double* H0, const double* Hk,
                       const double* c, double* omega, double* tau, double* norm1, int shift,
                       int write_shifted, double* scratch, cudaStream_t s, int out_df32 = 0);

// tau_b = Re tr(A_b)/d (0 unless shift), dst_b = A_b - tau_b I, norm1_b = ||dst_b||_1
int launch_shift_norm(int batch, int d, const double* A, double* dst, double* tau, double* norm1,
                      unsigned long long* bits, int shift, cudaStream_t s);

// out[0] = max|H - H^dag|, out[1] = max|H| over `count` stacked d x d operators (as double bits)
int launch_hermitian_defect(int d, int count, const double* H, unsigned long long* out, cudaStream_t s);

// *out |= 1 if an entry of the count stacked d x d operators at M has a nonzero imaginary
// part, |= 2 if a real part differs from its transpose's
int launch_operator_structure(int d, long long count, const double* M, int* out, cudaStream_t s);

// X_b = (-i) 2^{-sq_b} src_b, sq from a device int array (sq_dev) or the constant sq
int launch_scale_minus_i(int batch, int d, const double* src, double* dst, const int* sq_dev,
                         int sq, cudaStream_t s);

// dst = sum_m coef[m] src_m + diag I over a batch (nsrc <= 4; sources may alias dst)
int launch_lincomb(int batch, int d, double* dst, int nsrc, const double* const* src,
                   const double* coef, double diag, cudaStream_t s);

// dst_b = exp(-i phase_b) src_b  (phase from device array)
int launch_apply_phase(int batch, int d, long long count_per_item, const double* phase,
                       const double* src, double* dst, cudaStream_t s);

int launch_identity(int batch, int d, double* dst, cudaStream_t s);

// copy a strided batch: dst[b] = src[b * src_stride] (strides in doubles)
// dst[p] = src[idx[p]] for p < n matrices of md doubles (idx on the device)
int launch_gather_mats(int n, long long md, const double* src, const int* idx_dev, double* dst, cudaStream_t s);
int launch_copy_strided(int batch, long long elems, const double* src, long long src_stride,
                        double* dst, long long dst_stride, cudaStream_t s);

// FP64 batched complex GEMM: C[b] = scale * opA(A[b]) B[b] + sum_m coef[m] P_m[b] + diag I.
// opA: 0 = A, 1 = A^dagger.  Batch strides in doubles.
struct AddTerms {
  int n = 0;
  const double* src[3] = {nullptr, nullptr, nullptr};
  double coef[3] = {0, 0, 0};
  long long stride = 0;   // batch stride of the addend matrices (doubles)
  double diag = 0.0;
  double scale = 1.0;
  // FP64 product only: with item_sq set, items with item_sq[b] <= sq_step are skipped
  const int* item_sq = nullptr;
  int sq_step = 0;
};
int launch_cgemm_f64(int batch, int d, const double* A, long long strideA, int opA,
                     const double* B, long long strideB, double* C, long long strideC,
                     const AddTerms& add, cudaStream_t s);

// max-abs reductions used for reports: out = max_b max_ij |U_b^dag U_b - I| computed
// from G_b = U_b^dag U_b (already formed), or |‖psi‖ - 1|.
int launch_max_identity_defect(int batch, int d, const double* G, double* out_dev, cudaStream_t s);

// Split-precision (BF16-digit, tcgen05) products; see split_gemm.cu.
int split_beta_for(int d);
size_t split_a_bytes(int d, int L, int batch);
size_t split_b_bytes(int d, int L, int batch);
// Inputs are FP64 (in_df32 = 0) or double-float (in_df32 = 1) complex matrices; the
// product C and the addends are double-float (see df32.cuh).
// Launch controls of the split product and its slicers.
struct SplitCtl {
  // limit of the waits a CTA may abandon (the MMA issuer's wait for a loaded stage,
  // the producer's wait for a free one); the others keep the 4 s limit
  unsigned long long wait_ns = 4000000000ull;
  int stall = 0;                 // test only: the MMA issuer waits on a barrier nothing completes
  const int* item_sq = nullptr;  // per-item squaring counts (device) or null: every item active
  int sq_step = 0;               // with item_sq: only items with item_sq[b] > sq_step are computed
  int stage_k = 32;              // K per pipeline stage of the product: 16, 32 or 64
  int pairs = 0;                 // paired digit layout (even digit counts; 1: 16-deep stages of 64-byte rows,
                                 // 2: 32-deep stages of 128-byte rows): slicers and product of one set of
                                 // digit buffers must agree on it (the memory layout is the same for 1 and 2)
  int cta_pairs = -1;            // M = 256 products on CTA pairs (tcgen05 cta_group::2) where d > 128:
                                 // 1 on, 0 off, -1 for five or more digits
  // Operand structure of one product (bit 0: the real part is exactly zero, bit 1: the
  // imaginary part is).  A's zero half of K is neither loaded nor multiplied; with one
  // part of B zero, each half of K multiplies the other plane only (N = 64) into the
  // output half it feeds, on one CTA per tile.  The skipped digit products are exact
  // zeros, so the product is the same; a flag set on an operand that is not so
  // structured gives a wrong product.  3 (both parts zero) is treated as 0.
  int a_zero = 0;
  int b_zero = 0;
  // The product is complex symmetric (C = C^T: polynomials in a symmetric matrix and
  // their products with one another) and its operands and addends are held in lower-block
  // storage (valid 32 x 32 blocks on and below the diagonal; entry (i, j) with j > i read
  // as (j, i)).  Output tiles wholly right of the diagonal are not computed; the result
  // is left in the same storage.
  int sym_out = 0;
};
int split_slice_a(int d, int L, int batch, const double* A, long long sA, int in_df32, void* buf, cudaStream_t s,
                  const SplitCtl& ctl = SplitCtl());
int split_slice_b(int d, int L, int batch, const double* B, long long sB, int in_df32, void* buf, cudaStream_t s,
                  const SplitCtl& ctl = SplitCtl());
int split_slice_sym(int d, int L, int batch, const double* M, long long sM, void* abuf, int askip, void* bbuf,
                    int bskip, cudaStream_t s, const SplitCtl& ctl = SplitCtl());
int split_sym_fill(int d, int batch, double* C, long long sC, cudaStream_t s);
int split_gemm(int d, int L, int batch, const void* abuf, const void* bbuf, double* C, long long sC,
               const AddTerms& add, int* status, cudaStream_t s, const SplitCtl& ctl = SplitCtl());

// State propagation; see propagate.cu.
int launch_state_chain(int n_steps, int d, const double* U, long long sU, double* psi, double* tmp,
                       int reorth_every, int step_offset, cudaStream_t s, double* traj = nullptr);
int launch_norm_defect(int d, const double* psi, double* out, cudaStream_t s);
// A job's stretch of intervals inside a chunk of the batched path.
struct ChainSeg {
  int job;          // index into the per-job state arrays
  int first;        // first interval of the segment within the chunk
  int count;        // intervals in the segment
  int done_before;  // intervals of this job already applied (for the re-normalisation period)
};
int launch_multi_chain(int nseg, int d, const ChainSeg* segs_dev, const double* U, long long sU,
                       double* const* psi_dev, int reorth_every, cudaStream_t s);
// One state job of the action-based path (action.cu).  The operators are one
// CSR pattern (union of the nonzeros of H0, H_1.. H_K plus the diagonal) with
// one complex value array per operator, operator-major: val[(op * nnz + e)].
constexpr int ACTION_REC = 72;   // doubles per interval record
// dynamic shared memory limit of the action chain kernels (their static
// shared memory, ~2.5 KB, stays within the 227 KB a block may hold)
constexpr int ACTION_SMEM_LIMIT = 220 * 1024;
struct ActionJob {
  int d;
  int K;
  int N;
  int first;            // first interval's row in c
  int nnz;
  double dt;
  const int* rowptr;    // d + 1
  const int* col;       // nnz
  const int* diag;      // d: position of the diagonal entry of each row
  const double* val;    // (1 + K) x nnz complex
  const double* c;      // coefficients c_{k,n}, row-major N x K
  double* cheb;         // N x ACTION_REC interval records (written by the bounds kernel)
  double* abuf;         // nnz complex: the interval matrix when it does not fit in shared memory
  double* psi;          // d complex, in and out
  double* traj;         // null, or (first + N + 1) x d complex: the state after interval n at row first + n + 1
  const uint16_t* sendmask;  // cluster variant: per row, bit q set if CTA q reads that row
  int status;           // MG_OK, or set by the kernel when the job stopped early
  long long max_steps;  // operator applications after which a launch stops at an interval end (0: none)
  int done;             // written by the kernel: intervals this launch completed
  // written by the kernel: operator applications, sub-step counts, degree, half-width
  long long matvecs;
  int max_sub, min_sub, max_terms;
  double max_nu;
};
// shared memory of the chain kernel for the largest d and the largest nonzero
// count held on chip (0: every interval matrix in global memory)
size_t action_smem_bytes(int dmax, int nnz_cap);
// the same for the cluster variant: C CTAs per job, cap_loc own-row nonzeros on chip
size_t action_cluster_smem_bytes(int dmax, int C, int cap_loc);
// largest power-of-two cluster size <= want that the device co-schedules, else 1
int action_cluster_size(int want, int dmax, int cap_loc);
// bounds kernel, then the chain: one CTA per job (cluster <= 1, nnz_cap = the
// nonzeros held on chip) or one cluster of `cluster` CTAs per job (nnz_cap =
// own-row nonzeros held on chip per CTA)
int launch_action_chain(int njobs, ActionJob* jobs_dev, int dmax, int nmax, int nnz_cap, int cluster,
                        cudaStream_t s);

// dst (dp x dp, zero padded) <- src (d x d), for `count` stacked matrices
int launch_pad_copy(int count, int d, int dp, const double* src, double* dst, cudaStream_t s);
// top-left d x d block of dst (dp x dp) <- src (d x d); the rest of dst untouched
int launch_pad_into(int d, int dp, const double* src, double* dst, cudaStream_t s);
// dst (d x d) <- top-left block of src (dp x dp)
int launch_unpad_copy(int d, int dp, const double* src, double* dst, cudaStream_t s);

// Device-side decisions of the batched path; see batch.cu.
// out[q] = ||A_q - tau_q I||_1 for `count` consecutive d x d operators
int launch_op_norm1(int count, int d, const double* ops, double* out, cudaStream_t s);
struct CoefRef {
  const double* c;   // N x K coefficients (device)
  int N, K;
  int off;           // first output slot of the job
};
// out[off_j + k] = max_n |c_j[n][k]| (NaN if any is non-finite), one block per job
int launch_coef_absmax(int njobs, const CoefRef* refs_dev, double* out, cudaStream_t s);
// per segment (seg_tab: job, first item, items): a non-finite norm or phase sets
// job_fail[job] and seg_bad, zeroes the segment's norms, phases and exponents W
int launch_fail_segments(int nseg, int fill, long long md, const int* seg_tab, const int* seg_of_item, double* norm,
                         double* tau, int* job_fail, int* seg_bad, double* W, cudaStream_t s);
// *out = max |a_e - b_e| over n doubles (device; a NaN difference gives NaN)
int launch_max_abs_diff(long long n, const double* a, const double* b, double* out, cudaStream_t s);
// dst[b] = src[b] (md doubles each) for the items with item_sq[b] > sq_step
int launch_copy_active(int batch, long long md, const double* src, double* dst, const int* item_sq, int sq_step,
                       cudaStream_t s);
// sq[i] = smallest s with 2^-s norm[i] <= theta (uniform: S for every item); s > S sets *overflow.
// flops_acc (may be null): += flops_per_square * sq[i] summed over the items (per-item mode)
int launch_squarings(int n, const double* norm, double theta, int S, int uniform, int* sq, int* overflow,
                     double* flops_acc, double flops_per_square, cudaStream_t s);

// Double-float (DF32) elementwise kernels of the split path; see elementwise.cu.  With
// lower != 0 they touch only the 32 x 32 blocks on and below the diagonal (the valid
// part of a symmetric matrix in lower-block storage).
// X_b = -i 2^{-sq_b} W_b with sq_b from sq_dev (device, per item) or the constant sq;
// W FP64 (in_df32 = 0) or double-float (in_df32 = 1), X double-float (may alias W)
int launch_scale_minus_i_df(int batch, int d, const double* src, double* dst_df, int sq, cudaStream_t s,
                            const int* sq_dev = nullptr, int in_df32 = 0, int lower = 0);
// dst[o] = sum_m coef[o * nsrc + m] src[m] + diag[o] I, o < nout <= 5, nsrc <= 4, one pass
// (a destination may alias a source); FP64 and double-float storage
int launch_lincomb_multi(int batch, int d, int nout, double* const* dst, int nsrc, const double* const* src,
                         const double* coef, const double* diag, cudaStream_t s);
int launch_lincomb_multi_df(int batch, int d, int nout, double* const* dst, int nsrc, const double* const* src,
                            const double* coef, const double* diag, cudaStream_t s, int lower = 0);
int launch_lincomb_df(int batch, int d, double* dst, int nsrc, const double* const* src, const double* coef,
                      double diag, cudaStream_t s, int lower = 0);
int launch_apply_phase_df(int batch, int d, const double* phase, const double* src, double* dst, cudaStream_t s);
// dst_b = e^{-i phase_b} src_b into full storage from a symmetric src in lower-block storage
int launch_apply_phase_sym_df(int batch, int d, const double* phase, const double* src, double* dst, cudaStream_t s);
int launch_identity_df(int batch, int d, double* dst, cudaStream_t s);
int launch_df_to_fp64(int batch, int d, const double* src, long long ss, double* dst, long long ds, cudaStream_t s);
int launch_fp64_to_df(int batch, int d, const double* src, long long ss, double* dst, long long ds, cudaStream_t s);

}  // namespace mg
