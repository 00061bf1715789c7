// Split-precision complex matrix product on the tcgen05 tensor cores.
//
// Every matrix product of the exponential (Taylor powers, Horner steps,
// squarings) and of the propagator product is a complex d x d GEMM
// C = A B.  In MG_PREC_SPLIT mode it runs as a real GEMM on BF16 digits:
//
//   * complex -> real:   [Cr | Ci] = [Ar | Ai] * [[Br, Bi], [-Bi, Br]]
//     (M = d, N = 2d, K = 2d; 8 d^3 real flops, the "4M" form).
//   * digits:  each FP64 row i of [Ar | Ai] (all entries below 2^{E_i}) is cut
//     into `L` signed digits of `beta` bits, a = 2^{E_i+1-beta} sum_s v_s with
//     v_s = q_s 2^{-beta s}, |q_s| <= 2^{beta-1}; every v_s is exact in BF16.
//     Columns of B are cut the same way.
//   * products: digit products v_s^A v_t^B with s + t <= L - 1 are accumulated
//     in four FP32 TMEM accumulators by level s + t = 0, 1, 2, >= 3.  beta is
//     chosen so that 2^{2 beta - 1} * 2d <= 2^24: the level-0 and level-1 sums are
//     then integers (in units of 1 and 2^-beta) below 2^24 and accumulate
//     exactly; level 2 is exact for all but adversarial inputs, and only the
//     level->=3 part, 2^{-3 beta} below the leading one, is rounded.
//   * epilogue: C_ij = 2^{(E_i+1-beta)+(F_j+1-beta)} (g0 + g1 + g2 + g3) in FP64, plus
//     optional FP64 addends (Taylor/Horner terms) and a diagonal.
//
// The error of one product is about 2^{-beta L} relative to max|A| max|B|, so
// L = 5..6 gives a far smaller per-product error than FP32 arithmetic and
// L = 7..8 approaches FP64.  This is the tensor-core replacement of the FP64
// products of the exponential; everything else of the path stays FP64.
//
// Kernel structure (one 128 x 64-complex output tile per CTA, 320 threads):
//   warp 0      TMA producer: per K-step of 32 one 4-D box of all L A-digit
//               tiles (128 x 32 BF16 each) and one 5-D box of all L B-digit tiles
//               (two consecutive planes of 64 rows), SWIZZLE_64B (64-byte rows:
//               half the TMA row requests of 32-byte rows, which capped operand
//               delivery at ~58 GB/s per SM), into a STAGES-deep ring of
//               shared-memory stages.  Every CTA loads its own operands from this
//               GPU's memory; no load is shared between CTAs.
//   warp 1      TMEM owner and MMA issuer: tcgen05.mma kind::f16 (BF16 in,
//               FP32 accumulate), M = 128, N = 128 (64 real + 64 imaginary
//               output columns), K = 16, two instructions per digit pair and
//               stage (the second starts 32 bytes into the swizzle atom).
//   warps 2..9  epilogue: tcgen05.ld of the four accumulators (two warps per TMEM
//               lane quarter, 32 complex columns each), double-float combine.
// Every mbarrier wait is bounded by a wall-clock deadline; a wait that gives up
// records MG_DEV_TIMEOUT in the status word and the CTA winds down.  Only the
// waits whose abandonment is safe take the caller's (possibly short) limit: the
// MMA issuer's wait for a loaded stage and the producer's wait for a free one.
// The epilogue's wait for the accumulators and the producer's final drain of
// its own copies always use the long limit, so no CTA releases TMEM or shared
// memory while a tensor-core operation or a copy into it is still in flight.
#include "common.cuh"
#include "df32.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>
#include <algorithm>
#include <cstring>

namespace mg {

// ---------------------------------------------------------------------------
// host-side geometry
// ---------------------------------------------------------------------------
constexpr int SG_BM = 128;      // output rows per tile
constexpr int SG_BNC = 64;      // complex output columns per tile (N = 128 real)
constexpr int SG_BK = 32;       // K granularity of the digit layout (each half of K is a multiple of it)
constexpr int SG_MMA_K = 16;    // K of one tcgen05.mma kind::f16
// K per pipeline stage: 32 (64-byte rows, SWIZZLE_64B, two MMA K-steps per stage) or 16
// (32-byte rows, SWIZZLE_32B, one K-step: half the bytes per stage, twice the stages)
template <int BK> struct StageK {
  static constexpr int tile_bytes = SG_BM * BK * 2;   // bytes per digit tile of one stage
};

struct SplitGeom {
  int d, L, beta;
  int Kp;      // 2 Kh, Kh = d rounded up to 32: the K axis holds [Re (d) | 0 | Im (d) | 0], each half Kh long
  int Mp;      // padded d rows (multiple of 128)
  int Np;      // 2 x padded d columns (128 per 64 complex columns)
  int Kh() const { return Kp / 2; }
  long long a_item_elems() const { return (long long)L * Mp * Kp; }   // BF16 elements
  // B: per digit, three planes (-Im B, Re B, Im B) of Np / 2 rows (one per column of B) of Kh
  long long b_item_elems() const { return (long long)L * 3 * (Np / 2) * Kh(); }
};

// The paired digit layout applies to even digit counts only (odd counts keep one plane per digit).
static inline int paired_layout(const SplitGeom& g, const SplitCtl& ctl) { return ctl.pairs && g.L % 2 == 0; }

// Where digit s of an operand element lives, relative to its batch item.  Digit-major
// layout (pairs = 0): one K-major plane per digit.  Paired layout (pairs = 1, even digit
// counts): digits 2g and 2g + 1 share the rows of group g, every 16-wide block of K
// holding 16 values of the even digit and then 16 of the odd one, so that one 64-byte
// row of a 16-deep K stage carries both digits: half the shared memory per stage of the
// digit-major form with 64-byte rows, hence twice the stages in the same ring.
__device__ __forceinline__ long long a_digit_off(int pairs, int s, int row, int k, int Mp, int Kp) {
  if (!pairs) return (long long)s * Mp * Kp + (long long)row * Kp + k;
  return (long long)(s >> 1) * Mp * Kp * 2 + (long long)row * Kp * 2 + (k >> 4) * 32 + (s & 1) * 16 + (k & 15);
}
__device__ __forceinline__ long long b_digit_off(int pairs, int s, int plane, int j, int k, int rows, int Kh) {
  if (!pairs) return ((long long)s * 3 + plane) * rows * Kh + (long long)j * Kh + k;
  return ((long long)(s >> 1) * 3 + plane) * rows * Kh * 2 + (long long)j * Kh * 2 + (k >> 4) * 32 + (s & 1) * 16 +
         (k & 15);
}

int split_beta_for(int d) {
  // largest beta <= 8 with 2^{2 beta - 1} * 2d <= 2^24
  for (int beta = 8; beta >= 2; --beta) {
    double lhs = std::ldexp(1.0, 2 * beta - 1) * 2.0 * d;
    if (lhs <= 16777216.0) return beta;
  }
  return 2;
}

SplitGeom split_geom(int d, int L) {
  SplitGeom g;
  g.d = d;
  g.L = L;
  g.beta = split_beta_for(d);
  g.Kp = 2 * ceil_div(d, SG_BK) * SG_BK;   // each half a whole number of K stages
  g.Mp = ceil_div(d, SG_BM) * SG_BM;
  g.Np = ceil_div(d, SG_BNC) * 2 * SG_BNC;
  return g;
}

// ---------------------------------------------------------------------------
// digit extraction (shared by the A and B slicers)
// ---------------------------------------------------------------------------
// A value a of a row (column) whose entries all lie below 2^E in magnitude is
// scaled to x = a 2^{beta - 1 - E}, |x| < 2^{beta-1}, held exactly as a pair of
// FP32 numbers x + y (a double-float input is exact in two FP32 numbers; an FP64
// input is first split into two).  Its balanced base-2^beta digits are peeled on
// the FP32 pipe, every step exact:
//     (x, y) <- TwoSum(x, y);  q_s = round(x);  (x, y) <- ((x - q_s) 2^beta, y 2^beta)
// (x - q_s is exact by Sterbenz's lemma, the scaling by a power of two), so
//     a = 2^{E+1-beta} (sum_{s<L} q_s 2^{-beta s} + r),  |r| <= 2^{-beta (L-1) - 1} (1 + 2^-20),
// with |q_s| <= 2^{beta-1}; every v_s = q_s 2^{-beta s} is exact in BF16.  The
// rounding to an integer is (x + 1.5 2^23) - 1.5 2^23 (to nearest even, exact for
// |x| < 2^22), so the whole extraction runs on the FMA pipe; the earlier
// 64-bit-integer form of the same digits kept GB300's integer pipe 72% busy.

// exponent E of |a| with |a| < 2^E (biased exponent - 1022); zero and subnormals -> -2^29
__device__ __forceinline__ int exp_bound(double a) {
  const long long bits = __double_as_longlong(a);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  return bexp == 0 ? -(1 << 29) : bexp - 1022;
}
// the same for a double-float hi + lo (|hi + lo| < 2^E whenever |hi| < 2^E)
__device__ __forceinline__ int exp_bound(df32 a) {
  const int bits = __float_as_int(a.hi);
  const int bexp = (bits >> 23) & 0xFF;
  return bexp == 0 ? -(1 << 29) : bexp - 126;
}

// one complex element of an FP64 or DF32 matrix (16 bytes either way)
struct c64 { double re, im; };
struct cdf { df32 re, im; };
template <typename T> struct Elem;
template <> struct Elem<double> {
  using type = c64;
  __device__ __forceinline__ static type load(const double* base, long long idx) {
    const double2 v = reinterpret_cast<const double2*>(base)[idx];
    return {v.x, v.y};
  }
};
template <> struct Elem<df32> {
  using type = cdf;
  __device__ __forceinline__ static type load(const double* base, long long idx) {
    const float4 v = reinterpret_cast<const float4*>(base)[idx];
    return {{v.x, v.y}, {v.z, v.w}};
  }
};

// 2^k as the product of two FP32 factors (each in range for |k| <= 250)
struct Pow2Pair {
  float f1, f2;
};
__device__ __forceinline__ Pow2Pair pow2_pair(int k) {
  const int k1 = k / 2, k2 = k - k1;
  return {__int_as_float((127 + k1) << 23), __int_as_float((127 + k2) << 23)};
}
// the scaled value as an exact pair of FP32 numbers
__device__ __forceinline__ df32 scaled_pair(df32 a, Pow2Pair f) { return {(a.hi * f.f1) * f.f2, (a.lo * f.f1) * f.f2}; }
__device__ __forceinline__ df32 scaled_pair(double a, Pow2Pair f) {
  const float hi = __double2float_rn(a);
  const float lo = __double2float_rn(a - (double)hi);
  return {(hi * f.f1) * f.f2, (lo * f.f1) * f.f2};
}

constexpr float kRoundMagic = 12582912.0f;   // 1.5 2^23
__device__ __forceinline__ float round_to_int(float x) { return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic); }

// digits of two scaled values (the first in the low half of every word): w[s] holds
// q_s 2^{-beta s} of both as BF16
template <int L>
__device__ __forceinline__ void digits_pair(df32 u, df32 v, int beta, uint32_t (&w)[L]) {
  const float B = __int_as_float((127 + beta) << 23);
#pragma unroll
  for (int s = 0; s < L; ++s) {
    const df32 a = two_sum(u.hi, u.lo), b = two_sum(v.hi, v.lo);
    const float qa = round_to_int(a.hi), qb = round_to_int(b.hi);
    const float p = __int_as_float((127 - beta * s) << 23);   // 2^{-beta s}
    const __nv_bfloat162 d2 = __floats2bfloat162_rn(qa * p, qb * p);
    w[s] = *reinterpret_cast<const uint32_t*>(&d2);
    u = {__fsub_rn(a.hi, qa) * B, a.lo * B};
    v = {__fsub_rn(b.hi, qb) * B, b.lo * B};
  }
}

// the word with every digit negated (BF16 sign bits)
__device__ __forceinline__ uint2 neg4(uint2 w) { return make_uint2(w.x ^ 0x80008000u, w.y ^ 0x80008000u); }

// A digits: rows of [Re A | 0 | Im A | 0] (halves of Kh = Kp / 2 columns).
// grid (ceil(Mp/8), batch), block 256 (one warp per row); each lane writes the
// digits of 4 consecutive elements per plane as one 8-byte store.
// T = double (FP64 input) or df32 (double-float input); strides count doubles.
template <int L, typename T>
__global__ void __launch_bounds__(256)
slice_a_kernel(int d, int Kp, int Mp, int beta, const double* __restrict__ A, long long sA,
               __nv_bfloat16* __restrict__ out, int* __restrict__ ea, const int* __restrict__ item_sq, int sq_step,
               long long item_elems, int pairs) {
  using E_ = Elem<T>;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int b = blockIdx.y;
  if (row >= Mp) return;
  if (item_sq && item_sq[b] <= sq_step) return;   // inactive item: its digits are not read
  const int Kh = Kp / 2;
  __nv_bfloat16* o = out + (long long)b * item_elems;
  if (row >= d) return;   // rows d..Mp are never read: the tensor map ends at row d (TMA fills zeros)
  const double* a = A + b * sA;
  const long long r0 = (long long)row * d;
  int E = -(1 << 29);
  for (int k = lane; k < d; k += 32) {
    const auto v = E_::load(a, r0 + k);
    E = max(E, max(exp_bound(v.re), exp_bound(v.im)));
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o2));
  if (E < -(1 << 28)) E = 0;   // all-zero row
  if (lane == 0) ea[(long long)b * Mp + row] = E;
  const Pow2Pair f = pow2_pair(beta - 1 - E);
  for (int k = 4 * lane; k < Kh; k += 128) {
    df32 re[4], im[4];   // the 4 elements, scaled (zero beyond d)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      re[q] = im[q] = df32{0.f, 0.f};
      if (k + q < d) {
        const auto v = E_::load(a, r0 + k + q);
        re[q] = scaled_pair(v.re, f);
        im[q] = scaled_pair(v.im, f);
      }
    }
    uint32_t r01[L], r23[L], i01[L], i23[L];
    digits_pair<L>(re[0], re[1], beta, r01);
    digits_pair<L>(re[2], re[3], beta, r23);
    digits_pair<L>(im[0], im[1], beta, i01);
    digits_pair<L>(im[2], im[3], beta, i23);
#pragma unroll
    for (int s = 0; s < L; ++s) {
      *reinterpret_cast<uint2*>(o + a_digit_off(pairs, s, row, k, Mp, Kp)) = make_uint2(r01[s], r23[s]);
      *reinterpret_cast<uint2*>(o + a_digit_off(pairs, s, row, Kh + k, Mp, Kp)) = make_uint2(i01[s], i23[s]);
    }
  }
}

// Complex symmetric matrices (M = M^T) of the exponential are held as their lower 32 x 32
// blocks: block (bi, bj) is valid for bj <= bi, and entry (i, j) with j > i is read as
// M[j][i] (also inside the diagonal blocks, so every use sees exactly symmetric values).
// Their digits come from two kernels: the row exponents, then the digits of every 32 x 32
// block of rows and K, each from its own block or its transposed partner.

// Row exponent bounds E_i (|M_ij| < 2^{E_i} over the whole row i) from the stored lower
// triangle: entry (i, j), j <= i, bounds row i and row j (its transpose's row).  grid
// (ceil(d/32), ceil(d/32), batch), blocks above the diagonal return; block 256 (thread =
// column tx of rows ty, ty + 8, ...).  e1 (stride n1 per item) and e2 (n2; may be null)
// must be preset below -2^28 (byte 0x80); combined by atomicMax.
__global__ void __launch_bounds__(256)
sym_exponent_kernel(int d, const float4* __restrict__ M, long long sM4, int* __restrict__ e1, long long n1,
                    int* __restrict__ e2, long long n2, const int* __restrict__ item_sq, int sq_step) {
  const int bj = blockIdx.x, bi = blockIdx.y, b = blockIdx.z;
  if (bj > bi) return;
  if (item_sq && item_sq[b] <= sq_step) return;
  __shared__ int rmax[32], cmax[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < 32) rmax[tx] = cmax[tx] = -(1 << 29);
  __syncthreads();
  const float4* Mb = M + b * sM4;
  const int j = bj * 32 + tx;
  int cm = -(1 << 29);
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r;
    int e = -(1 << 29);
    if (i < d && j < d && j <= i) {
      const float4 v = Mb[(long long)i * d + j];
      e = max(exp_bound(df32{v.x, v.y}), exp_bound(df32{v.z, v.w}));
    }
    cm = max(cm, e);
    // every lane of the warp takes part (no divergent shuffle)
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (tx == 0) rmax[r] = e;   // row r is this warp's alone
  }
  atomicMax(&cmax[tx], cm);
  __syncthreads();
  if (threadIdx.x < 64) {
    const int c = threadIdx.x & 31;
    const int idx = threadIdx.x < 32 ? bi * 32 + c : bj * 32 + c;
    const int e = threadIdx.x < 32 ? rmax[c] : cmax[c];
    if (idx < d && e > -(1 << 29)) {
      atomicMax(e1 + b * n1 + idx, e);
      if (e2) atomicMax(e2 + b * n2 + idx, e);
    }
  }
}

// Digits of a complex symmetric matrix in lower-block storage for the A operand, the B
// operand or both: B's column j is its row j, so B's column exponents are the row
// exponents and B's plane rows are M's rows (plane 0: -Im, 1: Re, 2: Im).  One 32 x 32
// block of rows i and K positions k per CTA, staged in shared memory from block (i, k)
// or, right of the diagonal, from the transposed block (k, i); thread = (row, 4 k).
// ea / eb hold the row exponents (sym_exponent_kernel); askip (bit 0: the real half,
// bit 1: the imaginary half of A's K axis) and bskip (bit p: plane p of B) name parts
// that are not written because no product reads them (the zero parts of a real or
// imaginary operand, which the products skip).  K positions d..Kh are written as zero
// digits (the tile padding along K).  grid (Kh/32, ceil(d/32), batch), block 256.
template <int L>
__global__ void __launch_bounds__(256)
slice_sym_block_kernel(int d, int Kp, int Mp, int beta, const float4* __restrict__ M, long long sM4,
                       __nv_bfloat16* __restrict__ aout, const int* __restrict__ ea, long long a_item_elems,
                       int askip, __nv_bfloat16* __restrict__ bout, const int* __restrict__ eb,
                       long long b_item_elems, int brows, int bskip, const int* __restrict__ item_sq, int sq_step,
                       int pairs) {
  const int bk = blockIdx.x, bi = blockIdx.y, b = blockIdx.z;
  if (item_sq && item_sq[b] <= sq_step) return;
  __shared__ float4 t[32][33];
  const int Kh = Kp / 2;
  const int i0 = bi * 32, k0 = bk * 32;
  const float4* Mb = M + b * sM4;
  {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (bk < bi) {   // t[r][tx] = M[i0 + r][k0 + tx]
        if (i0 + r < d && k0 + tx < d) v = Mb[(long long)(i0 + r) * d + k0 + tx];
        t[r][tx] = v;
      } else if (bk > bi) {   // t[tx][r] = M[k0 + r][i0 + tx]
        if (k0 + r < d && i0 + tx < d) v = Mb[(long long)(k0 + r) * d + i0 + tx];
        t[tx][r] = v;
      } else {   // the diagonal block as stored, its upper half replaced below
        if (i0 + r < d && k0 + tx < d) v = Mb[(long long)(i0 + r) * d + k0 + tx];
        t[r][tx] = v;
      }
    }
  }
  __syncthreads();
  const int r = threadIdx.x >> 3, g = threadIdx.x & 7;   // row r of the block, K positions 4g..4g+3
  const int row = i0 + r;
  if (row >= d) return;
  const int k = k0 + 4 * g;
  if (k >= Kh) return;
  const int E0 = ea ? ea[(long long)b * Mp + row] : eb[(long long)b * brows + row];
  const int E = E0 < -(1 << 28) ? 0 : E0;   // all-zero row
  const Pow2Pair f = pow2_pair(beta - 1 - E);
  df32 re[4], im[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = 4 * g + q;
    // inside the diagonal block the entries right of the diagonal come from the left
    const float4 v = (bk == bi && c > r) ? t[c][r] : t[r][c];
    re[q] = k + q < d ? scaled_pair(df32{v.x, v.y}, f) : df32{0.f, 0.f};
    im[q] = k + q < d ? scaled_pair(df32{v.z, v.w}, f) : df32{0.f, 0.f};
  }
  uint32_t r01[L], r23[L], i01[L], i23[L];
  digits_pair<L>(re[0], re[1], beta, r01);
  digits_pair<L>(re[2], re[3], beta, r23);
  digits_pair<L>(im[0], im[1], beta, i01);
  digits_pair<L>(im[2], im[3], beta, i23);
  // digit s of an element lies (s >> 1) * S2 + (s & 1) * S1 past digit 0 (both layouts)
  if (aout) {
    __nv_bfloat16* oa = aout + (long long)b * a_item_elems;
    const long long s1 = pairs ? 16 : (long long)Mp * Kp, s2 = pairs ? 2LL * Mp * Kp : 2 * s1;
    __nv_bfloat16* pr = oa + a_digit_off(pairs, 0, row, k, Mp, Kp);
    __nv_bfloat16* pi = oa + a_digit_off(pairs, 0, row, Kh + k, Mp, Kp);
#pragma unroll
    for (int s = 0; s < L; ++s) {
      const long long o = (s >> 1) * s2 + (s & 1) * s1;
      if (!(askip & 1)) *reinterpret_cast<uint2*>(pr + o) = make_uint2(r01[s], r23[s]);
      if (!(askip & 2)) *reinterpret_cast<uint2*>(pi + o) = make_uint2(i01[s], i23[s]);
    }
  }
  if (bout) {
    __nv_bfloat16* ob = bout + (long long)b * b_item_elems;
    const long long s1 = pairs ? 16 : 3LL * brows * Kh, s2 = pairs ? 6LL * brows * Kh : 2 * s1;
    const long long plane = pairs ? 2LL * brows * Kh : (long long)brows * Kh;
    __nv_bfloat16* p0 = ob + b_digit_off(pairs, 0, 0, row, k, brows, Kh);
#pragma unroll
    for (int s = 0; s < L; ++s) {
      const long long o = (s >> 1) * s2 + (s & 1) * s1;
      const uint2 wi = make_uint2(i01[s], i23[s]);
      if (!(bskip & 1)) *reinterpret_cast<uint2*>(p0 + o) = neg4(wi);
      if (!(bskip & 2)) *reinterpret_cast<uint2*>(p0 + o + plane) = make_uint2(r01[s], r23[s]);
      if (!(bskip & 4)) *reinterpret_cast<uint2*>(p0 + o + 2 * plane) = wi;
    }
  }
}

// B digits: for every digit, three planes of K-major rows in the order
// -Im B, Re B, Im B: row j of a plane holds column j of that part of B along k
// (Kh = Kp / 2 entries, zero beyond d); rows j >= d up to Np / 2 are zero.  The
// real embedding [[Br, Bi], [-Bi, Br]] needs, for the real half of K, the rows
// [Br; Bi] (planes 1, 2) and, for the imaginary half, [-Bi; Br] (planes 0, 1):
// both are two consecutive planes, so one box per stage loads them.
// Two launches with many CTAs each (a column-exponent pass, then the digits of
// 32 x 64 blocks), so that the HBM-bound work has enough warps in flight.

// Column exponent bounds: grid (ceil(d/64), ceil(d/64), batch), block 256.
// eb must be preset below -2^28 (byte 0x80); blocks combine with atomicMax.
template <typename T>
__global__ void __launch_bounds__(256)
col_exponent_kernel(int d, int Np, const double* __restrict__ B, long long sB, int* __restrict__ eb,
                    const int* __restrict__ item_sq, int sq_step) {
  using E_ = Elem<T>;
  __shared__ int red[4][SG_BNC];
  const int j0 = blockIdx.x * SG_BNC, k0 = blockIdx.y * 64, b = blockIdx.z;
  if (item_sq && item_sq[b] <= sq_step) return;
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  const double* Bb = B + b * sB;
  int E = -(1 << 29);
  if (j0 + c < d) {
    const int kend = min(d, k0 + 64);
    for (int k = k0 + g; k < kend; k += 4) {
      const auto v = E_::load(Bb, (long long)k * d + j0 + c);
      E = max(E, max(exp_bound(v.re), exp_bound(v.im)));
    }
  }
  red[g][c] = E;
  __syncthreads();
  if (g == 0 && j0 + c < d) {
    const int EE = max(max(red[0][c], red[1][c]), max(red[2][c], red[3][c]));
    atomicMax(eb + (long long)b * (Np / 2) + j0 + c, EE);
  }
}

constexpr int SB_KCHUNK = 32;
// Digits of one 32 (k) x 64 (j) block: grid (ceil(d/64), ceil(d/32), batch), block 256.
// Each thread writes 4 consecutive k of one column per plane as 8-byte stores.
template <int L, typename T>
__global__ void __launch_bounds__(256)
slice_b_kernel(int d, int Kp, int Np, int beta, const double* __restrict__ B, long long sB,
               __nv_bfloat16* __restrict__ out, const int* __restrict__ eb, const int* __restrict__ item_sq,
               int sq_step, long long item_elems, int pairs) {
  using E_ = Elem<T>;
  using V = typename E_::type;
  __shared__ V tile[SB_KCHUNK][SG_BNC + 1];
  __shared__ int shift[SG_BNC];   // beta - 1 - F_j: the scaling exponent of column j
  const int t = blockIdx.x, b = blockIdx.z;
  if (item_sq && item_sq[b] <= sq_step) return;
  const int j0 = t * SG_BNC, k0 = blockIdx.y * SB_KCHUNK;
  const int tid = threadIdx.x;
  const int Kh = Kp / 2, rows = Np / 2;
  const double* Bb = B + b * sB;
  __nv_bfloat16* ob = out + (long long)b * item_elems;
  if (tid < SG_BNC) {
    int E = j0 + tid < d ? eb[(long long)b * rows + j0 + tid] : 0;
    if (E < -(1 << 28)) E = 0;   // all-zero column
    shift[tid] = beta - 1 - E;
  }
  for (int e = tid; e < SB_KCHUNK * SG_BNC; e += 256) {
    const int kk = e / SG_BNC, c = e % SG_BNC;
    V v{};
    if (k0 + kk < d && j0 + c < d) v = E_::load(Bb, (long long)(k0 + kk) * d + j0 + c);
    tile[kk][c] = v;
  }
  __syncthreads();
  for (int e = tid; e < (SB_KCHUNK / 4) * SG_BNC; e += 256) {
    const int g = e % (SB_KCHUNK / 4), r = e / (SB_KCHUNK / 4);
    const int k = k0 + 4 * g;
    if (k >= Kh || j0 + r >= d) continue;
    const Pow2Pair f = pow2_pair(shift[r]);
    df32 re[4], im[4];   // the 4 elements, scaled (zero beyond d)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      re[q] = im[q] = df32{0.f, 0.f};
      if (k + q < d) {
        const V v = tile[4 * g + q][r];
        re[q] = scaled_pair(v.re, f);
        im[q] = scaled_pair(v.im, f);
      }
    }
    uint32_t r01[L], r23[L], i01[L], i23[L];
    digits_pair<L>(re[0], re[1], beta, r01);
    digits_pair<L>(re[2], re[3], beta, r23);
    digits_pair<L>(im[0], im[1], beta, i01);
    digits_pair<L>(im[2], im[3], beta, i23);
    const int j = j0 + r;   // plane 0: -Im B, 1: Re B, 2: Im B
#pragma unroll
    for (int s = 0; s < L; ++s) {
      const uint2 wr = make_uint2(r01[s], r23[s]), wi = make_uint2(i01[s], i23[s]);
      *reinterpret_cast<uint2*>(ob + b_digit_off(pairs, s, 0, j, k, rows, Kh)) = neg4(wi);
      *reinterpret_cast<uint2*>(ob + b_digit_off(pairs, s, 1, j, k, rows, Kh)) = wr;
      *reinterpret_cast<uint2*>(ob + b_digit_off(pairs, s, 2, j, k, rows, Kh)) = wi;
    }
  }
  // rows d..Np/2 of every plane are never read: the tensor map ends at row d (TMA fills zeros)
}

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Poll until the phase of `parity` completes or the deadline passes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
// CTA-pair forms (cta_group::2): the copy may signal the barrier of either CTA of the pair
__device__ __forceinline__ void tma_load_4d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int c0,
                                                 int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int c0,
                                                 int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of this CTA's variable `p` as it lies in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tc_mma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                 uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the barrier at this offset in both CTAs of the pair once the issued MMAs
// complete: one commit per CTA, each naming that CTA's barrier by its cluster address
__device__ __forceinline__ void tc_commit_pair(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   cluster_addr(bar, 0))
               : "memory");
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   cluster_addr(bar, 1))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand tile, 64-byte swizzle,
// 8-row core groups 512 bytes apart (rows are 64 bytes), descriptor version 1.
// The second K = 16 step of a 64-byte row starts 32 bytes further: the swizzle
// is applied to the final address bits, so advancing the start address inside
// the atom selects the next 16 elements of every row.
__device__ __forceinline__ uint64_t sw64_kmajor_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)1 << 16;            // leading-dimension offset (unused with swizzle)
  desc |= (uint64_t)(512 >> 4) << 32;   // stride-dimension offset
  desc |= (uint64_t)1 << 46;            // descriptor version
  desc |= (uint64_t)4 << 61;            // SWIZZLE_64B
  return desc;
}

// The same for 32-byte rows: SWIZZLE_32B, 8-row core groups 256 bytes apart.
__device__ __forceinline__ uint64_t sw32_kmajor_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)1 << 16;            // leading-dimension offset (unused with swizzle)
  desc |= (uint64_t)(256 >> 4) << 32;   // stride-dimension offset
  desc |= (uint64_t)1 << 46;            // descriptor version
  desc |= (uint64_t)6 << 61;            // SWIZZLE_32B
  return desc;
}
// The same for 128-byte rows: SWIZZLE_128B, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)1 << 16;            // leading-dimension offset (unused with swizzle)
  desc |= (uint64_t)(1024 >> 4) << 32;  // stride-dimension offset
  desc |= (uint64_t)1 << 46;            // descriptor version
  desc |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return desc;
}
template <int BK>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  return BK == 64 ? sw128_kmajor_desc(saddr) : (BK == 32 ? sw64_kmajor_desc(saddr) : sw32_kmajor_desc(saddr));
}
// the paired layout's rows hold two digits: 64 bytes at BK = 16, 128 bytes at BK = 32
template <int BK>
__device__ __forceinline__ uint64_t pair_desc(uint32_t saddr) {
  return BK == 32 ? sw128_kmajor_desc(saddr) : sw64_kmajor_desc(saddr);
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
// the same with N = 64: one B plane (a product whose B operand has a zero part)
constexpr uint32_t kIdescBf16N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// the same with M = 256 (a CTA pair, cta_group::2)
constexpr uint32_t kIdescBf16M256 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((256u >> 4) << 24);

constexpr int SG_THREADS = 320;   // producer warp, MMA warp, 8 epilogue warps
constexpr int SG_EPI_WARPS = 8;
// epilogue staging tile: 128 rows x 64 complex (float4) with one float4 of padding per row
constexpr int SG_EPI_PITCH = SG_BNC + 1;
constexpr int SG_EPI_BYTES = SG_BM * SG_EPI_PITCH * 16;
// TMEM accumulators: digit-pair levels 0, 1, 2 and >= 3, 128 columns each (all 512).
constexpr int SG_GROUPS = 4;
constexpr uint64_t SG_WAIT_NS = 4000000000ull;   // 4 s: far beyond any legitimate wait

// The four level accumulators hold (in units of the leading digit product)
//   g0: integers, g1: multiples of 2^-beta, g2: multiples of 2^-2beta (all exact),
//   g3: the rounded remainder.
// Their sum is formed in double-float with error-free FP32 transformations and
// scaled by 2^k exactly: no instruction of GB300's narrow FP64 pipe.
__device__ __forceinline__ df32 combine_levels(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, int k) {
  const df32 a = two_sum(__uint_as_float(u0), __uint_as_float(u1));
  const df32 b = two_sum(__uint_as_float(u2), __uint_as_float(u3));
  return df_ldexp(df_add(a, b), k);
}

struct SplitEpi {
  const double* add_src[3];   // DF32 matrices (float4 per complex element)
  df32 add_coef[3];
  long long add_stride;       // in doubles
  int add_n;
  df32 diag;
};

// One CTA per 128 x 64-complex output tile of one batch item.  With ctl.item_sq set,
// item b is computed only while ctl.item_sq[b] > ctl.sq_step (per-item squaring
// counts: an item whose squarings are done keeps its matrix, which the product
// would otherwise overwrite in place); the CTAs of an inactive item return at once.
//
// PAIRS: operands in the paired digit layout (BK = 16).  The A box of a stage is then
// L / 2 tiles of 128 rows x 64 bytes, one per digit pair, and digit s sits 32 bytes into
// the rows of tile s / 2; B likewise.  The MMAs are issued in the same order as with the
// digit-major layout at any BK (per 16-deep step of K, the pairs (sa, sb) in the same
// order), so the two layouts give bit-identical products.
//
// CTAS = 2: the two CTAs of a cluster (row tiles mt = 2c, 2c + 1 along x of the grid, the
// same columns) form
// one M = 256 product (tcgen05 cta_group::2).  Each CTA loads its own 128 rows of A and
// one of the two B planes of the stage (64 rows: rank 0 the Re-C plane, rank 1 the
// Im-C plane); all four copies signal the barrier of rank 0, whose single thread issues
// every MMA of the pair.  Each SM's tensor core reads its A tile and half the B tile
// from its own shared memory and the other half from its partner's, so the operand
// traffic through one SM's shared memory per MMA drops from 8 KiB to 6 KiB and the
// bytes it loads per stage by a quarter.  TMEM accumulators, layout and epilogue are
// those of the single-CTA form (each CTA holds its 128 rows).
template <int L, int STAGES, int BK, bool PAIRS, int CTAS = 1>
__global__ void __launch_bounds__(SG_THREADS, 1)
split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  int d, int Kp, int Mp, int Np, int beta, const int* __restrict__ ea,
                  const int* __restrict__ eb, double* __restrict__ C, long long sC, SplitEpi epi,
                  int* __restrict__ status, SplitCtl ctl) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int TILE_BYTES = StageK<BK>::tile_bytes;
  constexpr int B_TILE_BYTES = TILE_BYTES / CTAS;   // one CTA's share of a digit's B tile
  constexpr int STAGE_BYTES = L * (TILE_BYTES + B_TILE_BYTES);   // loaded into this CTA per stage
  constexpr int RING_BYTES = STAGES * STAGE_BYTES > SG_EPI_BYTES ? STAGES * STAGE_BYTES : SG_EPI_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + RING_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint64_t* never = accfull + 1;   // no thread ever arrives here (the stall test waits on it)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* eb_s = abort_flag + 1;   // column exponents of this tile's 64 (real mode: 128) columns
  int* epi_flag = eb_s + 2 * SG_BNC;  // epilogue verdict (accumulators ready and no abort)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a CTA pair lies along x of the grid (clusters of 2 x 1 x 1): row tiles on x there
  const int nt = CTAS == 2 ? blockIdx.y : blockIdx.x, mt = CTAS == 2 ? blockIdx.x : blockIdx.y, b = blockIdx.z;
  // uniform over the CTA (and over a CTA pair, which shares b): no cluster barrier is reached
  if (ctl.item_sq && ctl.item_sq[b] <= ctl.sq_step) return;
  const uint32_t crank = CTAS == 2 ? cluster_rank() : 0u;
  const bool leader = crank == 0;
  const int num_k = Kp / BK;
  const int nkh = num_k / 2;   // K stages of the real half
  // operand structure (uniform over the launch; see SplitCtl): the K stages [kbeg, kend)
  // are loaded and multiplied; bz != 0 (one CTA per tile only) selects N = 64 products
  const int az = ctl.a_zero == 3 ? 0 : ctl.a_zero;
  const int bzr = ctl.b_zero == 3 ? 0 : ctl.b_zero;
  const int bz = CTAS == 1 ? bzr : 0;
  const int kbeg = (az & 1) ? nkh : 0, kend = (az & 2) ? nkh : num_k;
  // Real mode (CTA pairs, both operands with a zero part): the one active half of K times
  // the one B plane it meets is a single real product into one output half (rh: 0 Re C,
  // 1 Im C).  The pair's M = 256 x N = 128 MMAs then cover 128 output columns of that half:
  // each CTA loads 64 rows of the plane, tiles are 128 complex columns wide (TNC), and the
  // epilogue writes them in two passes of 64 with the other half zero.
  const bool real_mode = CTAS == 2 && az != 0 && bzr != 0;
  const int rh = (bzr & 2) ? (kbeg == nkh ? 1 : 0) : (kbeg == nkh ? 0 : 1);
  const int TNC = real_mode ? 2 * SG_BNC : SG_BNC;
  // a symmetric product computes no tile (of a CTA pair: no pair of tiles) whose columns
  // all lie right of all its rows; split_gemm then copies the entries above the diagonal
  if (ctl.sym_out && nt * TNC >= (CTAS == 2 ? ((mt | 1) + 1) : (mt + 1)) * SG_BM)
    return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp >= 2 && warp < 2 + TNC / 32) {
    const int c = (warp - 2) * 32 + lane, j = nt * TNC + c;
    eb_s[c] = j < d ? eb[(long long)b * (Np / 2) + j] : 0;
  }
  if (warp == 1) {
    if constexpr (CTAS == 2) {
      // one warp of each CTA of the pair takes part; each CTA receives its own address
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(512)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(512)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  // both CTAs' barriers initialised and TMEM allocated before any copy or MMA of the pair
  if constexpr (CTAS == 2) cluster_sync_all();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t t_start = global_ns();
  const uint64_t deadline = t_start + SG_WAIT_NS;   // waits that must not be abandoned early
  const uint64_t deadline_short = t_start + (ctl.wait_ns < SG_WAIT_NS ? ctl.wait_ns : SG_WAIT_NS);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int issued = 0;
      for (int kb = kbeg; kb < kend; ++kb) {
        const int i = kb - kbeg;   // position in the ring's sequence of stages
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, deadline_short)) {
          atomicExch(status, MG_DEV_TIMEOUT);
          *(volatile int*)abort_flag = 1;
          break;
        }
        unsigned char* st = smem + s * STAGE_BYTES;
        // B: the same K range in both halves of K; planes [Re B; Im B] (1, 2) for the
        // real half, [-Im B; Re B] (0, 1) for the imaginary half
        const bool imag = kb >= nkh;
        const int kbb = imag ? kb - nkh : kb;
        const int plane0 = imag ? 0 : 1;
        if constexpr (CTAS == 2) {
          // rank 0 expects the bytes of both CTAs; the copies of both signal its barrier
          if (leader) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
          const uint32_t bar = cluster_addr(&full[s], 0);
          // the B rows this CTA loads: one plane of the tile's 64 columns each, or in real
          // mode 64 of the tile's 128 columns of the one plane the active half of K meets
          // (Re B where Im B = 0; else Im B for the real half of K, -Im B for the imaginary)
          const int brow = real_mode ? nt * 2 * SG_BNC + SG_BNC * (int)crank : nt * SG_BNC;
          const int bplane = real_mode ? ((bzr & 2) ? 1 : (imag ? 0 : 2)) : plane0 + (int)crank;
          if constexpr (PAIRS) {
            tma_load_4d_pair(st, &tmA, bar, 0, kb, mt * SG_BM, b * (L / 2));
            tma_load_5d_pair(st + L * TILE_BYTES, &tmB, bar, 0, kbb, brow, bplane, b * (L / 2));
          } else {
            tma_load_4d_pair(st, &tmA, bar, kb * BK, mt * SG_BM, 0, b);
            tma_load_5d_pair(st + L * TILE_BYTES, &tmB, bar, kbb * BK, brow, bplane, 0, b);
          }
        } else if constexpr (PAIRS) {
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_4d(st, &tmA, &full[s], 0, kb, mt * SG_BM, b * (L / 2));
          tma_load_5d(st + L * TILE_BYTES, &tmB, &full[s], 0, kbb, nt * SG_BNC, plane0, b * (L / 2));
        } else {
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_4d(st, &tmA, &full[s], kb * BK, mt * SG_BM, 0, b);
          tma_load_5d(st + L * TILE_BYTES, &tmB, &full[s], kbb * BK, nt * SG_BNC, plane0, 0, b);
        }
        issued = i + 1;
      }
      // never leave the CTA with a bulk copy still in flight into its shared memory.  In
      // a pair the barriers of rank 0 count the copies of both CTAs: rank 0 drains them,
      // and rank 1 leaves only after the closing cluster barrier, which rank 0 reaches
      // after this drain.  (Both producers wait on commits issued together, so they
      // issue the same stages; a timeout is the one way they could differ.)
      if (CTAS == 1 || leader) {
        const uint64_t drain_deadline = global_ns() + SG_WAIT_NS;
        for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
          mbar_wait(&full[i % STAGES], (i / STAGES) & 1, drain_deadline);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer ----------------
      bool ok = true;
      if (ctl.stall && !mbar_wait(never, 0, deadline_short)) {
        atomicExch(status, MG_DEV_TIMEOUT);
        ok = false;
      }
      // N = 64 products (bz != 0): each half of K feeds one output half, from one B plane
      // (the tile's first or second 64 rows): with Im B = 0 the real half feeds Re C from
      // Re B and the imaginary half Im C from Re B; with Re B = 0 the real half feeds Im C
      // from Im B and the imaginary half Re C from -Im B
      constexpr uint32_t B_HALF = PAIRS ? B_TILE_BYTES : B_TILE_BYTES / 2;
      for (int kb = kbeg; kb < kend && ok; ++kb) {
        const int i = kb - kbeg;
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(&full[s], ph, deadline_short)) {
          atomicExch(status, MG_DEV_TIMEOUT);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
        const int oh = bz == 0 ? 0 : ((bz & 2) ? (kb >= nkh) : (kb < nkh));   // output half (N = 64)
        // in a pair: this CTA's half, the partner's at the same offset
        const uint32_t b0 = a0 + L * TILE_BYTES + (uint32_t)oh * B_HALF;
        const uint32_t dcol = (uint32_t)oh * SG_BNC;
        const uint32_t idesc = bz ? kIdescBf16N64 : kIdescBf16;
        // the first stage of an accumulator: the first loaded one, and with N = 64 the
        // first of each half of K (which writes the other output half)
        const bool fst = kb == kbeg || (bz != 0 && kb == nkh);
        bool first[SG_GROUPS] = {fst, fst, fst, fst};
#pragma unroll
        for (int kk = 0; kk < BK / SG_MMA_K; ++kk) {
#pragma unroll
          for (int sa = 0; sa < L; ++sa) {
#pragma unroll
            for (int sb = 0; sb < L - sa; ++sb) {
              const int g = (sa + sb) < SG_GROUPS - 1 ? (sa + sb) : SG_GROUPS - 1;
              const uint32_t acc = first[g] ? 0u : 1u;
              first[g] = false;
              uint64_t ad, bd;
              if constexpr (PAIRS) {
                // digit s: tile s / 2 (two digits per row), 16-value block kk, the odd digit's
                // 16 values after the even one's
                ad = pair_desc<BK>(a0 + (sa >> 1) * 2 * TILE_BYTES + kk * 4 * SG_MMA_K + (sa & 1) * SG_MMA_K * 2);
                bd = pair_desc<BK>(b0 + (sb >> 1) * 2 * B_TILE_BYTES + kk * 4 * SG_MMA_K + (sb & 1) * SG_MMA_K * 2);
              } else {
                ad = kmajor_desc<BK>(a0 + sa * TILE_BYTES + kk * SG_MMA_K * 2);
                bd = kmajor_desc<BK>(b0 + sb * B_TILE_BYTES + kk * SG_MMA_K * 2);
              }
              if constexpr (CTAS == 2) tc_mma_bf16_pair(tmem + g * 128, ad, bd, kIdescBf16M256, acc);
              else tc_mma_bf16(tmem + g * 128 + dcol, ad, bd, idesc, acc);
            }
          }
        }
        if constexpr (CTAS == 2) tc_commit_pair(&empty[s]);
        else tc_commit(&empty[s]);
      }
      // the verdict is written before the accumulator barrier can complete
      if (!ok) {
        *(volatile int*)abort_flag = 1;
        if constexpr (CTAS == 2) {
          asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr(abort_flag, 1)), "r"(1) : "memory");
          asm volatile("fence.acq_rel.cluster;" ::: "memory");
        } else {
          __threadfence_block();
        }
      }
      // fires once every issued MMA has completed (in both CTAs of a pair)
      if constexpr (CTAS == 2) tc_commit_pair(accfull);
      else tc_commit(accfull);
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int q = warp & 3;                   // TMEM lane quarter this warp may access
    const int c0 = ((warp - 2) >> 2) * (SG_BNC / 2);   // first of this warp's 32 complex columns
    // one thread polls; all eight epilogue warps follow its verdict, so that they
    // either all reach both named barriers below or none does
    if (warp == 2 && lane == 0) {
      bool got;
      if constexpr (CTAS == 2) {   // acquire at cluster scope: the verdict may come from rank 0
        got = true;
        while (!mbar_try_wait_cluster(accfull, 0)) {
          if (global_ns() > deadline) {
            got = false;
            break;
          }
        }
      } else {
        got = mbar_wait(accfull, 0, deadline);
      }
      if (!got) atomicExch(status, MG_DEV_TIMEOUT);
      *epi_flag = (got && *(volatile int*)abort_flag == 0) ? 1 : 0;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(SG_EPI_WARPS * 32) : "memory");
    tc_fence_after();
    if (*(volatile int*)epi_flag != 0) {
      // pull this tile's addend rows into L2 while phase 1 drains TMEM (8 x 128-byte
      // lines cover a row's 64 complex double-float values)
      if (epi.add_n > 0) {
        const int et = threadIdx.x - 2 * 32, lines = TNC / 8;
        for (int idx = et; idx < epi.add_n * SG_BM * lines; idx += SG_EPI_WARPS * 32) {
          const int m = idx / (SG_BM * lines), rem = idx % (SG_BM * lines), rr = rem / lines, q = rem % lines;
          const int grow = mt * SG_BM + rr, j = nt * TNC + q * 8;
          if (grow < d && j < d) {
            const double* src = m == 0 ? epi.add_src[0] : (m == 1 ? epi.add_src[1] : epi.add_src[2]);
            const double* p = src + b * epi.add_stride + 4 * ((long long)grow * d + j);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
          }
        }
      }
      float4* stile = reinterpret_cast<float4*>(smem);
      const int r = q * 32 + lane;                 // tile-local row
      const int row = mt * SG_BM + r;
      const int Ea = row < d ? ea[(long long)b * Mp + row] : 0;
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      // output halves no MMA wrote (N = 64 products with one half of K skipped) are zero
      bool wr[2] = {true, true};
      if (bz) {
        wr[0] = wr[1] = false;
        if (kbeg == 0) wr[(bz & 2) ? 0 : 1] = true;     // the real half of K was multiplied
        if (kend == num_k) wr[(bz & 2) ? 1 : 0] = true; // the imaginary half was
      }
      const float4* addp[3];
#pragma unroll
      for (int m = 0; m < 3; ++m)
        addp[m] = epi.add_src[m] ? reinterpret_cast<const float4*>(epi.add_src[m] + b * epi.add_stride) : nullptr;
      float4* Cb = reinterpret_cast<float4*>(C + b * sC);
      const int ew = warp - 2;
      // one pass per 64 output columns (two in real mode, whose TMEM columns all hold
      // the one computed half)
      for (int pass = 0; pass * SG_BNC < TNC; ++pass) {
        const int cb = pass * SG_BNC;   // first tile column of this pass
        if (pass > 0) asm volatile("bar.sync 1, %0;" ::"n"(SG_EPI_WARPS * 32) : "memory");   // stile free
        // phase 1 (thread = row): TMEM -> level combine -> double-float tile in shared memory
        // (the stage ring is idle once every MMA has completed)
        constexpr int CW = 4;   // complex columns per step
        for (int jc = c0; jc < c0 + SG_BNC / 2; jc += CW) {
          uint32_t re_acc[SG_GROUPS][CW], im_acc[SG_GROUPS][CW];
#pragma unroll
          for (int g = 0; g < SG_GROUPS; ++g) {
            if (real_mode) {   // the computed half goes to re_acc first (moved below for rh = 1)
              tmem_ld4(lane_base + g * 128 + cb + jc, re_acc[g]);
              im_acc[g][0] = im_acc[g][1] = im_acc[g][2] = im_acc[g][3] = 0u;
            } else {
              if (wr[0]) tmem_ld4(lane_base + g * 128 + jc, re_acc[g]);
              else re_acc[g][0] = re_acc[g][1] = re_acc[g][2] = re_acc[g][3] = 0u;
              if (wr[1]) tmem_ld4(lane_base + g * 128 + SG_BNC + jc, im_acc[g]);
              else im_acc[g][0] = im_acc[g][1] = im_acc[g][2] = im_acc[g][3] = 0u;
            }
          }
          tmem_wait_ld();
          if (real_mode && rh == 1) {
#pragma unroll
            for (int g = 0; g < SG_GROUPS; ++g)
#pragma unroll
              for (int jj = 0; jj < CW; ++jj) {
                im_acc[g][jj] = re_acc[g][jj];
                re_acc[g][jj] = 0u;
              }
          }
#pragma unroll
          for (int jj = 0; jj < CW; ++jj) {
            const int k = Ea + eb_s[cb + jc + jj] + 2 - 2 * beta;
            // levels that no digit pair reaches (L < 4) were never written: they hold
            // whatever an earlier kernel left in TMEM and must not be read as data
            const df32 re = combine_levels(re_acc[0][jj], L > 1 ? re_acc[1][jj] : 0u, L > 2 ? re_acc[2][jj] : 0u,
                                           L > 3 ? re_acc[3][jj] : 0u, k);
            const df32 im = combine_levels(im_acc[0][jj], L > 1 ? im_acc[1][jj] : 0u, L > 2 ? im_acc[2][jj] : 0u,
                                           L > 3 ? im_acc[3][jj] : 0u, k);
            stile[r * SG_EPI_PITCH + jc + jj] = make_float4(re.hi, re.lo, im.hi, im.lo);
          }
        }
        tc_fence_before();
        asm volatile("bar.sync 1, %0;" ::"n"(SG_EPI_WARPS * 32) : "memory");
        // phase 2 (warp = row, lane = column): addends and coalesced row stores
        // The warp's (row, half) items, EPI_GROUP at a time: every addend load of a group
        // is issued before the first is used, so that a warp keeps several rows of loads
        // in flight (one row at a time left the addend products latency-bound).
        constexpr int HALVES = SG_BNC / 32;
        constexpr int ITEMS = (SG_BM / SG_EPI_WARPS) * HALVES;
        constexpr int EPI_GROUP = 4;
        for (int i0 = 0; i0 < ITEMS; i0 += EPI_GROUP) {
          float4 ad[EPI_GROUP][3];
          long long offs[EPI_GROUP];
          bool ok[EPI_GROUP];
#pragma unroll
          for (int u = 0; u < EPI_GROUP; ++u) {
            const int it = i0 + u, rr = ew + SG_EPI_WARPS * (it / HALVES), c = (it % HALVES) * 32 + lane;
            const int grow = mt * SG_BM + rr, j = nt * TNC + cb + c;
            ok[u] = grow < d && j < d;
            offs[u] = ok[u] ? (long long)grow * d + j : 0;
#pragma unroll
            for (int m = 0; m < 3; ++m)
              ad[u][m] = (ok[u] && m < epi.add_n) ? addp[m][offs[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < EPI_GROUP; ++u) {
            if (!ok[u]) continue;
            const int it = i0 + u, rr = ew + SG_EPI_WARPS * (it / HALVES), c = (it % HALVES) * 32 + lane;
            const float4 v = stile[rr * SG_EPI_PITCH + c];
            df32 re{v.x, v.y}, im{v.z, v.w};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              if (m < epi.add_n) {
                re = df_add(re, df_mul(df32{ad[u][m].x, ad[u][m].y}, epi.add_coef[m]));
                im = df_add(im, df_mul(df32{ad[u][m].z, ad[u][m].w}, epi.add_coef[m]));
              }
            }
            if (mt * SG_BM + rr == nt * TNC + cb + c) re = df_add(re, epi.diag);
            Cb[offs[u]] = make_float4(re.hi, re.lo, im.hi, im.lo);
          }
        }
      }
    }
    tc_fence_before();
  }
  // a pair: neither CTA frees TMEM or leaves while its partner may still use them
  if constexpr (CTAS == 2) {
    __syncwarp();
    cluster_sync_all();
  } else {
    __syncthreads();
  }
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if constexpr (CTAS == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// C_ij = C_ji for every i < j of a symmetric matrix in lower-block storage: the blocks
// right of the diagonal and the upper halves of the diagonal blocks (whose entries, where
// a product computed them, differ from their transposes by the rounding order of the
// level->=3 accumulator).  Every source lies on or below the diagonal and is never written
// here, so the result is exactly symmetric.  One 32 x 32 block per CTA: grid (ceil(d/32),
// ceil(d/32), batch), blocks below the diagonal return at once; 256 threads; DF32
// storage (float4 per element).
__global__ void __launch_bounds__(256)
sym_mirror_kernel(int d, float4* __restrict__ C, long long sC4, const int* __restrict__ item_sq, int sq_step) {
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, b = blockIdx.z;
  if (j0 < i0) return;
  if (item_sq && item_sq[b] <= sq_step) return;
  __shared__ float4 t[32][33];
  float4* Cb = C + b * sC4;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {   // source rows j0 + r, columns i0 + tx
    const int si = j0 + r, sj = i0 + tx;
    if (si < d && sj < d) t[r][tx] = Cb[(long long)si * d + sj];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int di = i0 + r, dj = j0 + tx;
    if (di < dj && dj < d) Cb[(long long)di * d + dj] = t[tx][r];
  }
}

// ---------------------------------------------------------------------------
// host side: tensor maps, launches, workspace
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static int get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) {
    set_last_message("cuTensorMapEncodeTiled is not available from the CUDA driver");
    return MG_ECUDA;
  }
  return MG_OK;
}

// 4-D map over digit tiles: (k, row, slice, batch), box (32, box_rows, box_slices, 1), SWIZZLE_64B.
// B digits: dims {Kh, d valid rows (of Np / 2 allocated), 3 planes, L, batch};
// box {32, 64, planes, digits, 1}; rows from d on read as zeros
static int make_bplane_map(CUtensorMap* map, const void* base, int Kh, int rows, int valid_rows, int L, int batch,
                           int box_planes, int box_digits, int bk) {
  MG_TRY(get_encoder());
  cuuint64_t dims[5] = {(cuuint64_t)Kh, (cuuint64_t)valid_rows, 3, (cuuint64_t)L, (cuuint64_t)batch};
  cuuint64_t strides[4] = {(cuuint64_t)Kh * 2, (cuuint64_t)rows * Kh * 2, (cuuint64_t)3 * rows * Kh * 2,
                           (cuuint64_t)L * 3 * rows * Kh * 2};
  cuuint32_t box[5] = {(cuuint32_t)bk, (cuuint32_t)SG_BNC, (cuuint32_t)box_planes, (cuuint32_t)box_digits, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_message("cuTensorMapEncodeTiled failed (%d): Kh=%d rows=%d L=%d batch=%d", (int)r, Kh, rows, L, batch);
    return MG_ECUDA;
  }
  return MG_OK;
}
// A digits: dims {Kp, d valid rows (of `rows` allocated), L, batch}; rows from d on read as zeros
static int make_digit_map(CUtensorMap* map, const void* base, int Kp, int rows, int valid_rows, int L, int batch,
                          int bk, int box_rows = SG_BM, int box_slices = -1) {
  MG_TRY(get_encoder());
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)valid_rows, (cuuint64_t)L, (cuuint64_t)batch};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2, (cuuint64_t)L * rows * Kp * 2};
  cuuint32_t box[4] = {(cuuint32_t)bk, (cuuint32_t)box_rows, (cuuint32_t)(box_slices < 0 ? L : box_slices), 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_message("cuTensorMapEncodeTiled failed (%d): Kp=%d rows=%d L=%d batch=%d", (int)r, Kp, rows, L,
                     batch);
    return MG_ECUDA;
  }
  return MG_OK;
}

// Paired layout (even L), stages bk = 16 or 32 deep: the two digits' values of bk
// consecutive k form one row of 4 bk bytes (the layout keeps 16-value blocks of the even
// and the odd digit in turn, so 32-deep stages read two blocks).  A dims {2 bk, Kp / bk,
// d valid rows, batch * L / 2 digit pairs}, box {2 bk, 1, 128, L / 2}; B dims {2 bk,
// Kh / bk, d valid rows, 3 planes, batch * L / 2}, box {2 bk, 1, 64, planes, L / 2}.
// SWIZZLE_64B for 64-byte rows, SWIZZLE_128B for 128-byte rows.
static int make_pair_maps(CUtensorMap* ma, CUtensorMap* mb, const SplitGeom& g, const void* Ad, const void* Bd,
                          int batch, int bk, int b_planes) {
  MG_TRY(get_encoder());
  const int L = g.L, Kp = g.Kp, Kh = g.Kh(), rows = g.Np / 2;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapSwizzle sw = bk == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  {
    cuuint64_t dims[4] = {(cuuint64_t)(2 * bk), (cuuint64_t)(Kp / bk), (cuuint64_t)g.d, (cuuint64_t)batch * (L / 2)};
    cuuint64_t strides[3] = {(cuuint64_t)(4 * bk), (cuuint64_t)Kp * 4, (cuuint64_t)g.Mp * Kp * 4};
    cuuint32_t box[4] = {(cuuint32_t)(2 * bk), 1, (cuuint32_t)SG_BM, (cuuint32_t)(L / 2)};
    CUresult r = g_encode(ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(Ad), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_last_message("cuTensorMapEncodeTiled failed (%d): paired A, Kp=%d L=%d batch=%d", (int)r, Kp, L, batch);
      return MG_ECUDA;
    }
  }
  {
    cuuint64_t dims[5] = {(cuuint64_t)(2 * bk), (cuuint64_t)(Kh / bk), (cuuint64_t)g.d, 3,
                          (cuuint64_t)batch * (L / 2)};
    cuuint64_t strides[4] = {(cuuint64_t)(4 * bk), (cuuint64_t)Kh * 4, (cuuint64_t)rows * Kh * 4,
                             (cuuint64_t)3 * rows * Kh * 4};
    cuuint32_t box[5] = {(cuuint32_t)(2 * bk), 1, (cuuint32_t)SG_BNC, (cuuint32_t)b_planes, (cuuint32_t)(L / 2)};
    CUresult r = g_encode(mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(Bd), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_last_message("cuTensorMapEncodeTiled failed (%d): paired B, Kh=%d L=%d batch=%d", (int)r, Kh, L, batch);
      return MG_ECUDA;
    }
  }
  return MG_OK;
}

// Whether a product runs on CTA pairs.  By default pairs run from 5 digits (measured at 6:
// +3% at d = 729, +7% at d = 4096, +6% at d = 256; with 2-4 digits 2-4% slower) where the
// row tiles pair up evenly from d = 256 on, or are 7 or more (an odd count leaves the last
// pair's second CTA multiplying zeros: -19% at d = 300, three tiles).  A product with a
// zero part of B and a general A runs N = 64 MMAs on one CTA per tile; with zero parts in
// both it may run in the real mode of a pair.
static bool split_uses_pairs(const SplitGeom& g, const SplitCtl& ctl) {
  const int mtiles = g.Mp / SG_BM;
  const bool shape_ok = (mtiles % 2 == 0) ? g.d >= 256 : mtiles >= 7;
  const bool bstruct = ctl.b_zero == 1 || ctl.b_zero == 2;
  const bool astruct = ctl.a_zero == 1 || ctl.a_zero == 2;
  // a symmetric product of general operands by default on single CTAs: its 128-row tiles
  // follow the diagonal more closely than a pair's 256 rows (d = 729: 42 of 72 tiles
  // against 24 of 36 pairs, 58% of the work against 67%)
  const bool sym_single = ctl.sym_out && !(astruct && bstruct);
  return mtiles >= 2 && (!bstruct || astruct) &&
         (ctl.cta_pairs > 0 || (ctl.cta_pairs < 0 && g.L >= 5 && shape_ok && !sym_single));
}

// Complex output columns per tile: 128 in the real mode of CTA pairs (both operands with a
// zero part: one real product into one output half), else 64.
static int split_tile_cols(const SplitGeom& g, const SplitCtl& ctl) {
  const bool real_mode = (ctl.a_zero == 1 || ctl.a_zero == 2) && (ctl.b_zero == 1 || ctl.b_zero == 2) &&
                         split_uses_pairs(g, ctl);
  return real_mode ? 2 * SG_BNC : SG_BNC;
}

// bytes one CTA loads per pipeline stage (a CTA pair splits the B tile)
template <int L, int BK, int CTAS>
static constexpr int stage_bytes() {
  return L * (StageK<BK>::tile_bytes + StageK<BK>::tile_bytes / CTAS);
}
template <int L, int BK, int CTAS = 1>
static constexpr int stages_for() {
  // ring budget 224 KiB (the opt-in limit is 227 KiB per block; 2 KiB go to barriers and alignment)
  return (229376 / stage_bytes<L, BK, CTAS>()) > 8 ? 8
         : ((229376 / stage_bytes<L, BK, CTAS>()) < 1 ? 1 : (229376 / stage_bytes<L, BK, CTAS>()));
}

template <int L, int BK, bool PAIRS = false, int CTAS = 1>
static int launch_split_gemm_LB(const SplitGeom& g, int batch, const __nv_bfloat16* Ad, const int* ea,
                                const __nv_bfloat16* Bd, const int* eb, double* C, long long sC,
                                const SplitEpi& epi, int* status, const SplitCtl& ctl, cudaStream_t s) {
  static_assert(!PAIRS || ((BK == 16 || BK == 32) && L % 2 == 0), "the paired layout: 16- or 32-deep stages, even L");
  constexpr int STAGES = stages_for<L, BK, CTAS>();
  CUtensorMap ma, mb;
  if constexpr (PAIRS) {
    MG_TRY(make_pair_maps(&ma, &mb, g, Ad, Bd, batch, BK, CTAS == 2 ? 1 : 2));
  } else {
    MG_TRY(make_digit_map(&ma, Ad, g.Kp, g.Mp, g.d, L, batch, BK));
    // a CTA of a pair loads one of the two planes of the stage
    MG_TRY(make_bplane_map(&mb, Bd, g.Kh(), g.Np / 2, g.d, L, batch, CTAS == 2 ? 1 : 2, L, BK));
  }
  const size_t ring = std::max<size_t>((size_t)STAGES * stage_bytes<L, BK, CTAS>(), (size_t)SG_EPI_BYTES);
  const size_t smem = ring + 1024 /*barriers, exponents*/ + 1024 /*align*/;
  auto kern = split_gemm_kernel<L, STAGES, BK, PAIRS, CTAS>;
  MG_TRY(ensure_smem_limit(reinterpret_cast<const void*>(kern), (int)smem));
  const int mtiles = g.Mp / SG_BM;
  if constexpr (CTAS == 1) {
    kern<<<dim3(ceil_div(g.d, SG_BNC), mtiles, batch), SG_THREADS, smem, s>>>(
        ma, mb, g.d, g.Kp, g.Mp, g.Np, g.beta, ea, eb, C, sC, epi, status, ctl);
    return check_launch("split_gemm_kernel");
  } else {
    // pairs of row tiles; with an odd count the last pair's second CTA lies wholly
    // beyond row d (its loads read zeros, its epilogue writes nothing)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ceil_div(mtiles, 2) * 2, ceil_div(g.d, split_tile_cols(g, ctl)), batch);
    cfg.blockDim = dim3(SG_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ma, mb, g.d, g.Kp, g.Mp, g.Np, g.beta, ea, eb, C, sC, epi,
                                             status, ctl);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "cudaLaunchKernelEx(split_gemm_kernel, CTA pairs)", __FILE__, __LINE__);
      return MG_ECUDA;
    }
    return check_launch("split_gemm_kernel");
  }
}

template <int L, int CTAS>
static int launch_split_gemm_LC(const SplitGeom& g, int batch, const __nv_bfloat16* Ad, const int* ea,
                                const __nv_bfloat16* Bd, const int* eb, double* C, long long sC,
                                const SplitEpi& epi, int* status, const SplitCtl& ctl, cudaStream_t s) {
  // 16-deep stages also where a 32-deep stage leaves room for only one (L = 8 on one
  // CTA: no overlap of loads and MMAs; 35 -> 53 algorithmic TFLOP/s measured at d = 512)
  if (ctl.stage_k == 16 || stages_for<L, 32, CTAS>() < 2)
    return launch_split_gemm_LB<L, 16, false, CTAS>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
  // 64 only where each half of K is a whole number of 64-wide stages and two stages fit
  if constexpr (stages_for<L, 64, CTAS>() >= 2)
    if (ctl.stage_k == 64 && g.Kh() % 64 == 0)
      return launch_split_gemm_LB<L, 64, false, CTAS>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
  return launch_split_gemm_LB<L, 32, false, CTAS>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
}

template <int L>
static int launch_split_gemm_L(const SplitGeom& g, int batch, const __nv_bfloat16* Ad, const int* ea,
                               const __nv_bfloat16* Bd, const int* eb, double* C, long long sC,
                               const SplitEpi& epi, int* status, const SplitCtl& ctl, cudaStream_t s) {
  const bool pair = split_uses_pairs(g, ctl);
  if constexpr (L % 2 == 0) {
    if (paired_layout(g, ctl)) {
      // pairs = 2: 32-deep stages of 128-byte rows where two stages fit, else 16-deep
      if (ctl.pairs == 2) {
        if constexpr (stages_for<L, 32, 2>() >= 2)
          if (pair) return launch_split_gemm_LB<L, 32, true, 2>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
        if constexpr (stages_for<L, 32, 1>() >= 2)
          if (!pair) return launch_split_gemm_LB<L, 32, true, 1>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
      }
      if (pair) return launch_split_gemm_LB<L, 16, true, 2>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
      return launch_split_gemm_LB<L, 16, true, 1>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
    }
  }
  if (pair) return launch_split_gemm_LC<L, 2>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
  return launch_split_gemm_LC<L, 1>(g, batch, Ad, ea, Bd, eb, C, sC, epi, status, ctl, s);
}

template <int L, typename T>
static int launch_slicers_LT(const SplitGeom& g, int batch, const double* A, long long sA, __nv_bfloat16* Ad,
                             int* ea, const double* B, long long sB, __nv_bfloat16* Bd, int* eb, cudaStream_t s,
                             const SplitCtl& ctl) {
  if (A) {
    slice_a_kernel<L, T><<<dim3(g.Mp / 8, batch), 256, 0, s>>>(g.d, g.Kp, g.Mp, g.beta, A, sA, Ad, ea, ctl.item_sq,
                                                                ctl.sq_step, g.a_item_elems(), paired_layout(g, ctl));
    MG_TRY(check_launch("slice_a_kernel"));
  }
  if (B) {
    MG_CUDA_TRY(cudaMemsetAsync(eb, 0x80, sizeof(int) * (size_t)(g.Np / 2) * batch, s));
    col_exponent_kernel<T><<<dim3(ceil_div(g.d, SG_BNC), ceil_div(g.d, 64), batch), 256, 0, s>>>(
        g.d, g.Np, B, sB, eb, ctl.item_sq, ctl.sq_step);
    MG_TRY(check_launch("col_exponent_kernel"));
    slice_b_kernel<L, T><<<dim3(ceil_div(g.d, SG_BNC), ceil_div(g.d, SB_KCHUNK), batch), 256, 0, s>>>(
        g.d, g.Kp, g.Np, g.beta, B, sB, Bd, eb, ctl.item_sq, ctl.sq_step, g.b_item_elems(), paired_layout(g, ctl));
    MG_TRY(check_launch("slice_b_kernel"));
  }
  return MG_OK;
}

template <int L>
static int launch_slice_sym_L(const SplitGeom& g, int batch, const double* M, long long sM, __nv_bfloat16* Ad,
                              int* ea, int askip, __nv_bfloat16* Bd, int* eb, int bskip, cudaStream_t s,
                              const SplitCtl& ctl) {
  const int nb = ceil_div(g.d, 32);
  const float4* M4 = reinterpret_cast<const float4*>(M);
  if (Ad) MG_CUDA_TRY(cudaMemsetAsync(ea, 0x80, sizeof(int) * (size_t)g.Mp * batch, s));
  if (Bd) MG_CUDA_TRY(cudaMemsetAsync(eb, 0x80, sizeof(int) * (size_t)(g.Np / 2) * batch, s));
  sym_exponent_kernel<<<dim3(nb, nb, batch), 256, 0, s>>>(g.d, M4, sM / 2, Ad ? ea : eb, Ad ? g.Mp : g.Np / 2,
                                                          Ad && Bd ? eb : nullptr, g.Np / 2, ctl.item_sq,
                                                          ctl.sq_step);
  MG_TRY(check_launch("sym_exponent_kernel"));
  slice_sym_block_kernel<L><<<dim3(g.Kh() / 32, nb, batch), 256, 0, s>>>(
      g.d, g.Kp, g.Mp, g.beta, M4, sM / 2, Ad, ea, g.a_item_elems(), askip, Bd, eb, g.b_item_elems(), g.Np / 2,
      bskip, ctl.item_sq, ctl.sq_step, paired_layout(g, ctl));
  return check_launch("slice_sym_block_kernel");
}

template <int L>
static int launch_slicers_L(const SplitGeom& g, int batch, int in_df32, const double* A, long long sA,
                            __nv_bfloat16* Ad, int* ea, const double* B, long long sB, __nv_bfloat16* Bd, int* eb,
                            cudaStream_t s, const SplitCtl& ctl) {
  if (in_df32) return launch_slicers_LT<L, df32>(g, batch, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
  return launch_slicers_LT<L, double>(g, batch, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
}

static int launch_slicers(const SplitGeom& g, int batch, int in_df32, const double* A, long long sA,
                          __nv_bfloat16* Ad, int* ea, const double* B, long long sB, __nv_bfloat16* Bd, int* eb,
                          cudaStream_t s, const SplitCtl& ctl) {
  switch (g.L) {
    case 2: return launch_slicers_L<2>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 3: return launch_slicers_L<3>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 4: return launch_slicers_L<4>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 5: return launch_slicers_L<5>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 6: return launch_slicers_L<6>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 7: return launch_slicers_L<7>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
    case 8: return launch_slicers_L<8>(g, batch, in_df32, A, sA, Ad, ea, B, sB, Bd, eb, s, ctl);
  }
  return MG_EINVAL;
}

// Public-to-the-library entry points ------------------------------------------

// Digits of a complex symmetric matrix in lower-block storage (double-float) for the A
// operand (abuf), the B operand (bbuf) or both (either may be null); askip / bskip as in
// slice_sym_block_kernel.
int split_slice_sym(int d, int L, int batch, const double* M, long long sM, void* abuf, int askip, void* bbuf,
                    int bskip, cudaStream_t s, const SplitCtl& ctl) {
  SplitGeom g = split_geom(d, L);
  if (batch > 65535) return MG_EUNSUPPORTED;
  __nv_bfloat16* Ad = reinterpret_cast<__nv_bfloat16*>(abuf);
  int* ea = Ad ? reinterpret_cast<int*>(Ad + g.a_item_elems() * batch) : nullptr;
  __nv_bfloat16* Bd = reinterpret_cast<__nv_bfloat16*>(bbuf);
  int* eb = Bd ? reinterpret_cast<int*>(Bd + g.b_item_elems() * batch) : nullptr;
  switch (L) {
    case 2: return launch_slice_sym_L<2>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 3: return launch_slice_sym_L<3>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 4: return launch_slice_sym_L<4>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 5: return launch_slice_sym_L<5>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 6: return launch_slice_sym_L<6>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 7: return launch_slice_sym_L<7>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
    case 8: return launch_slice_sym_L<8>(g, batch, M, sM, Ad, ea, askip, Bd, eb, bskip, s, ctl);
  }
  return MG_EINVAL;
}

size_t split_a_bytes(int d, int L, int batch) {
  SplitGeom g = split_geom(d, L);
  return (size_t)g.a_item_elems() * 2 * batch + (size_t)g.Mp * 4 * batch;
}
size_t split_b_bytes(int d, int L, int batch) {
  SplitGeom g = split_geom(d, L);
  return (size_t)g.b_item_elems() * 2 * batch + (size_t)(g.Np / 2) * 4 * batch;
}

// A-side digits of a batch (FP64 or DF32 input): layout [digits | exponents] in one buffer.
int split_slice_a(int d, int L, int batch, const double* A, long long sA, int in_df32, void* buf, cudaStream_t s,
                  const SplitCtl& ctl) {
  SplitGeom g = split_geom(d, L);
  __nv_bfloat16* Ad = reinterpret_cast<__nv_bfloat16*>(buf);
  int* ea = reinterpret_cast<int*>(Ad + g.a_item_elems() * batch);
  return launch_slicers(g, batch, in_df32, A, sA, Ad, ea, nullptr, 0, nullptr, nullptr, s, ctl);
}

int split_slice_b(int d, int L, int batch, const double* B, long long sB, int in_df32, void* buf, cudaStream_t s,
                  const SplitCtl& ctl) {
  SplitGeom g = split_geom(d, L);
  __nv_bfloat16* Bd = reinterpret_cast<__nv_bfloat16*>(buf);
  int* eb = reinterpret_cast<int*>(Bd + g.b_item_elems() * batch);
  return launch_slicers(g, batch, in_df32, nullptr, 0, nullptr, nullptr, B, sB, Bd, eb, s, ctl);
}

// C[b] = A[b] B[b] + addends (C and addends DF32), from digit buffers made by split_slice_a/b.
int split_gemm(int d, int L, int batch, const void* abuf, const void* bbuf, double* C, long long sC,
               const AddTerms& add, int* status, cudaStream_t s, const SplitCtl& ctl) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  if (add.scale != 1.0) return MG_EINVAL;
  SplitGeom g = split_geom(d, L);
  const __nv_bfloat16* Ad = reinterpret_cast<const __nv_bfloat16*>(abuf);
  const int* ea = reinterpret_cast<const int*>(Ad + g.a_item_elems() * batch);
  const __nv_bfloat16* Bd = reinterpret_cast<const __nv_bfloat16*>(bbuf);
  const int* eb = reinterpret_cast<const int*>(Bd + g.b_item_elems() * batch);
  SplitEpi e{};
  e.add_n = add.n;
  for (int m = 0; m < 3; ++m) { e.add_src[m] = add.src[m]; e.add_coef[m] = df_from_double(add.coef[m]); }
  e.add_stride = add.stride;
  e.diag = df_from_double(add.diag);
  int r = MG_EINVAL;
  switch (L) {
    case 2: r = launch_split_gemm_L<2>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 3: r = launch_split_gemm_L<3>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 4: r = launch_split_gemm_L<4>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 5: r = launch_split_gemm_L<5>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 6: r = launch_split_gemm_L<6>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 7: r = launch_split_gemm_L<7>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
    case 8: r = launch_split_gemm_L<8>(g, batch, Ad, ea, Bd, eb, C, sC, e, status, ctl, s); break;
  }
  // a symmetric result stays in lower-block storage: its consumers read the lower blocks
  return r;
}

// C_ij = C_ji for every i < j of a batch of symmetric matrices in lower-block storage (the
// full matrix, for a consumer that reads every entry).
int split_sym_fill(int d, int batch, double* C, long long sC, cudaStream_t s) {
  if (batch <= 0) return MG_OK;
  if (batch > 65535) return MG_EUNSUPPORTED;
  const int nb = ceil_div(d, 32);
  sym_mirror_kernel<<<dim3(nb, nb, batch), 256, 0, s>>>(d, reinterpret_cast<float4*>(C), sC / 2, nullptr, 0);
  return check_launch("sym_mirror_kernel");
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the split-precision product
// ---------------------------------------------------------------------------
// Its scratch (digit operands, the double-float product and the status word of
// the bounded waits) lives in one file-scope device array instead of memory
// from cudaMalloc.  The array exists on every device that loads this library,
// for the life of the process.  Host code must not pass the symbol itself to a
// kernel (on the host it only names a stand-in object): the device address is
// resolved once per device with cudaGetSymbolAddress, that device current.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[128];

static int static_scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (device < 0 || device >= 128) {
    set_last_message("mg_cgemm_split_static: device %d is outside 0..127", device);
    return MG_EINVAL;
  }
  if (!g_static_addr[device]) {
    int prev = 0;
    MG_CUDA_TRY(cudaGetDevice(&prev));
    MG_CUDA_TRY(cudaSetDevice(device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
      return MG_ECUDA;
    }
    g_static_addr[device] = p;
  }
  *out = g_static_addr[device];
  return MG_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t static_scratch_bytes_needed(int d, int L, int batch) {
  return 256 + align256(split_a_bytes(d, L, batch)) + align256(split_b_bytes(d, L, batch)) +
         align256((size_t)16 * d * d * batch);
}

}  // namespace mg

extern "C" int mg_cgemm_split_static(int device, void* stream, int batch, int d, const double* A, const double* B,
                                     double* C, int slices) {
  using namespace mg;
  if (batch < 1 || batch > 65535 || d < 1 || d > 4096 || !A || !B || !C || slices < 2 || slices > 8) {
    set_last_message("mg_cgemm_split_static: invalid argument");
    return MG_EINVAL;
  }
  const size_t need = static_scratch_bytes_needed(d, slices, batch);
  if (need > kStaticScratchBytes) {
    set_last_message("mg_cgemm_split_static: batch %d of d = %d with %d digits needs %zu bytes of scratch; "
                     "the static scratch holds %zu",
                     batch, d, slices, need, kStaticScratchBytes);
    return MG_EUNSUPPORTED;
  }
  int prev = 0;
  MG_CUDA_TRY(cudaGetDevice(&prev));
  void* base = nullptr;
  int r = static_scratch_address(device, &base);
  if (r != MG_OK) return r;
  MG_CUDA_TRY(cudaSetDevice(device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  int* status = reinterpret_cast<int*>(p);
  void* abuf = p + 256;
  void* bbuf = p + 256 + align256(split_a_bytes(d, slices, batch));
  double* prod = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(bbuf) +
                                           align256(split_b_bytes(d, slices, batch)));
  const long long md = 2LL * d * d;
  AddTerms none;
  int st = 0;
  // the status word is the only scratch that must start at zero; the digit
  // buffers (padding included) and the product are fully rewritten
  const cudaError_t me = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (me != cudaSuccess) {
    set_last_cuda_error(me, "cudaMemsetAsync(status word)", __FILE__, __LINE__);
    r = MG_ECUDA;
  }
  if (r == MG_OK) r = split_slice_a(d, slices, batch, A, md, 0, abuf, s);
  if (r == MG_OK) r = split_slice_b(d, slices, batch, B, md, 0, bbuf, s);
  if (r == MG_OK) r = split_gemm(d, slices, batch, abuf, bbuf, prod, md, none, status, s);
  if (r == MG_OK) r = launch_df_to_fp64(batch, d, prod, md, C, md, s);
  if (r == MG_OK) {
    const cudaError_t ce = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) {
      set_last_cuda_error(ce, "cudaMemcpyAsync(status word)", __FILE__, __LINE__);
      r = MG_ECUDA;
    }
  }
  if (r == MG_OK) {
    const cudaError_t se = cudaStreamSynchronize(s);
    if (se != cudaSuccess) {
      set_last_cuda_error(se, "cudaStreamSynchronize", __FILE__, __LINE__);
      r = MG_ECUDA;
    }
  }
  if (r == MG_OK && st == MG_DEV_TIMEOUT) {
    set_last_message("mg_cgemm_split_static: a bounded device-side wait gave up");
    r = MG_ETIMEOUT;
  }
  cudaSetDevice(prev);
  return r;
}

