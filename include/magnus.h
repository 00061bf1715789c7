/*
 * magnus.h -- C ABI of the GB300 first-order Magnus time-evolution library.
 *
 * The library evolves a driven Hamiltonian
 *
 *     H(t) = H0 + sum_k u^(k)(t) H_k                      (Eq. magnus-generic-ham)
 *
 * over N uniform Magnus intervals t_n = t0 + n dt.  For every interval it forms
 * the first-order Magnus term
 *
 *     Hbar_n = dt H0 + sum_k c_{k,n} H_k,                 (Eq. magnus-first-order-term)
 *     c_{k,n} = int_{t_n}^{t_n + dt} u^(k)(t) dt,         (Eq. magnus-first-order-coeff)
 *
 * exponentiates it to U_n = exp(-i Hbar_n) (hbar = 1), and carries a state or
 * the full propagator through the product U_{N-1} ... U_0 (later intervals on
 * the left).  This follows the paper's statement of the problem in Sec. "Time
 * Coarse-Graining Hamiltonians" and the package interface of App. A.5
 * (`magnus(tlist, drift_ham, control_sigs, control_hams)`,
 * `update_control_sigs()`, `evolve()`).
 *
 * Conventions
 *   - Complex matrices are d x d, row-major, interleaved (re, im) doubles:
 *     element (i, j) is at doubles [2(i d + j), 2(i d + j) + 1].  Vectors are d
 *     interleaved complex doubles.
 *   - Pointers are DEVICE pointers unless a call says otherwise or the
 *     MG_FLAG_HOST_PTRS flag is given.  The caller owns every buffer it passes;
 *     the library copies what it keeps (operators) into its own device memory.
 *   - Every call returns MG_OK (0) or a negative MG_E* code; mg_strerror()
 *     turns a code into text and mg_last_error_message() gives the detail of
 *     the most recent failure on the calling thread.  No C++ exception crosses
 *     this interface.
 *   - Work is queued on the context's CUDA stream.  Outputs are valid once that
 *     stream has been synchronised; calls that fill an mg_report synchronise
 *     the stream before returning.
 *   - The library requires a GPU of compute capability 10.3 (sm_103a).  There is
 *     no CPU fallback: without such a device mg_ctx_create fails with MG_ECUDA.
 */
#ifndef MAGNUS_H_
#define MAGNUS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define MG_OK            0
#define MG_EINVAL       -1   /* bad argument (size, null pointer, mode)            */
#define MG_ENOMEM       -2   /* device allocation failed                           */
#define MG_ECUDA        -3   /* a CUDA runtime/driver call failed                  */
#define MG_ENONFINITE   -4   /* NaN/Inf in a norm (bad samples or operators)       */
#define MG_ENOTHERM     -5   /* operator not Hermitian (MG_FLAG_CHECK_HERMITIAN)   */
#define MG_ETIMEOUT     -6   /* a bounded device-side wait gave up                 */
#define MG_EAGAIN       -7   /* not admissible now (serving: memory budget)        */
#define MG_EUNSUPPORTED -8   /* size or mode outside what the library supports     */

/* ---- precision modes ------------------------------------------------------ */
/* MG_PREC_FP64: every matrix product in native FP64 arithmetic.
 * MG_PREC_SPLIT: matrix products on the tcgen05 tensor cores.  Each operand row
 *   (column) is scaled by a power of two and cut into `slices` signed BF16
 *   digits of `beta` bits; digit products are accumulated in FP32 TMEM
 *   accumulators that stay exact for the leading digits, and combined in
 *   double-float (FP32 hi + lo, about 48 bits).  The exponential's intermediate
 *   matrices (powers, Taylor blocks, squarings, U_n) are stored and combined as
 *   double-float, and so is Hbar_n (formed with error-free FP32
 *   transformations from the operators and coefficients).  More slices give
 *   more accuracy (about beta*slices bits, down to the rounding of the FP32
 *   accumulators).  Operand entries are taken as FP32 pairs: magnitudes outside
 *   about 2^-100 .. 2^100 lose precision.  The quadrature, the trace phases, the
 *   norms' column sums, the state chain and re-orthonormalisation run in FP64. */
#define MG_PREC_FP64   0
#define MG_PREC_SPLIT  1
/* mg_job only: the server looks the job's configuration up in its context's
 * tuning cache (mg_ctx_set_tune_cache; see mg_plan_autotune). */
#define MG_PREC_AUTO   2

/* Taylor scheme of the exponential (mg_plan_set_taylor, tuning entries). */
#define MG_TAYLOR_AUTO 0  /* split precision may take degree 18 in five products */
#define MG_TAYLOR_PS   1  /* Paterson-Stockmeyer degrees only */

/* ---- outputs --------------------------------------------------------------- */
#define MG_OUT_STATE       0  /* psi(T) = U_{N-1} ... U_0 psi0            */
#define MG_OUT_PROPAGATOR  1  /* U(T)   = U_{N-1} ... U_0                 */
/* mg_evolve only: the stroboscopic states psi_n = U_{n-1} ... U_0 psi0 at every
 * interval end, n = 0..N, written as (N + 1) x d complex rows (row 0 = psi0). */
#define MG_OUT_TRAJECTORY  2

/* ---- flags ----------------------------------------------------------------- */
#define MG_FLAG_HOST_PTRS        1  /* the call's data pointers are host memory */
#define MG_FLAG_CHECK_HERMITIAN  2  /* plan: reject operators with |H - H^dag| > 1e-12 |H| */
#define MG_FLAG_NO_TRACE_SHIFT   4  /* plan: exponentiate Hbar_n itself, not Hbar_n - tr/d I */
/* plan: state outputs apply exp(-i Hbar_n) to the state instead of forming
 * U_n (Eq. magnus-first-order-term and the ordered product of the interval
 * propagators, evaluated by their action on psi): a Chebyshev expansion
 * (Tal-Ezer and Kosloff 1984) over the Gershgorin interval of Hbar_n, with
 * sparse (CSR) matrix-vector products in FP64; exact up to the unit roundoff,
 * cheaper whenever the operators are sparse.  One thread block per job, so it
 * suits batches of jobs or large sparse d.  Limits: d <= 4693, at most 255
 * operators (after the commutators of order 2), and a Gershgorin half-width of
 * Hbar_n of at most 327680 (16384 sub-steps of 20); beyond it the call (or the
 * job's batch status) returns MG_EUNSUPPORTED, a non-finite bound
 * MG_ENONFINITE.  The CSR copy of the operators is built on the host at the
 * first such call.  Propagator outputs are unaffected.  In the report,
 * taylor_degree is the largest Chebyshev degree, max/min_squarings the sub-step
 * counts and max_norm1 the largest half-width. */
#define MG_FLAG_STATE_ACTION     8

typedef struct mg_ctx mg_ctx;
typedef struct mg_plan mg_plan;

/* Per-call report (FP64 diagnostics).  Filled by mg_evolve when non-NULL. */
typedef struct mg_report {
  int32_t intervals;          /* Magnus intervals processed                     */
  int32_t taylor_degree;      /* Taylor degree m used by the exponential        */
  int32_t max_squarings;      /* largest squaring count s_n over the intervals  */
  int32_t min_squarings;      /* smallest s_n                                   */
  double  max_norm1;          /* largest ||Hbar_n - tau_n I||_1                 */
  double  unitarity_defect;   /* max|U^dag U - I| (propagator) or |‖psi‖ - 1|  */
  double  ms_total;           /* wall time of the call on the device stream     */
  int64_t matrix_products;    /* complex d x d products issued                  */
  int64_t sparse_matvecs;     /* operator applications (MG_FLAG_STATE_ACTION)   */
  int64_t sparse_nnz;         /* stored nonzeros of H0 and the H_k (same path)  */
  int64_t action_ctas;        /* CTAs per job of the action chain (1 or a cluster size) */
} mg_report;

/* ---- context ---------------------------------------------------------------- */
/* Create a context bound to CUDA device `device` and the CUDA stream `stream`
 * (a cudaStream_t cast to void*, NULL for the legacy default stream).  The
 * context owns the scratch workspace of later calls.  Fails with MG_ECUDA when
 * the device is absent or is not compute capability 10.3. */
int mg_ctx_create(mg_ctx** out, int device, void* stream);
int mg_ctx_destroy(mg_ctx* ctx);
/* Upper bound (bytes) on the scratch workspace the context may hold; default
 * 16 GiB.  Larger jobs are processed in interval chunks that fit. */
int mg_ctx_set_workspace_limit(mg_ctx* ctx, size_t bytes);

/* ---- quadrature ------------------------------------------------------------- */
/* Gauss-Legendre nodes x[p] and weights w[p] (p < P) on [-1, 1], HOST arrays.
 * The drive samples a plan consumes are u^(k) evaluated at
 *     t_{n,p} = t0 + n dt + (1 + x[p]) dt / 2,
 * so that c_{k,n} = (dt/2) sum_p w[p] u^(k)(t_{n,p}) integrates
 * Eq. magnus-first-order-coeff exactly for polynomial u of degree <= 2P - 1.
 * 1 <= P <= 64. */
int mg_quadrature_nodes(int P, double* x, double* w);

/* ---- sparse pattern of the action path (host only) ----------------------- */
/* The CSR form MG_FLAG_STATE_ACTION plans build from their nops = 1 + K dense
 * operators (`dense`: HOST, nops x d x d complex, H0 first): one pattern, the
 * union of the operators' nonzero entries plus the whole diagonal, with columns
 * ascending in each row, and one value array per operator on that pattern.
 * *nnz receives the pattern's size.  With rowptr NULL the call only reports
 * *nnz; otherwise rowptr (d + 1 ints), col (nnz ints), diag (d ints: the index in
 * col of each row's diagonal entry) and val (nops x nnz complex, operator-major)
 * are filled (HOST arrays).  1 <= d <= 4096, 1 <= nops <= 256. */
int mg_csr_pattern(int d, int nops, const double* dense, int64_t* nnz, int* rowptr, int* col, int* diag,
                   double* val);

/* ---- second-order weights (host only) ------------------------------------ */
/* The P x P matrix behind the second-order term (Eq. magnus-avg, second line) as
 * the plans of order 2 use it: with s_r = (1 + x_r)/2 the mg_quadrature_nodes
 * mapped to [0, 1] and l_r their Lagrange basis,
 *     M[p][q] = int_0^1 l_p(s1) int_0^{s1} l_q(s2) ds2 ds1,
 * so that the double integral over t_n <= t2 <= t1 <= t_n + dt of g(t1) f(t2) is
 * dt^2 sum_{p,q} g_p f_q M[p][q] for the interpolating polynomials of the samples.
 * M (HOST, P*P + 2P doubles) receives M row-major (row p: the t1 node), then the
 * column sums C_q, then the row sums R_p.  1 <= P <= 64. */
int mg_second_order_weights(int P, double* M);

/* ---- exponential parameters (host only) ---------------------------------- */
/* The Taylor degree m and squaring count s that mg_expm and mg_evolve take for a
 * batch whose largest FP64 1-norm of Hbar_n - tau_n I is norm1 (Sec. "Magnus
 * Expansion": U_n = exp(-i Hbar_n) by scaling and squaring), and theta, the
 * largest 1-norm that degree m takes unscaled: the largest theta with
 * sum_{j>m} theta^j / j! <= u theta, u = 2^-53 in FP64 and max(2^-53,
 * 2^(-beta slices)) in split precision (beta = the digit width the split
 * product uses at dimension d).  m is one of 2, 4, 6, 9, 12, 16 (Paterson-
 * Stockmeyer) or 18 (five products, split precision only); (m, s) minimises
 * products + s, ties to the smaller s.  No context or device is used.
 * Errors: MG_EINVAL for a negative or non-finite norm1, d outside 1..4096,
 * NULL outputs, or precision/slices as for plans. */
int mg_taylor_choice(double norm1, int precision, int slices, int d, int* m, int* s, double* theta);
/* Host only: the digit width beta of the split product at dimension d (the largest
 * beta <= 8 with 2^(2 beta - 1) 2d <= 2^24, which keeps the two leading accumulator
 * levels exact: 7 up to d = 1024, 6 up to 4096) and, in *slices, the digit count
 * ceil(bits / beta) clamped to 2..8 that carries at least `bits` bits (42 for the
 * default: 6 digits up to d = 1024, 7 above).  MG_EINVAL for d outside 1..4096 or
 * bits outside 1..64, or NULL outputs. */
int mg_split_digits(int d, int bits, int* beta, int* slices);

/* ---- plan: resident operators -------------------------------------------- */
/* Copy H0 (d x d) and H_k (K x d x d, consecutive) into device memory owned by
 * the plan.  `precision` is MG_PREC_FP64 or MG_PREC_SPLIT; `slices` (2..8) is
 * the number of BF16 digits per operand in MG_PREC_SPLIT (ignored for FP64).
 * Flags: MG_FLAG_HOST_PTRS (H0/Hk are host memory), MG_FLAG_CHECK_HERMITIAN,
 * MG_FLAG_NO_TRACE_SHIFT.  1 <= d <= 4096, 0 <= K <= 64. */
int mg_plan_create(mg_ctx* ctx, mg_plan** out, int d, int K, const double* H0,
                   const double* Hk, int precision, int slices, int flags);
/* Free the plan's device memory.  Does not use the plan's context, so plans may
 * be destroyed before or after their context. */
int mg_plan_destroy(mg_plan* plan);

/* Magnus order of the plan's exponents: 1 (the default, the paper's method) or 2,
 * which adds the second-order term of Eq. magnus-avg,
 *   Hbar^(2)_n = -(i/2) int int_{t_n <= t2 <= t1 <= t_n + dt} [H(t1), H(t2)],
 * as sum_k alpha_{k,n} (-i/2)[H0, H_k] + sum_{k<l} beta_{kl,n} (-i/2)[H_k, H_l]:
 * the K + K(K-1)/2 commutators are formed once here (FP64 products) and the
 * scalar double integrals alpha, beta come from the interpolating polynomial of
 * the P samples of each interval (exact for drives polynomial in t of degree
 * < P).  Takes effect with the next mg_set_controls (controls must be set again).
 * mg_evolve and mg_evolve_batch honour it; the server uses order 1. */
int mg_plan_set_magnus_order(mg_plan* plan, int order);

/* Replace the control signals (the `update_control_sigs()` step of App. A.5).
 * samples: N x P x K doubles, u^(k)(t_{n,p}) at the nodes documented at
 * mg_quadrature_nodes; w: the P quadrature weights (HOST array).  The samples
 * are copied into the plan.  flags: MG_FLAG_HOST_PTRS when `samples` is host
 * memory.  Any N >= 1 and 1 <= P <= 64. */
int mg_set_controls(mg_plan* plan, int N, int P, double t0, double dt, const double* w,
                    const double* samples, int flags);

/* Evolve through all N intervals of the current controls (`evolve()` of App. A.5).
 *   output = MG_OUT_STATE:      in = psi0 (d complex), out = psi(T) (d complex)
 *   output = MG_OUT_PROPAGATOR: in = NULL (identity start) or U0 (d x d),
 *                               out = U(T) U0 (d x d)
 *   output = MG_OUT_TRAJECTORY: in = psi0, out = psi_0 .. psi_N ((N + 1) x d
 *                               complex), the state at every interval end
 * A run can be resumed from any psi_n (or U) with controls for the remaining
 * intervals (t0 moved to t0 + n dt). 
 * reorth_every = R > 0 re-orthonormalises the running product every R
 * intervals in FP64 (propagator: one Newton-Schulz polar step
 * U <- U (3I - U^dag U)/2; state: psi <- psi/|psi|); 0 disables it.
 * flags: MG_FLAG_HOST_PTRS when in/out are host memory (the copies are then
 * part of the call).  rep may be NULL. */
int mg_evolve(mg_plan* plan, int output, const double* in, double* out, int reorth_every,
              int flags, mg_report* rep);

/* Evolve n independent jobs (plans with their controls set) of uneven
 * dimension and length together: jobs are grouped by precision mode and by
 * dimension rounded up to a multiple of 16 (zero padding is exact: the padded
 * block of exp(-i Hbar) is the identity), and within a group all intervals of
 * all jobs share one batched launch per step of the exponential, each interval
 * with its own squaring count (see mg_batch_graph_create).  Propagator
 * jobs fold each chunk by a tree product; state jobs of d <= 256 (without
 * renormalisation) reduce each chunk by a segmented tree shared by all jobs and
 * then advance in one multi-job launch, larger ones by matrix-vector steps.
 * State jobs whose plan has MG_FLAG_STATE_ACTION run together in one
 * action-path launch instead.  outputs[i], in[i], out[i] are as for mg_evolve
 * (MG_OUT_STATE or MG_OUT_PROPAGATOR; in[i] may be NULL for propagators; in may
 * be NULL when no job needs an input).  job_status (HOST, may be NULL) receives
 * MG_OK or the job's own error: a job whose Magnus exponent has a NaN/Inf norm
 * fails alone with MG_ENONFINITE (an action-path job also with MG_EUNSUPPORTED
 * when its spectral bound exceeds the sub-step limit), the others complete.
 * flags: MG_FLAG_HOST_PTRS when every in[i]/out[i] is host memory. */
int mg_evolve_batch(mg_ctx* ctx, int n, mg_plan* const* plans, const int* outputs, const double* const* in,
                    double* const* out, int reorth_every, int flags, int* job_status);

/* ---- autotuning ------------------------------------------------------------ */
/* One way of evolving a job and what it measured: the arithmetic of the matrix
 * products (precision, slices), the Taylor scheme (MG_TAYLOR_*), for state
 * outputs the action-based path (action = 1), the estimated max-abs error over
 * the job's N intervals and the device time per interval in microseconds. */
typedef struct mg_tune_entry {
  int32_t precision;
  int32_t slices;
  int32_t taylor;
  int32_t action;
  double error;
  double us_per_interval;
  double taylor_target;   /* mg_plan_set_taylor_target's u (0: the arithmetic's unit roundoff) */
} mg_tune_entry;

/* Host only: the index of the fastest entry whose error times `safety` (>= 1)
 * is at most `tolerance` (> 0).  MG_EUNSUPPORTED when none qualifies. */
int mg_tune_select(int n, const mg_tune_entry* entries, double tolerance, double safety, int* index);
/* Host only: append a tuning (key, all measured entries, the selected one) to
 * the cache file at `path` (created if absent; appends are serialised with a
 * file lock).  Keys contain no tab, newline or ';'. */
int mg_tune_cache_store(const char* path, const char* key, int n, const mg_tune_entry* entries, int selected);
/* Host only: the selected entry of the last tuning stored under `key` -- the key
 * itself, or a longer key that continues it after a '|' (so a caller that knows
 * only the leading fields of a key finds the latest tuning of that family).
 * MG_EAGAIN when the file or the key is absent. */
int mg_tune_cache_lookup(const char* path, const char* key, mg_tune_entry* entry);

/* Choose, by measurement on this GPU, how `plan` evolves `output`
 * (MG_OUT_STATE or MG_OUT_PROPAGATOR) within max-abs `tolerance`, and set it on
 * the plan (precision, slices, Taylor scheme, MG_FLAG_STATE_ACTION).  The
 * controls must be set.  The cache at `cache_path` (may be NULL: no cache) is
 * consulted first under the key
 *   gpu=<name>|d=<d>|K=<K>|out=<output>|tol=<tolerance>|nu=<e>|N=<n>
 * with nu = the binary exponent of the largest bound on ||Hbar_n - tau_n I||_1
 * and N the interval count rounded up to a power of two.  On a miss every
 * candidate -- FP64; split with 4..7 digits, each with and without the
 * degree-18 scheme; for 5..7 digits with the degree-18 scheme also coarser Taylor
 * truncation targets (mg_plan_set_taylor_target): 2^-34, 2^-28 and the smallest
 * targets that save one and two squarings at the largest norm bound (each only
 * where coarser than the digits' roundoff 2^-(beta L)); for states the action
 * path -- evolves the plan's first
 * n_probe <= 64 intervals (8 for d > 1024); the reference is the FP64 path (for
 * d > 1024 run once and not itself a candidate: seconds per interval); a candidate's
 * error is its deviation from the reference times N / n_probe (errors of
 * near-identical intervals add up), FP64's own u nu N; the fastest candidate
 * within tolerance / 4 is taken and the whole table is stored.  chosen (may be
 * NULL) receives it.  MG_EUNSUPPORTED when no candidate qualifies (the plan is
 * left unchanged). */
int mg_plan_autotune(mg_plan* plan, int output, double tolerance, const char* cache_path, mg_tune_entry* chosen);
/* Taylor scheme of a plan (MG_TAYLOR_AUTO, the default, or MG_TAYLOR_PS). */
int mg_plan_set_taylor(mg_plan* plan, int taylor);
/* Truncation target u of the plan's Taylor series (scaling and squaring of
 * App. A.5): the degree m and squaring count s are chosen so that the series'
 * tail, sum_{j>m} theta^j / j!, stays within u theta for ||2^-s X|| <= theta, so
 * each interval's exponential errs by about u ||Hbar_n||_1 (1-norm) from
 * truncation.  u = 0 (the default) takes the unit roundoff of the products'
 * arithmetic (2^-53 for FP64, 2^-(beta L) for split digits); a larger u (at most
 * 1e-3) trades accuracy for fewer squarings, errors that may add up over N
 * intervals to N u max ||Hbar_n||_1.  mg_evolve and mg_evolve_batch honour it
 * (batched plans with different targets form separate groups).  MG_EINVAL for u
 * outside [0, 1e-3]. */
int mg_plan_set_taylor_target(mg_plan* plan, double u);
/* Tuning cache of a context's servers (NULL: none); see MG_PREC_AUTO. */
int mg_ctx_set_tune_cache(mg_ctx* ctx, const char* path);

/* ---- a batch captured once, replayed many times ------------------------------ */
/* mg_evolve_batch issues every launch of a batch without reading anything back to
 * the host between them: the Taylor degree m and the number S of squaring
 * launches come from a bound on every interval's ||Hbar_n - tau_n I||_1 (the
 * operators' norms times the largest coefficients, formed when the batch is
 * planned), while each interval's own squaring count s_n (Sec. "Magnus
 * Expansion": U_n = exp(-i Hbar_n) by scaling and squaring) and the failure of a
 * job with a non-finite norm are decided on the device; each squaring launch
 * multiplies only the intervals whose s_n exceeds it.
 * mg_batch_graph_create plans such a batch and captures all of its launches
 * (every chunk of every group: Hbar_n, exponentials, tree products, state
 * chains, output copies) in one CUDA graph; mg_batch_graph_launch replays it
 * with one graph launch.  Arguments are those of mg_evolve_batch with device
 * pointers only; the input and output buffers and the plans' coefficient
 * buffers are bound into the graph, so a replay evolves whatever they hold at
 * launch time: call mg_set_controls with the same N, P and dt (new drive
 * samples) and/or rewrite in[i] between launches.  The plans, the buffers and
 * the context must outlive the graph.  The context's stream must not be the
 * legacy default stream (it cannot be captured); the graph has a workspace of
 * its own.  Action-flagged state jobs (MG_FLAG_STATE_ACTION) are
 * rejected with MG_EUNSUPPORTED.  Creation runs the batch once uncaptured (which
 * sizes the workspace), so it costs one evolution.
 * mg_batch_graph_launch synchronises the context's stream; job_status (HOST,
 * may be NULL) is filled as by mg_evolve_batch.  It returns MG_EINVAL when a
 * plan's N, dt or coefficient buffer changed since the capture, and
 * MG_EUNSUPPORTED when new controls made an interval's norm exceed the bound
 * the squaring launches were planned for (recreate the graph).
 * mg_batch_graph_stats gives the graph's kernel nodes and all nodes. */
typedef struct mg_batch_graph mg_batch_graph;
int mg_batch_graph_create(mg_ctx* ctx, int n, mg_plan* const* plans, const int* outputs, const double* const* in,
                          double* const* out, int reorth_every, mg_batch_graph** graph);
int mg_batch_graph_launch(mg_batch_graph* graph, int* job_status);
int mg_batch_graph_stats(mg_batch_graph* graph, int64_t* kernel_nodes, int64_t* nodes);
int mg_batch_graph_destroy(mg_batch_graph* graph);

/* ---- serving ---------------------------------------------------------------- */
/* A request loop over one context: mg_submit admits a job if its device memory
 * (padded operators, coefficients, state, upload staging) fits the budget next
 * to the jobs already resident, otherwise returns MG_EAGAIN; the job's inputs
 * are uploaded on a separate stream and stay resident until it completes.  A
 * worker thread repeatedly takes every admitted job that shares the key
 * (precision, padded dimension) of the job with the least remaining work
 * (d^3 x intervals left: shortest remaining work first) and advances each by up to
 * `quantum_intervals` intervals in one shared chunk step (batched exponential,
 * multi-job propagation), admitting new arrivals at every chunk boundary, so
 * requests that arrive while others run join them on the device instead of
 * waiting for them to finish (continuous batching).  State jobs flagged
 * MG_FLAG_STATE_ACTION take the action-based path instead: a second thread
 * launches them on four high-priority streams of their own, concurrently with
 * the chunk steps, in slices of about 10 ms of work per job, and completes
 * each job at the end of the slice that finishes it (so no long kernel holds
 * up work queued behind it on the device's shared hardware queues).  While a
 * server runs, the caller must not use its context for anything else. */
typedef struct mg_server mg_server;

typedef struct mg_job {
  int d, K;                 /* dimension, number of controls */
  const double* H0;         /* d x d complex */
  const double* Hk;         /* K x d x d complex */
  int N, P;                 /* intervals, quadrature points per interval */
  double t0, dt;
  const double* w;          /* P quadrature weights (HOST) */
  const double* samples;    /* N x P x K drive samples at the nodes of mg_quadrature_nodes */
  int output;               /* MG_OUT_STATE (in = psi0) or MG_OUT_PROPAGATOR (in must be NULL) */
  const double* in;
  double* out;              /* written when the job completes; keep it valid until mg_wait returns */
  int precision, slices;    /* MG_PREC_AUTO: the latest tuning of the context's cache under
                               gpu|d|K|out|tol (tolerance below); on a miss split with the
                               42-bit digit count of mg_split_digits (6, or 7 above d = 1024) */
  int flags;                /* MG_FLAG_HOST_PTRS: H0, Hk, samples, in and out are host memory;
                               MG_FLAG_STATE_ACTION: a state job of d >= 256 runs on the
                               action-based path (FP64; precision and slices are ignored) on one
                               of the server's action streams, concurrently with the chunk steps
                               of the other jobs; smaller flagged jobs, which finish sooner in the
                               shared chunk steps, stay there */
  double tolerance;         /* MG_PREC_AUTO only: the max-abs error the job was tuned for */
} mg_job;

typedef struct mg_job_report {
  int32_t status;           /* MG_OK or the job's error */
  double latency_ms;        /* submit -> result written */
  double queue_ms;          /* submit -> first chunk step */
  int64_t intervals;
} mg_job_report;

/* Start a server on `ctx`: mem_budget_bytes (> 0) bounds the device memory of
 * the admitted jobs together; quantum_intervals (>= 1) is how many intervals a
 * job advances per chunk step.  Starts the worker threads and the action
 * streams.  MG_EINVAL for bad arguments, MG_ENOMEM if its streams or tables
 * cannot be created. */
int mg_server_create(mg_ctx* ctx, size_t mem_budget_bytes, int quantum_intervals, mg_server** out);
/* Admit one job (see mg_job); *job_id names it for mg_wait.  MG_EAGAIN when it
 * does not fit the memory budget now (retry after jobs complete), MG_EINVAL for
 * bad arguments, MG_EUNSUPPORTED for an action-path job beyond that path's
 * limits, MG_ENOMEM if its upload allocation fails. */
int mg_submit(mg_server* srv, const mg_job* job, uint64_t* job_id);
/* Block until the job completes (timeout_s < 0: no limit).  Returns the job's
 * status, or MG_ETIMEOUT if it has not completed in time (the job keeps
 * running and can be waited for again).  A completed job is forgotten once
 * waited for: an unknown id, or a job whose result another (concurrent) mg_wait
 * took, gives MG_EINVAL. */
int mg_wait(mg_server* srv, uint64_t job_id, double timeout_s, mg_job_report* rep);
/* Latency percentiles of completed jobs and intervals completed per second of
 * wall time since the first submission. */
int mg_server_stats(mg_server* srv, double* p50_ms, double* p99_ms, double* intervals_per_s, int64_t* completed);
/* Stop the server: waits until every admitted job has completed (their outputs
 * are written), then frees the server's streams and memory.  Results that were
 * not waited for are discarded. */
int mg_server_destroy(mg_server* srv);

/* ---- steps of the path (device pointers) --------------------------------- */
/* c[n][k] = (dt/2) sum_p w[p] samples[n][p][k]   (Eq. magnus-first-order-coeff).
 * samples N x P x K, w P doubles (device), c N x K.  1 <= P <= 64. */
int mg_coefficients(mg_ctx* ctx, int N, int P, int K, double dt, const double* w,
                    const double* samples, double* c);

/* Hbar[n] = dt H0 + sum_k c[n][k] H_k   (Eq. magnus-first-order-term), N x d x d
 * complex output; also tau[n] = Re tr(Hbar_n)/d and norm1[n] =
 * ||Hbar_n - tau_n I||_1 (largest absolute column sum), both N doubles (device,
 * may be NULL).  1 <= d <= 4096, 0 <= K <= 64. */
int mg_build_omega(mg_ctx* ctx, int N, int d, int K, double dt, const double* H0,
                   const double* Hk, const double* c, double* Hbar, double* tau, double* norm1);

/* U[b] = exp(-i A[b]) for a batch of Hermitian d x d matrices A (trace shift,
 * scaling and squaring of a Taylor polynomial).  precision/slices as for plans.
 * The batch runs in chunks that fit the workspace; every chunk takes one degree
 * and squaring count, mg_taylor_choice of its largest FP64 1-norm of
 * A[b] - tau_b I (tau_b = Re tr(A[b])/d).  squarings (device int[batch], may be
 * NULL) receives the count applied to each matrix. */
int mg_expm(mg_ctx* ctx, int batch, int d, const double* A, double* U, int precision,
            int slices, int* squarings);

/* C[b] = A[b] B[b] for a batch of complex d x d matrices (the matrix product
 * every exponential and propagation step is built from). */
int mg_cgemm(mg_ctx* ctx, int batch, int d, const double* A, const double* B, double* C,
             int precision, int slices);

/* Carry a state or a propagator through given interval propagators U (N x d x d):
 * the propagation step of mg_evolve on its own.  Arguments as for mg_evolve. */
int mg_propagate(mg_ctx* ctx, int N, int d, const double* U, int output, const double* in,
                 double* out, int reorth_every, int precision, int slices);

/* ---- allocation-free product ---------------------------------------------- */
/* C[b] = A[b] B[b] for a batch of complex d x d matrices (device pointers, the
 * layout of mg_cgemm), computed exactly like mg_cgemm in MG_PREC_SPLIT mode with
 * `slices` digits, but without allocating any device memory and without a
 * context.  It is meant for callers that cannot call cudaMalloc: code whose
 * device memory is owned by another allocator or pool, which must not take the
 * implicit device-wide synchronisation of cudaMalloc/cudaFree, and fixed-latency
 * loops (pulse optimisation, control feedback) that must not allocate once
 * running.  The paper has no counterpart: it is an interface convenience.
 *
 * Scratch comes from one static device array of MG_STATIC_SCRATCH_BYTES that
 * every GPU which loads the library holds until the process exits.  A call
 * whose digit operands and product do not fit returns MG_EUNSUPPORTED (about
 * batch * d^2 * (16 + 12 slices) bytes plus tile padding are needed; one d = 729
 * product with 6 digits fits).  The first call on a device resolves the array's device address;
 * make that first call before any stream capture.  Every call reuses the same
 * array, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Work runs on `stream`
 * (a cudaStream_t, NULL for the legacy stream) of CUDA device `device`; the
 * call synchronises that stream before returning and restores the caller's
 * current device. */
#define MG_STATIC_SCRATCH_BYTES (64u << 20)
int mg_cgemm_split_static(int device, void* stream, int batch, int d, const double* A, const double* B,
                          double* C, int slices);

/* ---- diagnostics ----------------------------------------------------------- */
/* Per-launch timing of the matrix-product kernels (the dominant kernels of the
 * path).  While enabled, the context records a CUDA event pair around every
 * product launch on its stream; mg_ctx_gemm_stats synchronises the stream and
 * returns the number of launches, their summed device time (ms) and their
 * summed algorithmic work (8 d^3 real flops per complex d x d product, the
 * 4-real-multiplication form), then optionally resets the counters.  The
 * action kernel of MG_FLAG_STATE_ACTION counts as one launch with 8 flops per
 * stored operator nonzero per operator application. */
int mg_ctx_enable_gemm_timing(mg_ctx* ctx, int enable);
/* Failure detection of the tensor-core product (MG_PREC_SPLIT).  Every wait of
 * its kernel on an mbarrier is bounded: a CTA that gives up records
 * MG_ETIMEOUT for the call and winds down without touching its outputs.  Only
 * the waits whose abandonment is safe take `seconds` (0 <= seconds <= 4; the
 * default is 4): the MMA issuer's wait for loaded operands and the loader's
 * wait for a free stage.  The wait for the accumulators and the loader's final
 * wait for its own copies keep the 4 s limit, so no CTA frees on-chip memory
 * while a copy or tensor-core operation into it is in flight.  stall_test != 0
 * (tests only) makes the MMA issuer of every product first wait on a barrier
 * that nothing completes, so each product of the context ends in MG_ETIMEOUT
 * after about `seconds`; the context stays usable, and calling again with
 * stall_test = 0 restores normal products.  MG_EINVAL for seconds outside
 * [0, 4]. */
int mg_ctx_set_wait_limit(mg_ctx* ctx, double seconds, int stall_test);
/* K per pipeline stage of the tensor-core product (MG_PREC_SPLIT): 32 (the default;
 * 64-byte operand rows, two MMA K-steps per stage), 16 (32-byte rows, one K-step per
 * stage: half the shared memory per stage, so twice as many stages in flight) or 64
 * (128-byte rows, four K-steps; taken where slices <= 3 and d rounded up to 32 is a
 * multiple of 64, else 32).  The result does not depend on it.  Measured on GB300
 * (algorithmic TFLOP/s of 32 products of d = 700): 3 digits 141 / 187 / 198 and
 * 2 digits 195 / 254 / 292 for K = 16 / 32 / 64; at d = 729 with 6 digits K = 16
 * is 5% slower than 32.  With 8 slices a 32-deep stage leaves room for only one
 * stage, so the product takes 16 there whatever is set (35 -> 53 TFLOP/s at d = 512).
 * MG_EINVAL for other values. */
int mg_ctx_set_stage_k(mg_ctx* ctx, int stage_k);
/* Operand layout of the tensor-core product (MG_PREC_SPLIT) for an even number of
 * slices: on = 1 stores digits 2g and 2g + 1 of an element side by side (per 16 K
 * values of a row, 16 of the even digit, then 16 of the odd one), so each 64-byte row
 * of a pipeline stage 16 deep in K carries two digits; the stage then takes half the
 * shared memory of the default 32-deep stage and twice as many stages are in flight.
 * on = 2 keeps that memory layout but reads it in 32-deep stages, two 16-value blocks
 * per row: 128-byte rows (SWIZZLE_128B), the shared memory of the default stage, half
 * its rows (where two such stages fit, else as on = 1).  Either replaces
 * mg_ctx_set_stage_k's choice for even slices and combines with CTA pairs; odd slice
 * counts keep the digit-major layout.  The result is bit-identical either way.  on = 0
 * (the default): one plane per digit.  MG_EINVAL for other values.  A change applies to products
 * issued afterwards (a captured batch graph keeps the layout it was captured with).
 * Measured on GB300 (algorithmic TFLOP/s, 32 products, single CTAs): on = 1: d = 729,
 * 6 slices 76.5 paired vs 78.7 digit-major; d = 700, 4 slices 124 vs 142; d = 512,
 * 8 slices 53.0 vs 35.2 (52.7 with digit-major 16-deep stages, which 8 slices take by
 * default).  on = 2: d = 729 78.8 vs 77.0, d = 4096 100.1 vs 94.9; with CTA pairs
 * (the default from 5 slices) within 0.4% of the digit-major layout. */
int mg_ctx_set_digit_pairs(mg_ctx* ctx, int on);
/* Tensor-core product (MG_PREC_SPLIT) on CTA pairs: on = 1 runs each product tile of
 * 256 rows x 64 complex columns as one M = 256 tcgen05 product of two CTAs on two SMs
 * (a 2-CTA cluster; each CTA loads its 128 rows of A and half the B tile, which both
 * tensor cores read), where d > 128; the digit-major layout only (the paired layout of
 * mg_ctx_set_digit_pairs takes precedence).  on = 0: one CTA per 128-row tile.
 * on = -1 (the default): pairs for 5 or more slices where the 128-row tiles pair up
 * evenly from d = 256 on or number 7 or more (measured at 6 slices: d = 300, three
 * tiles, 45.6 vs 36.9 TFLOP/s on single CTAs; d = 144 and 200 within 5%).  The same digit products are
 * accumulated in the same order, so the result is bit-identical.  Measured on GB300
 * (algorithmic TFLOP/s, one CTA vs pairs, 32-deep stages): 6 slices 78.3 vs 80.4 at
 * d = 729 (32 products) and 96.8 vs 103.4 at d = 4096; 8 slices 52.9 vs 55.2 at d = 512;
 * 4 slices 142.0 vs 137.7 and 2 slices 255.2 vs 246.1 at d = 700.  The pairs relieve
 * each SM's shared-memory port, which every MMA reads its operands through (8 KiB
 * per MMA on one CTA, 6 KiB on a pair).  MG_EINVAL for other values. */
int mg_ctx_set_cta_pairs(mg_ctx* ctx, int on);
/* Structure of the tensor-core products (MG_PREC_SPLIT) of real operators.  When every
 * operator of a plan (H0 and the H_k, with the commutator operators of the second-order
 * term where mg_plan_set_magnus_order(2) adds them) has an exactly zero imaginary part --
 * the drive operators b + b^dag and the Hamiltonians of the Sec. "Magnus Expansion"
 * workloads in a real basis -- every first-order Hbar_n is real, so the exponent
 * X_n = -i 2^-s (Hbar_n - tau_n I) of Eq. magnus-first-order-term is purely imaginary,
 * its even powers real and its odd powers imaginary; when the operators are also exactly
 * symmetric (real Hermitian), every polynomial in X_n, and so every Taylor polynomial,
 * squaring and U_n, is complex symmetric (U = U^T).  mg_plan_create (and
 * mg_plan_set_magnus_order) check both on the device.  `on` is a bit mask:
 *   bit 0: the products X X, X^2 X and X^3 X^3 of the Taylor polynomial (and the power
 *          products of the Paterson-Stockmeyer forms) leave out the digit products of the
 *          zero parts: the zero half of the K axis of A is not loaded, and only the B
 *          plane that the remaining half meets is multiplied -- one real product into
 *          one output half (on CTA pairs as M = 256 x N = 128 MMAs over 128 output
 *          columns of that half; on single CTAs as N = 64 MMAs): a quarter of a general
 *          product's tensor-core work.  Only exact zeros are left out: the result is the
 *          same as without.
 *   bit 1: every product of the exponential (Taylor polynomial and squarings) computes
 *          only the output tiles on or below the diagonal (128-row tiles on single CTAs,
 *          256 on CTA pairs), and its symmetric matrices are kept as their 32 x 32 blocks
 *          on and below the diagonal, entry (i, j) with j > i read as (j, i); each U_n is
 *          written in full, exactly symmetric, the same on either tiling, and differs from
 *          the full products' by their own rounding asymmetry.  The tree product of the
 *          U_n is general.
 * 3 (the default) sets both, 0 issues every product in full.  Applies to mg_evolve,
 * mg_evolve_batch (a batch only when all of its plans qualify) and the chunk steps of a
 * server (mg_submit checks each job's operators; a step only when all of its jobs
 * qualify, so a result in a mix can differ from the same job alone by the rounding
 * asymmetry of bit 1, within the split tolerance); gemm statistics count
 * the algorithmic work of such a product: a quarter of 8 d^3 with two zero parts, and
 * the d (d + 1) / 2 entries on and below the diagonal of a symmetric result.  MG_EINVAL
 * outside 0..3. */
int mg_ctx_set_structure(mg_ctx* ctx, int on);
int mg_ctx_gemm_stats(mg_ctx* ctx, int64_t* launches, double* ms, double* flops, int reset);

const char* mg_strerror(int code);
const char* mg_last_error_message(void);
/* Number of kernels this process has launched through the library. */
int64_t mg_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MAGNUS_H_ */
