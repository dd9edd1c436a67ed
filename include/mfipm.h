/*
 * mfipm.h -- C ABI of the GB300 matrix-free primal-dual interior-point solver for
 *
 *     min_x  tau*||x||_1 + 1/2*||A x - b||_2^2                         (1)
 *
 * solved through the split x = u - v, z = [u; v] >= 0 and the quadratic program
 * min tau*1^T z + 1/2*||F^T z - b||^2, F^T = [A, -A]   (arXiv:1208.5435, Sec. 1,
 * Eqs. uvDef, lintechni, wrightBPDN).  Each Newton system of the primal-dual IPM
 * (Sec. 3, Eqs. sepregaugeq, fzfs, redNewtonA/B) is solved by preconditioned
 * conjugate gradients that touch A only through A*x and A^T*y, with the block
 * preconditioner P of Sec. 4, Eq. eq:ne2_P.  The outer loop is the single-corrector
 * IPM of Sec. 5.1 (Algorithm; sigma1=0.1, sigma2=0.5, sigma3=0.8, alpha_bar=0.5,
 * alpha_tilde=0.1).
 *
 * Conventions for every entry point:
 *   - Pointers named in a comment as DEVICE point to GPU memory owned by the caller;
 *     HOST pointers point to host memory owned by the caller.  The library never frees
 *     or retains a caller pointer after the call returns.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *     default stream).  Entry points that return per-problem information through a HOST
 *     pointer synchronise `stream` once before returning.
 *   - Return value: an mfipm_status code.  On any code other than MFIPM_OK or
 *     MFIPM_NOT_CONVERGED, mfipm_last_error() holds a one-line message (thread-local).
 *   - Arguments are validated before anything is launched; an invalid argument launches
 *     nothing and leaves outputs untouched.
 *   - All scratch memory comes from the caller's `workspace` (DEVICE, at least
 *     mfipm_workspace_size() bytes, 256-byte aligned); the library allocates no device
 *     memory in these calls.
 *   - Calls on the same stream are ordered; calls on different streams must not share a
 *     workspace.
 */
#ifndef MFIPM_H_
#define MFIPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MFIPM_OK = 0,
  MFIPM_INVALID_ARG = 1,    /* null pointer, m > n, bad DCT size or rows, tau <= 0, small workspace */
  MFIPM_NOT_CONVERGED = 2,  /* max_iter reached, or the gap test passed while the KKT residual
                               of x (info.kkt_rel) exceeds sqrt(tol); x and info are written */
  MFIPM_NUMERIC = 3,        /* NaN/Inf met in the data or during the iteration */
  MFIPM_CUDA = 4,           /* CUDA runtime error (message in mfipm_last_error) */
  MFIPM_TIMEOUT = 5,        /* a bounded device-side wait expired */
  MFIPM_UNSUPPORTED = 6     /* valid request this build does not implement */
} mfipm_status;

/* Operator kinds (Sec. 2):
 *   MFIPM_OP_DENSE        A is an explicit m x n matrix (e.g. the Gaussian ensemble).
 *   MFIPM_OP_PARTIAL_DCT  A = m distinct rows of the orthonormal n x n DCT-II matrix
 *                         C[j,k] = a_j cos(pi*j*(2k+1)/(2n)), a_0 = sqrt(1/n), a_j = sqrt(2/n),
 *                         so that A A^T = I_m (Eq. eq:orthonormality).  n is a power of
 *                         two with 64 <= n <= 1048576: up to 65536 one thread-block
 *                         cluster holds a problem's FFT in shared memory; from 131072 the
 *                         problems of one length run in lockstep with a three-pass FFT
 *                         through device memory (see mfipm_set_large_dct_threshold).  Or n
 *                         is any even length 8 <= n <= 16384 whose half n/2 has no prime
 *                         factor above 5 (n = 1000 of the phase-transition experiment,
 *                         Sec. 5.8): a mixed-radix FFT (radices 4, 2, 3, 5) in one CTA's
 *                         shared memory per problem.  A batch that holds such a length runs
 *                         every problem of it that way (so all its n <= 16384, cluster_size
 *                         0 or 1); mfipm_solve, mfipm_solve_batched and mfipm_solve_noalloc
 *                         take it with either PCG precision and either outer loop,
 *                         mfipm_backward with the float32 adjoint PCG; the operator products
 *                         (mfipm_apply_A, mfipm_apply_At, mfipm_kkt_residual) evaluate such
 *                         rows from the definition (direct sums, O(m n)).
 *   MFIPM_OP_PARTIAL_HAAR: A = the rows `rows` of the orthonormal n x n Haar matrix (Sec. 2
 *                         names Haar wavelets among the orthonormal systems with O(n)
 *                         products): row 0 = 1/sqrt(n); row 2^j + k (0 <= j < log2 n,
 *                         0 <= k < 2^j) = +-2^(j/2)/sqrt(n) on the two halves of
 *                         [k n/2^j, (k+1) n/2^j).  A A^T = I_m.  n a power of two with
 *                         64 <= n <= 65536 (one cluster); solve, solve_batched and backward,
 *                         with precision MFIPM_PREC_FP32_PCG or MFIPM_PREC_FP64 (float64 PCG)
 *                         and the double-float outer loop. */
typedef enum { MFIPM_OP_DENSE = 0, MFIPM_OP_PARTIAL_DCT = 1, MFIPM_OP_PARTIAL_HAAR = 2 } mfipm_op_kind;

/* Storage type of a dense A. */
typedef enum { MFIPM_A_F64 = 0, MFIPM_A_F32 = 1, MFIPM_A_BF16 = 2 } mfipm_a_dtype;

/* Arithmetic of the PCG solve.  The outer loop (IPM residuals, duality gap, step lengths and
 * iterate updates) is float64 for dense operators; for the partial-DCT and partial-Haar
 * operators its per-index arithmetic follows mfipm_outer below (double-float by default),
 * while its scalar reductions and every output stay float64.
 *   MFIPM_PREC_FP64      PCG vectors and operator products in float64 (dense A; partial DCT
 *                        below the multi-pass threshold, with the float64 outer loop; partial
 *                        Haar, with the double-float outer loop: the PCG tolerances of basis
 *                        pursuit, tol_pcg down to 1e-6, Sec. 5.4).
 *   MFIPM_PREC_FP32_PCG  PCG vectors and operator products in float32 (the inexact Newton
 *                        direction is corrected by the float64 residuals of the outer loop).
 *   MFIPM_PREC_BF16_A    dense A stored bf16 (times a_scale) on the tensor cores with float32
 *                        accumulation; float32 PCG. */
typedef enum { MFIPM_PREC_FP64 = 0, MFIPM_PREC_FP32_PCG = 1, MFIPM_PREC_BF16_A = 2 } mfipm_precision;

/* Arithmetic of the outer IPM loop of the partial-DCT solver: the iterate (z, s) and its
 * update, x = u - v, the residual A^T(Ax - b) (the FFT chain that corrects the inexact
 * float32 Newton directions) and the dual-residual terms tau +/- g.
 *   MFIPM_OUTER_DF    double-float: every value is the sum of two float32 words (about 48
 *                     significant bits; relative rounding ~1e-14), computed on the float32
 *                     pipes.  GB300 runs float64 at 1/64 of its float32 rate.
 *   MFIPM_OUTER_FP64  native float64.
 * Scalar reductions (gap, mu, step lengths) are float64 in both modes, and the outputs
 * (x, zs_out, info) are float64.  Dense operators always use MFIPM_OUTER_FP64. */
typedef enum { MFIPM_OUTER_DF = 0, MFIPM_OUTER_FP64 = 1 } mfipm_outer;

typedef struct {
  int32_t kind;          /* mfipm_op_kind */
  int32_t a_dtype;       /* mfipm_a_dtype (dense only) */
  int64_t m, n;          /* A is m x n, 0 <= m <= n */
  const void* A;         /* DEVICE, dense only: row-major, entry (i,j) = a_scale * A[i*lda + j] */
  double a_scale;        /* dense only; 1.0 for plain storage */
  int64_t lda;           /* dense only; >= n */
  const int64_t* rows;   /* DEVICE, partial DCT and Haar: m distinct row indices in [0, n), ascending */
} mfipm_operator;

typedef struct {
  double tol;            /* relative duality gap z^T s / (1 + |P(z)|) to stop at (Sec. 5.4 "tol"); 1e-10.
                            MFIPM_OK also needs kkt_rel <= sqrt(tol) at the stop */
  int32_t max_iter;      /* IPM iteration cap (Sec. 5.4 "maxiters"); 100 */
  double tol_pcg;        /* PCG tolerance (Sec. 5.4 "tolpcg") on the preconditioned residual norm
                            sqrt(r^T P^-1 r) relative to its initial value; 1e-2 */
  int32_t max_iter_pcg;  /* PCG iteration cap (Sec. 5.4 "mxiterpcg"); 200 */
  double sigma1, sigma2, sigma3;  /* centering parameters (Sec. 5.1); 0.1, 0.5, 0.8 */
  double alpha_bar, alpha_tilde;  /* step-size thresholds (Sec. 5.1); 0.5, 0.1 */
  double eta;            /* fraction of the step to the boundary; 0.995 */
  int32_t precision;     /* mfipm_precision; default MFIPM_PREC_FP32_PCG (the Python binding passes
                            MFIPM_PREC_FP64 for a dense float64 A unless told otherwise) */
  int32_t equal_steps;   /* 0: separate primal and dual steps as in Sec. 5.1; 1: common step */
  int32_t cluster_size;  /* CTAs that cooperate on one problem (1,2,4,8,16); 0 = automatic */
  int32_t outer;         /* mfipm_outer; MFIPM_OUTER_DF */
  double outer_f32_gap;  /* partial DCT and shared bf16 A: while the relative duality gap exceeds
                            this value the outer residual A^T(Ax - b) runs through a float32-grade
                            chain (the float32 FFT chain; for bf16 A two tensor-core GEMMs with x
                            and r as three bf16 pieces, in place of the exact digit slices); at
                            the first iterate at or below it, and before any stop, it is
                            recomputed in the outer loop's precision, which every later
                            iteration keeps (in the lockstep solvers, multi-pass partial DCT and
                            bf16 A, once any problem of the group gets there).  Applied only when
                            tau >= 1e-3 ||A^T b||_inf (for every problem of a lockstep group; the
                            float32-grade chains err by ~1e-6 ||A^T b||_inf); smaller tau (basis
                            pursuit, the phase-transition workload) always use the outer
                            precision.  0 = always the outer precision.  1e-8 */
  int32_t centrality_correctors;  /* 0 (default): the single conditional corrector of the
                            Algorithm (Sec. 5.1).  K in 1..16: the multiple-centrality-corrector
                            variant that Sec. 5.1 names as the method's origin: after each
                            predictor, up to K correctors, each one more PCG solve with
                            right-hand side (0, t) of Eq. sepregaugeq, t moving the trial
                            point's products z_i s_i (at the steps alpha + 0.1) into
                            [0.1, 10] * sigma * mu; a corrector is kept while the smaller step
                            grows by at least 0.01.  Persistent-kernel paths only (partial DCT
                            and Haar below the multi-pass threshold, dense float64 A);
                            MFIPM_UNSUPPORTED elsewhere.  info.correctors counts the kept ones. */
} mfipm_params;

typedef struct {
  int32_t status;        /* mfipm_status of this problem */
  int32_t ipm_iters;     /* outer iterations taken */
  int32_t correctors;    /* corrector directions computed */
  int32_t pcg_iters;     /* total PCG iterations */
  int64_t n_mat;         /* products with A and A^T (the paper's nMat, Table tablesymbabb) */
  double rel_gap;        /* z^T s / (1 + |P(z)|) at exit */
  double dual_res;       /* ||s - c - F F^T z||_2 / (1 + ||c||_2) at exit */
  double kkt_rel;        /* ||x - S_tau(x - A^T(Ax-b))||_2 / (1 + ||x||_2) at exit, float64 */
  double primal_obj;     /* tau*||x||_1 + 1/2||Ax-b||^2 evaluated at z (tau*1^T z + ...) */
} mfipm_info;

/* Fill *p with the defaults listed above.  Returns MFIPM_OK, or MFIPM_INVALID_ARG if p is NULL. */
int mfipm_params_default(mfipm_params* p);

/* Bytes of DEVICE workspace needed to solve `batch` problems whose operators are ops[0..batch)
 * (HOST array) with parameters *p (HOST).  Writes *bytes (HOST).  Errors: MFIPM_INVALID_ARG for a
 * malformed operator, MFIPM_UNSUPPORTED for an operator/precision pair this build lacks. */
int mfipm_workspace_size(const mfipm_operator* ops, int32_t batch, const mfipm_params* p, size_t* bytes);

/* Solve one problem (1).
 *   op       HOST struct describing A (its A / rows pointers are DEVICE).
 *   b        DEVICE, m float64.       tau  > 0.
 *   x        DEVICE, n float64, output: the minimiser x = u - v.
 *   zs_out   DEVICE, 4n float64 or NULL: final [u; v; s_u; s_v] (input of mfipm_backward).
 *   info     HOST, output.
 * Returns the problem's status (MFIPM_NOT_CONVERGED still writes x). */
int mfipm_solve(const mfipm_operator* op, const double* b, double tau, const mfipm_params* p,
                double* x, double* zs_out, void* workspace, size_t ws_bytes, mfipm_info* info,
                void* stream);

/* mfipm_solve without a caller workspace, for callers that cannot allocate device memory:
 * code that runs where cudaMalloc is forbidden or unavailable (a plugin whose host framework
 * owns every device allocation, a process started under a fixed memory budget, a real-time
 * loop that must not enter the allocator).  The paper has no counterpart; this is a
 * deployment convenience.
 * Scratch comes from one 8 MiB array in device memory that every GPU loading this library
 * holds until the process exits; the library allocates nothing.  The call takes the same
 * path as mfipm_solve would for the same arguments (the persistent kernel, the multi-pass
 * partial DCT when its threshold has been lowered, the shared-A bf16 solver for a dense bf16
 * A with MFIPM_PREC_BF16_A) and needs the scratch that mfipm_workspace_size reports for it:
 * problems above 8 MiB (partial DCT up to n = 16384 fits, small dense and bf16 problems fit)
 * are rejected with MFIPM_INVALID_ARG before any launch.  All calls share the array and it
 * keeps the last call's contents: each call re-initialises everything it reads, and calls
 * that may overlap on the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  Arguments and results as for mfipm_solve. */
int mfipm_solve_noalloc(const mfipm_operator* op, const double* b, double tau, const mfipm_params* p,
                        double* x, double* zs_out, mfipm_info* info, void* stream);

/* Solve `batch` independent problems in one persistent launch (one CTA cluster per problem,
 * problems taken from a device work queue, largest first).  Partial-DCT problems at or above
 * the multi-pass threshold are solved after it, each group of equal n as one lockstep batch
 * (every problem keeps its own IPM scalars; the operator passes cover the whole group).  ops, b, tau, x, zs_out, infos are
 * HOST arrays of length batch; b[j], x[j], zs_out[j] are DEVICE pointers (zs_out may be NULL or
 * hold NULLs).  Returns MFIPM_OK if every problem converged, else the first non-OK problem
 * status. */
int mfipm_solve_batched(int32_t batch, const mfipm_operator* ops, const double* const* b,
                        const double* tau, const mfipm_params* p, double* const* x,
                        double* const* zs_out, void* workspace, size_t ws_bytes,
                        mfipm_info* infos, void* stream);

/* Reverse-mode derivative of the solution map (b, tau, A) -> x* of (1) at a solution returned by
 * mfipm_solve[_batched] (the paper has no derivative).  Differentiating the perturbed KKT
 * conditions Q z + c - s = 0, Z S e = mu e of Sec. 3, Eq. fzfs at the final iterate, with mu
 * fixed, gives (Theta^-1 + F F^T) dz = -dc - dQ z.  Hence, for dL/dx* = grad_x and
 * J = [I; -I]: y = H^-1 J grad_x is solved by the same PCG and preconditioner as a Newton
 * system (tolerance min(tol_pcg, 1e-6)), w = y_u - y_v, and
 *   grad_b = A w,   grad_tau = -sum(y),   grad_A = r w^T - (A w) x^T with r = b - A x.
 * These are the derivatives of x* wherever its support is locally constant (strict
 * complementarity).
 *   x         DEVICE n: the forward solution.     zs  DEVICE 4n: the zs_out of the forward solve.
 *   grad_x    DEVICE n.   grad_b DEVICE m or NULL.   grad_tau HOST (batch) or NULL.
 *   grad_A    DEVICE m x n row-major or NULL (dense operators only; MFIPM_UNSUPPORTED otherwise).
 * Arrays are HOST arrays of DEVICE pointers, as in mfipm_solve_batched; infos[i].pcg_iters and
 * n_mat count the work of each derivative.  Dense, partial-DCT and partial-Haar operators
 * (A w of the Haar operator by its float64 analysis pyramid). */
int mfipm_backward(int32_t batch, const mfipm_operator* ops, const double* const* b,
                   const double* tau, const double* const* x, const double* const* zs,
                   const double* const* grad_x, double* const* grad_b, double* grad_tau,
                   double* const* grad_A, const mfipm_params* p, void* workspace,
                   size_t ws_bytes, mfipm_info* infos, void* stream);

/* Matrix-free products with the operator (the only way the solver touches A, Sec. 1):
 *   mfipm_apply_A:   y (DEVICE, m) = A x (x DEVICE, n)
 *   mfipm_apply_At:  x (DEVICE, n) = A^T y (y DEVICE, m)
 * float64 in and out (input and output must not overlap).  Partial DCT with n >= 1024: the
 * multi-pass FFT chain in double-float (about 2^-44 relative, Sec. 2's A = rows of the
 * orthonormal DCT-II); n < 1024, partial Haar and dense A: direct float64 sums (a Haar row
 * touches its support only; a column sums its log2(n) + 1 rows).  `workspace`: DEVICE,
 * 256-byte aligned, at least the bytes mfipm_workspace_size reports for this operator with
 * batch 1 (a bf16 A: with precision MFIPM_PREC_BF16_A); the caller owns it.  Synchronises
 * `stream`.  MFIPM_INVALID_ARG for NULL vectors, a small workspace or bad rows. */
int mfipm_apply_A(const mfipm_operator* op, const double* x, double* y, void* workspace,
                  size_t ws_bytes, void* stream);
int mfipm_apply_At(const mfipm_operator* op, const double* y, double* x, void* workspace,
                   size_t ws_bytes, void* stream);

/* kkt_rel(x) = ||x - S_tau(x - A^T(Ax - b))||_2 / (1 + ||x||_2) (the l1 optimality residual:
 * zero exactly at the minimiser of Eq. formulationsnoisy1's 1/2 form) for a candidate x
 * (DEVICE, n) and b (DEVICE, m); result in *out (HOST).  Residual by the same arithmetic as
 * mfipm_apply_A/At; workspace as there.  Synchronises `stream`. */
int mfipm_kkt_residual(const mfipm_operator* op, const double* b, double tau, const double* x,
                       void* workspace, size_t ws_bytes, double* out, void* stream);

/* Instrumentation (this thread only): with timing enabled, each solve records CUDA events on
 * its stream around the persistent solver kernel; mfipm_last_kernel_ms() returns that kernel's
 * device time of the last solve in milliseconds (-1 if none).  Not in the paper. */
int mfipm_set_timing(int32_t enable);
double mfipm_last_kernel_ms(void);
/* With timing enabled, the multi-pass partial-DCT solver (n at or above the threshold of
 * mfipm_set_large_dct_threshold) records CUDA events around each operator product
 * y = A^T A w of its PCG (the three FFT passes, Sec. 4's only use of A).  For the last such
 * solve or backward on this thread: *ms = their summed device time (-1 if none),
 * *bytes = their algorithmic bytes (w read and y written: 8 bytes per index of every problem
 * the product covers), *products = how many products.  *launches = how many kernels the last
 * mfipm_solve, mfipm_solve_batched or mfipm_backward call on this thread launched, on any
 * solver path (with timing on or off).  Not in the paper. */
int mfipm_last_operator_stats(double* ms, double* bytes, int64_t* products, int64_t* launches);

/* Measured float32 FMA throughput of the current device, in TFLOP/s (*tflops, HOST): the
 * best of three timed launches of a plain fused-multiply-add loop on every SM (8 independent
 * chains per thread, 32 warps per SM), timed with CUDA events on `stream` after one warm-up
 * launch.  The denominator of the float32 ALU roofline of the shared-memory FFT chain (the
 * partial-DCT operator), which runs near the float32 ridge.  Synchronises `stream`.  Not in
 * the paper. */
int mfipm_fp32_fma_peak(double* tflops, void* stream);

/* The bf16 GEMM of the shared-A solver (MFIPM_PREC_BF16_A), exposed for testing and reuse (not
 * in the paper):  C_s[c][r] = sum_{k in slice s} Aop[r][k] * Bop[c][k]  for s < splits, with
 * Aop (rows x K) and Bop (N x K) bf16 row-major DEVICE arrays and C a DEVICE array of
 * splits x N x rows float32 (the sum of the slices is the product; split-K).  tensor_cores = 1
 * or 4 runs the tcgen05/TMA kernel with a four-stage shared-memory ring, 3 with three stages
 * (N <= 256, K % 8 == 0, 16-byte aligned operands), 0 a plain CUDA-core kernel (splits = 1).  Synchronises `stream`; MFIPM_TIMEOUT if a bounded device
 * wait expired. */
int mfipm_gemm_bf16(const void* Aop, const void* Bop, float* C, int32_t rows, int32_t N, int32_t K, int32_t splits,
                    int32_t tensor_cores, void* stream);
/* Use (1, default) or bypass (0) the tensor-core GEMM inside the bf16 solver on this process. */
int mfipm_set_gemm_mode(int32_t tensor_cores);
/* Outer residual A^T(A x - b) of the bf16 solver on this process (not in the paper; both are
 * float64-grade, below 1e-10 of ||a|| ||x|| per entry): 1 (default) = exact integer digit
 * slices of A and x on the tcgen05 GEMM (error-free splitting: float32 accumulation of integer
 * products over chunks of 1024 is exact), 0 = a biased float32 accumulator on the CUDA cores. */
int mfipm_set_residual_mode(int32_t tensor_cores);
/* Partial-DCT problems with n >= threshold (a power of two, default 131072 = twice the
 * cluster solver's largest n; accepted range [1024, 131072]) are solved by the lockstep
 * multi-pass solver, whose operator is the same chain of Sec. 2 (Eq. eq:orthonormality) as
 * a three-pass four-step FFT over global memory; smaller ones by the cluster-resident
 * persistent kernel.  Not in the paper: a process-wide switch, mainly so that tests can run
 * the multi-pass path at sizes the oracle reaches.  MFIPM_INVALID_ARG below 1024. */
int mfipm_set_large_dct_threshold(int64_t n);

/* Autotuner (not in the paper): times candidate decompositions on the caller's actual batch
 * and keeps the fastest, process-wide, for later calls with cluster_size = 0:
 *   path 1, partial DCT on the persistent kernel: the cluster size G (the radix of the FFT's
 *     distributed exchange step; every G that fits the batch's n) and the largest n a single
 *     CTA solves alone (2048 .. 16384), keyed by the batch's largest n and ceil(log2 batch);
 *     each candidate is timed by the solver kernel's CUDA events over the real solve;
 *   path 2, shared bf16 A (MFIPM_PREC_BF16_A): the split-K count (1 .. 8) and the number of
 *     shared-memory ring stages (4, or 3 to fit two CTAs per SM) of each of the two tcgen05
 *     GEMMs of the PCG product, timed alone on their real shapes, keyed by (m, n, batch).
 * Other batches are solved without tuning (path 0).  Arguments as for mfipm_solve_batched;
 * x and infos receive a solve with the chosen configuration.  *tuning (HOST, nullable):
 * the choice, the number of timed candidates, and the device times (ms) of the best and of
 * the default configuration. */
typedef struct {
  int32_t path;
  int32_t candidates;
  int32_t cluster_size;     /* path 1 */
  int32_t splits1, splits2; /* path 2 */
  int64_t cta_max_n;        /* path 1 */
  double best_ms, default_ms;
  int32_t stages1, stages2; /* path 2: tcgen05 ring stages (3 or 4) of the two GEMMs */
} mfipm_tuning;
int mfipm_autotune(int32_t batch, const mfipm_operator* ops, const double* const* b,
                   const double* tau, const mfipm_params* p, double* const* x, void* workspace,
                   size_t ws_bytes, mfipm_info* infos, mfipm_tuning* tuning, void* stream);
/* Forget every tuned configuration of this process. */
int mfipm_clear_tuning(void);

/* Message of the last failing call on this thread ("" if none). */
const char* mfipm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MFIPM_H_ */
