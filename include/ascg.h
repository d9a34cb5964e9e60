/*
 * ascg.h - C ABI of libascg, an FP64 adaptive s-step conjugate gradient solver
 * for one NVIDIA GB300 (sm_103a).
 *
 * Method: E. Carson, "The Adaptive s-step Conjugate Gradient Method",
 * arXiv:1701.03989. Names below follow the paper's notation:
 *   Alg. 1 classical CG; Alg. 2 s-step CG; Alg. 4 adaptive s-step CG;
 *   eq. (polybasiscg) basis recurrence; eq. (cg-krylovbasis) bases P, R;
 *   eq. (AVVB) A*Yunder = Y*B; eq. (coords) recovery; eq. (condy) choice of
 *   s~_k; eq. (check) in-loop break test.
 *
 * Conventions for every call:
 *  - Every call returns an ascg_status and never aborts. On an error,
 *    ascg_last_error() returns a message (per thread, valid until the next
 *    call on that thread).
 *  - "device" pointers are CUDA device memory of the current device. "host"
 *    pointers are ordinary (pageable or pinned) host memory.
 *  - Calls are ordered on the given CUDA stream (NULL = the legacy default
 *    stream). Calls that report results on the host or free temporaries
 *    (ascg_solve*, ascg_block_step, ascg_newton_shifts, ascg_matrix_powers,
 *    ascg_gram) synchronise that stream before they return. The others return
 *    as soon as their work is enqueued.
 *  - Sizes are int64_t. Matrices have n >= 1 rows and nnz < 2^31 nonzeros.
 *  - All arithmetic is IEEE double. eps = 2^-53.
 *  - An ascg_op is not safe for concurrent use from several threads or
 *    streams: it owns one workspace.
 */
#ifndef ASCG_H
#define ASCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque operator handle: owns device copies of a CSR matrix and a workspace. */
typedef struct ascg_op_s* ascg_op;

#define ASCG_MAX_S 16                     /* largest s (s_max) supported   */
#define ASCG_MAX_W (2 * ASCG_MAX_S + 1)   /* basis columns at s = s_max    */

typedef enum {
  ASCG_OK = 0,
  ASCG_ERR_INVALID = 1,      /* bad argument or malformed CSR                    */
  ASCG_ERR_OOM = 2,          /* device allocation failed                         */
  ASCG_ERR_CUDA = 3,         /* a CUDA runtime call failed                       */
  ASCG_ERR_BREAKDOWN = 4,    /* a block could not take a single inner step       */
  ASCG_NOT_CONVERGED = 5,    /* max_iters reached before the target              */
  ASCG_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up: a wait of the
                                tensor-core Gram (about 2 s) ran out, its CTA
                                gave up cleanly and the GPU context stays usable */
  ASCG_ERR_NOT_SPD = 7       /* a diagonal entry is missing or not positive      */
} ascg_status;

typedef enum {
  ASCG_CLASSICAL = 0,        /* Alg. 1                                            */
  ASCG_FIXED_S = 1,          /* Alg. 2 with s = s_max                             */
  ASCG_ADAPTIVE = 2,         /* Alg. 4                                            */
  ASCG_VARIABLE_S = 3        /* Alg. 3: block k takes s_k = s_seq[min(k, len-1)]  */
} ascg_method;

typedef enum {
  ASCG_MONOMIAL = 0,         /* theta = sigma = 0, gamma = 1 (Sec. 2)             */
  ASCG_NEWTON = 1,           /* Leja-ordered Ritz values as shifts                */
  ASCG_CHEBYSHEV = 2         /* T_j((z - c)/h) on [lambda_min, lambda_max]        */
} ascg_basis;

/* Why a block's inner loop ended (Alg. 4). */
typedef enum {
  ASCG_STOP_DONE = 0,        /* ran all s~_k steps                                 */
  ASCG_STOP_CONVERGED = 1,   /* sqrt(r'^T G r') <= eps* after step s_k             */
  ASCG_STOP_BREAK = 2,       /* eq. (check) failed after step s_k                  */
  ASCG_STOP_BREAKDOWN = 3,   /* a denominator was not positive and finite          */
  ASCG_STOP_MAXITER = 4      /* the iteration cap ended the block                  */
} ascg_stop;

/* One record per outer loop (block) k. */
typedef struct {
  int sbar;                  /* basis size built, sbar_k                          */
  int stilde;                /* size accepted by eq. (condy), s~_k                */
  int s_k;                   /* inner steps taken                                 */
  int stop;                  /* ascg_stop                                         */
  int m;                     /* iterations done before this block                 */
  int pad_;
  double rnorm;              /* ||r_{m+1}|| = sqrt(G[r0, r0])                     */
  double threshold;          /* eps* / (c eps ||r_{m+1}||), eq. (condy)           */
  double gamma;              /* sqrt(kappa(G_{k,s~})) (+inf when uncertified)     */
  double sqrt_kappa[ASCG_MAX_S]; /* sqrt(kappa(G_{k,i})), i = 1..sbar; +inf when
                                    lambda_min <= (2i+1) sqrt(n) eps lambda_max;
                                    0 where not computed                          */
} ascg_block_info;

typedef struct {
  int method;                /* ascg_method                                       */
  int basis;                 /* ascg_basis                                        */
  int s_max;                 /* Alg. 4: s_max; Alg. 2: s; Alg. 3: >= every s_k.
                                1 <= s_max <= 16                                  */
  int s0;                    /* sbar_0 (Alg. 4 "initial s value")                 */
  int f;                     /* basis growth cap: sbar_k = min(s_{k-1}+f, s_max)  */
  int newton_warmup;         /* classical steps whose Ritz values give the shifts */
  int max_iters;             /* cap on total iterations                           */
  int check_in_loop;         /* 1: eq. (check) break test on, 0: off (Sec. 3.2)   */
  int flags;                 /* ASCG_FLAG_* bits                                  */
  int pad_;
  double eps_target;         /* relative target: eps* = eps_target * ||b||        */
  double c;                  /* c_{k,j}, a constant (Alg. 4 "function c_{k,j}")   */
  double lambda_min, lambda_max; /* Chebyshev interval (required for CHEBYSHEV)   */
  /* optional host output buffers (may be NULL) */
  double* res_hist; int res_hist_cap;   /* ||r_i||/||b||, i = 0 .. iters          */
  int pad2_;
  ascg_block_info* block_hist; int block_hist_cap;  /* per block                   */
  int pad3_;
  double* alpha_hist; double* beta_hist; int coef_hist_cap; /* alpha_i, beta_i     */
  int pad4_;
  /* ASCG_VARIABLE_S: host int[s_seq_len], each in 1..s_max; the last value
     repeats (for example a Fibonacci sequence min(s_max, s_{k-1} + s_{k-2})).
     Unused (may be NULL) for the other methods. */
  const int* s_seq; int s_seq_len;
  int pad5_;
  /* ASCG_FLAG_C_FORMULA (ASCG_ADAPTIVE, ascg_solve only): estimates of
     kappa(A) (>= 1) and ||A||_2 (> 0) for c_{k,j} = 6 N_k j kappa(A) */
  double kappa_A, norm_A;
  /* batched solves and the server: rows from which a system's Gram runs in
     the tensor-core launch (w >= 9) instead of the FP64 one; 0: 1024;
     < 0: never. ascg_tune_gram_schedule measures a value for this GPU. The
     two kernels round differently: keep it fixed for reproducible results. */
  int64_t tc_lane_rows;
} ascg_options;

#define ASCG_FLAG_TIMING 1   /* time the Gram kernel and phases with CUDA events  */
#define ASCG_FLAG_GRAM_FP64 2 /* Gram by FP64 FMAs on the CUDA cores for every w,
                                 instead of the tensor-core kernel. By default
                                 ascg_solve runs the Gram on the tensor cores
                                 when w >= 9 and n w(w+1)/2 >= 2^25 (below
                                 that the FP64 kernel costs less than the
                                 tensor-core kernel's fixed cost)               */
#define ASCG_FLAG_GRAM_TC 32  /* ascg_solve: the tensor-core Gram for every
                                 block with w >= 9, whatever n (excludes
                                 ASCG_FLAG_GRAM_FP64 and ASCG_FLAG_MOMENT_GRAM) */
#define ASCG_FLAG_RECOVER_FP64 64 /* ascg_solve: the recovery (eq. coords) by
                                 FP64 FMAs for every block. By default a block
                                 whose Gram took the tensor cores also recovers
                                 x, r and p on them, in one pass over Y (see
                                 ascg_recover_tc for its error bound)          */
#define ASCG_FLAG_MOMENT_GRAM 8 /* monomial basis only: G from 6 sbar moments
                                 (ascg_gram_moments) instead of Y^T Y; a
                                 variant that rounds differently            */
#define ASCG_FLAG_TEST_GRAM_STALL 16 /* failure-path test only (ascg_solve with
                                 an s-step method): in the first block, the
                                 tensor-core Gram's first CTA never issues its
                                 first tensor copy and every wait is limited
                                 to a few milliseconds, so a wait runs out by
                                 construction. The CTA gives up cleanly (its
                                 copies and MMAs land, its tensor memory is
                                 freed) and the solve returns ASCG_ERR_TIMEOUT
                                 with x = x_1. No effect when the block's Gram
                                 takes the FP64 kernel (see ASCG_FLAG_GRAM_TC). */
#define ASCG_FLAG_C_FORMULA 4 /* c_{k,j} = 6 N_k j kappa(A), the factor of the gap
                                 bound eq. (fb), instead of the constant c:
                                 N_k = 7 + 2 N_A + 14 ||B_k|| / ||A||, N_A = most
                                 nonzeros in a row of A, B_k of the block's basis
                                 (size sbar_k), eq. (condy) with c_{k,s_max} and
                                 eq. (check) after step j with c_{k,j}. Needs
                                 kappa_A and norm_A; ASCG_ADAPTIVE only.         */

typedef struct {
  int status;                /* ascg_status of the solve                          */
  int iters;                 /* total CG iterations (warm-up included)            */
  int blocks;                /* outer loops = global reductions of G              */
  int grid_reductions;       /* device-wide reductions issued                     */
  int wasted_vecs;           /* sum over blocks of 2 (sbar_k - s_k) basis vectors */
  int launches;              /* kernels launched by this call                     */
  double bnorm;              /* ||b||                                             */
  double rel_res_updated;    /* last updated residual norm / ||b||                */
  double rel_res_true;       /* ||b - A x|| / ||b|| of the returned x             */
  /* device times (ms) when ASCG_FLAG_TIMING is set, else 0 */
  double t_total_ms, t_mpk_ms, t_gram_ms, t_ctrl_ms, t_recover_ms, t_cg_ms;
  int gram_launches;         /* Gram kernel launches timed in t_gram_ms            */
  int mpk_launches;          /* matrix powers step launches timed in t_mpk_ms     */
  double gram_flops;         /* algorithmic FP64 flops of those launches          */
  double gram_bytes;         /* algorithmic bytes read by those launches           */
  double mpk_flops, mpk_bytes, recover_flops, recover_bytes;
} ascg_result;

/* Fills *o with the defaults: ADAPTIVE, MONOMIAL, s_max = 8, s0 = f = s_max,
 * eps_target = 1e-10, c = 1, check_in_loop = 1, max_iters = 100000,
 * newton_warmup = 0 (meaning 2 s_max), no history buffers. */
ascg_status ascg_options_default(ascg_options* o);

/* --- operator ------------------------------------------------------------ */

/* Creates an operator from a square CSR matrix (the matrix A of Alg. 1-4).
 * rowptr: int64[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = nnz;
 * colind: int32[nnz] in [0, n); val: double[nnz]. Every row must hold a
 * positive diagonal entry (else ASCG_ERR_NOT_SPD). A must be symmetric; that
 * is not checked. on_device = 0: the three arrays are host memory;
 * 1: device memory. The library copies them; the caller keeps ownership.
 * On error *out is NULL. */
ascg_status ascg_op_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr,
                               const int32_t* colind, const double* val,
                               int on_device, ascg_op* out);

/* Frees the operator and its workspace. NULL is accepted. */
ascg_status ascg_op_destroy(ascg_op op);

/* n and nnz of the operator (host out-pointers may be NULL). */
ascg_status ascg_op_size(ascg_op op, int64_t* n, int64_t* nnz);

/* --- solve (Alg. 1, 2, 4) --------------------------------------------------- */

/* Solves A x = b. b: device double[n]; x: device double[n], holds x_1 on entry
 * and the solution on return. opts: host; NULL means the defaults. result:
 * host, always written (result->status == the return value). Returns after
 * the result is on the host. Returns ASCG_NOT_CONVERGED (with x = the last
 * iterate) if max_iters is reached. */
ascg_status ascg_solve(ascg_op op, const double* b, double* x, const ascg_options* opts,
                       ascg_result* result, void* cuda_stream);

/* As ascg_solve, with b and x in host memory. The library copies b and x_1 to
 * the device and the solution back, on the same stream. */
ascg_status ascg_solve_host(ascg_op op, const double* b, double* x, const ascg_options* opts,
                            ascg_result* result, void* cuda_stream);

/* --- steps of one block, exposed for testing (Alg. 4) --------------------------
 * Basis layout used by every step: Y is column-major, leading dimension
 * ldY >= n (device). The columns interleave the two bases of
 * eq. (cg-krylovbasis):
 *   column 2j   = rho_j(A) p,  j = 0..s     (P_{k,s})
 *   column 2j+1 = rho_j(A) r,  j = 0..s-1   (R_{k,s})
 * so w = 2s+1 columns. The i-step basis Y_{k,i} of Sec. 3.2 is then the
 * leading 2i+1 columns, and every Gram submatrix G_{k,i} is a leading
 * principal submatrix. */

/* Batched solves: `count` independent SPD systems A_q x_q = b_q of any sizes
 * in one call (Alg. 4 per system, run in lockstep). Each system keeps its own
 * operator, basis, x and b; a device table of per-system descriptors and a
 * list of row items (up to 256 rows of one system each) let every phase of a
 * block be one launch for all systems. A system that has converged drops out
 * of the following blocks. Each system's arithmetic depends on that system
 * alone: its result is bitwise the same alone and in any batch.
 *  - ops: host array of count operators (any sizes) on the current device.
 *  - b, x: host arrays of count device pointers (n_q doubles each); x[q] holds
 *    x_1 on entry and the solution on exit (updated in place; x[q] = 0 when
 *    b[q] = 0). b[q] and x[q] must not overlap each other or another system's.
 *  - eps_target: host double[count] of relative targets (eps*_q =
 *    eps_target[q] ||b_q||), or NULL for opts->eps_target.
 *  - opts: method ASCG_ADAPTIVE, ASCG_FIXED_S or ASCG_VARIABLE_S, basis
 *    ASCG_MONOMIAL (the other bases need per-system parameters and are not
 *    batched); s_max, s0, f, s_seq, c, check_in_loop, max_iters,
 *    tc_lane_rows and ASCG_FLAG_MOMENT_GRAM apply to every system
 *    (ASCG_FLAG_C_FORMULA is refused). Histories are per system: res_hist is
 *    count x res_hist_cap, block_hist count x block_hist_cap, alpha_hist and
 *    beta_hist count x coef_hist_cap (row q is system q); the caps must be
 *    >= 1 when the arrays are given.
 *  - results: host ascg_result[count] or NULL: per system status, iters,
 *    blocks, wasted_vecs, bnorm, rel_res_updated, rel_res_true; launches holds
 *    the number of lockstep blocks of the whole call. Device times are not
 *    recorded.
 * Temporary device memory: the bases, (2 s_max + 1) 8 round_up(n_q, 1024)
 * bytes per system as row ranges of one shared matrix, plus (2 s_max + 1)
 * (s_max + 1) 8 bytes of Gram partials per FP64 Gram item (1024 to 8192
 * rows: about n_q/16 as a power of two) and per tensor-core Gram item (8192
 * rows). n_tot = the sum of round_up(n_q, 1024) must be < 2^31. Runs on a
 * stream of its own, ordered after the caller's stream's earlier work.
 * Returns ASCG_OK when every system converged, else ASCG_NOT_CONVERGED or
 * ASCG_ERR_BREAKDOWN (the worst over the systems; results[q].status tells
 * which); ASCG_ERR_INVALID if some b or x_1 is not finite. Synchronises the
 * stream. */
ascg_status ascg_solve_batch(int count, const ascg_op* ops, const double* const* b, double* const* x,
                             const double* eps_target, const ascg_options* opts, ascg_result* results,
                             void* cuda_stream);

/* y = A x (device x, y of length n; x and y must not overlap). */
ascg_status ascg_spmv(ascg_op op, const double* x, double* y, void* cuda_stream);

/* Matrix powers, eq. (polybasiscg): on entry columns 0 (p) and 1 (r) of Y hold
 * p and r. Fills columns 2..2s by
 *   rho_{j+1} = ((A - theta_j) rho_j - sigma_{j-1} rho_{j-1}) / gamma_j.
 * theta, sigma, gamma: host double[s] (eq. (polybasiscg) coefficients;
 * sigma[j] multiplies rho_j when rho_{j+2} is formed; gamma[j] != 0; at most
 * two distinct gamma values other than 1). 1 <= s <= 16. The coefficients are
 * folded into the operator first ((D - theta_j)/gamma_j and O/gamma_j for
 * A = D + O), exactly as ascg_solve does, so this call runs the solver's own
 * kernel. */
ascg_status ascg_matrix_powers(ascg_op op, int s, const double* theta, const double* sigma,
                               const double* gamma, double* Y, int64_t ldY, void* cuda_stream);

/* Gram matrix G = Y^T Y of the first w columns of Y (Sec. 2.1): device Y as
 * above with n rows, device G double[w*w], row-major, symmetric (both halves
 * written). 1 <= w <= 33. Sums run in a fixed order: the result is bitwise
 * reproducible for a given n, w and device.
 * For w < 9 the products are FP64 FMAs (error <= gamma_n |Y|^T |Y| per
 * entry). For w >= 9 they run on the bf16 tensor cores with an error-free
 * split of Y: entries of column a are rounded to the grid 2^(E_a - 56), where
 * 2^(E_a - 1) <= max|y_a| < 2^E_a, written in seven base-256 digits, and the
 * digit products are summed exactly in integers. Per entry the error is at
 * most 2^-51 (max|y_a| ||y_b||_1 + max|y_b| ||y_a||_1) + gamma_(m) |y_a|^T |y_b|
 * (m = CTAs + 7); a column holding Inf or NaN gives NaN in its row and
 * column. If a bounded wait of the tensor-core kernel runs out (about 2 s),
 * G is NaN and the call returns ASCG_ERR_TIMEOUT. */
ascg_status ascg_gram(int64_t n, int w, const double* Y, int64_t ldY, double* G, void* cuda_stream);

/* Gram matrix of a monomial basis from its moments (a variant of ascg_gram;
 * the paper forms Y^T Y). With A symmetric and rho_j(z) = z^j, the blocks
 * P^T P, P^T R and R^T R of G depend on i + j only (Hankel matrices), so
 * 6s dot products replace w(w+1)/2, w = 2s + 1. Y: device, interleaved
 * columns as above (P_j = column 2j, R_j = column 2j+1), n rows, ldY >= n;
 * 1 <= s <= 16. The moments are
 *   mu_pp[k] = P_floor(k/2)^T P_ceil(k/2),  k = 0 .. 2s
 *   mu_pr[k] = P_ceil(k/2)^T R_floor(k/2),  k = 0 .. 2s-1
 *   mu_rr[k] = R_floor(k/2)^T R_ceil(k/2),  k = 0 .. 2s-2
 * each an FP64 dot product summed in a fixed order (error <= gamma_n
 * |y_a|^T |y_b|), and G[2i+a][2j+b] = mu_(ab)[i+j] (device, row-major w x w).
 * In exact arithmetic this is Y^T Y; in floating point it differs from it by
 * the rounding of the basis recurrence. Synchronises the stream. */
ascg_status ascg_gram_moments(int64_t n, int s, const double* Y, int64_t ldY, double* G, void* cuda_stream);

/* One block controller step on a given Gram matrix (Alg. 4, Sec. 3.2: the
 * choice of s~_k by eq. (condy), then the inner loop). G: device double[(2 sbar+1)^2],
 * interleaved order as above. method: ASCG_ADAPTIVE (eq. (condy) and, if
 * check_in_loop, eq. (check)) or ASCG_FIXED_S (s~ = sbar, no test).
 * nrows: length n of the basis vectors (sets the certification floor
 * (2i+1) sqrt(n) eps of kappa(G_{k,i})). eps_star: absolute target.
 * max_steps: cap on inner steps. bnorm: scales the residual history.
 * Outputs: coords: device double[3 * (2 sbar+1)] = x', r', p' (interleaved
 * order, zero beyond 2 s~+1); info: host record of the block; hist: host
 * double[3 * sbar] = alpha_j, beta_j, sqrt(max(r'^T G r', 0))/bnorm for
 * j = 1..s_k (may be NULL). Synchronises the stream. */
ascg_status ascg_block_step(int sbar, const double* G, int method, const double* theta,
                            const double* sigma, const double* gamma, int64_t nrows,
                            double eps_star, double c, int check_in_loop, int max_steps,
                            double bnorm, double* coords, ascg_block_info* info, double* hist,
                            void* cuda_stream);

/* Recovery, eq. (coords): x += Y x', r = Y r', p = Y p' using the first w
 * columns of Y. coords: device double[3w] (x', r', p'). x, r, p: device
 * double[n]. r and p may alias columns 1 and 0 of Y (each row is read before
 * it is written). */
ascg_status ascg_recover(int64_t n, int w, const double* Y, int64_t ldY, const double* coords,
                         double* x, double* r, double* p, void* cuda_stream);

/* Recovery, eq. (coords), on the tensor cores, as the solver runs it for a
 * block whose Gram took the tensor cores: x += Y x', r = Y r', p = Y p' in
 * one pass over Y. Each column of Y becomes a 55-bit fixed-point integer
 * relative to its largest entry (the Gram's digit split); each coefficient
 * vector takes its columns' scales in and becomes a 55-bit fixed-point
 * integer too; the digit products are summed exactly and each result is
 * rounded once to FP64. Error against the exact sum_j Y_ij c_j: at most
 * 2^-53 |result| + 2^-54 sum_j ||y_j||_inf |c_j| +
 * (w + 2) 2^-52 max_j ||y_j||_inf |c_j| (normwise; ascg_recover's is
 * componentwise), plus the rounding of x + (Y x')_i.
 *  - n, w, Y, ldY, coords, x, r, p: as for ascg_recover, with
 *    9 <= w <= 33, Y 16-byte aligned and ldY even (else ASCG_ERR_INVALID),
 *    n <= 2^31 - 1. r and p may alias columns 1 and 0 of Y.
 *  - Allocates 136 bytes of device memory for the column exponents and
 *    synchronises the stream. ASCG_ERR_TIMEOUT: a bounded wait of the kernel
 *    ran out (the outputs are then incomplete). */
ascg_status ascg_recover_tc(int64_t n, int w, const double* Y, int64_t ldY, const double* coords,
                            double* x, double* r, double* p, void* cuda_stream);

/* Newton basis shifts: Ritz values of the Lanczos tridiagonal of k classical
 * CG steps (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} =
 * sqrt(beta_j)/alpha_j), put in Leja order (first the largest magnitude, then
 * each next maximises the product of distances; ties to the larger value).
 * alphas: host double[k], betas: host double[k-1]; shifts: host double[s]
 * receives the first s values (s <= k <= 32). Synchronises the stream. */
ascg_status ascg_newton_shifts(const double* alphas, const double* betas, int k, int s,
                               double* shifts, void* cuda_stream);

/* Gram matrix G = Y^T Y exactly as ascg_gram computes it (same kernels, same
 * summation order, so the same bits), but without allocating device memory.
 * The paper has no counterpart: this exists for callers that must not call
 * cudaMalloc or cudaFree, such as code running under a fixed device-memory
 * budget owned by a host framework, or latency-sensitive loops where the
 * device-wide synchronisation of cudaFree would stall other streams.
 *  - Y, ldY, n, w, G: as for ascg_gram (device Y; device G of w*w doubles,
 *    row-major, both halves written). 1 <= w <= 33; larger w returns
 *    ASCG_ERR_INVALID.
 *  - The per-CTA partial sums live in one static device array of 160 x 561
 *    doubles (701 KB), and the per-CTA column exponents of the tensor-core
 *    kernel in one of 160 x 33 ints (21 KB). Every GPU that loads the library
 *    holds them until the process exits. A GPU that would use more than 160
 *    CTAs (more than 160 SMs) gets ASCG_ERR_INVALID.
 *  - Calls nothing that allocates: no cudaMalloc, cudaFree or allocating
 *    library routine. The first call on each device looks up the array's
 *    device address (cudaGetSymbolAddress) with that device current. Make
 *    that first call before any stream capture.
 *  - Every call uses the same array. Calls whose work overlaps on the GPU
 *    (for example on two streams at once) race and give wrong results:
 *    order them on one stream.
 *  - Returns once the work is enqueued on the stream (it does not
 *    synchronise), so it cannot report a device-side timeout: if a bounded
 *    wait of the tensor-core kernel runs out (about 2 s), every entry of G
 *    that the giving-up CTA contributes to is NaN. NaN in G with finite Y
 *    means exactly that. */
ascg_status ascg_gram_noalloc(int64_t n, int w, const double* Y, int64_t ldY, double* G, void* cuda_stream);

/* --- solve server (continuous batching) ------------------------------------
 * A request loop over the batched engine: requests of different sizes and
 * targets are submitted at any time, admitted while device memory and system
 * slots allow, and run block by block (Alg. 4) until they finish. Bases and
 * coefficients stay on the device between blocks. Running systems are split
 * by size into three classes (n < 2^16, < 2^19, larger); each class runs its
 * systems in lockstep on a stream of its own, and starts its next block as
 * soon as its previous one has landed, so the classes' blocks interleave on
 * the GPU and small systems do not wait for the blocks of large ones; the
 * smaller the class, the higher its stream priority. A
 * system's arithmetic depends on that system alone: its x, iteration count
 * and residuals are bitwise the same as from ascg_solve_batch with that
 * system alone, whatever else runs beside it.
 * Not safe for concurrent use from several threads. */
typedef struct ascg_server_s* ascg_server;

typedef struct {
  int64_t tag;               /* the caller's tag from ascg_server_submit           */
  ascg_result result;        /* as from ascg_solve_batch; result.launches = blocks
                                landed (all size classes) from admission to
                                completion                                       */
  double queue_ms;           /* host time from submit to admission                */
  double latency_ms;         /* host time from submit to completion               */
  int64_t step_admitted;     /* server block counter at admission / completion    */
  int64_t step_done;
} ascg_completion;

typedef struct {
  int64_t budget_bytes;      /* hbm_budget given at creation                       */
  int64_t basis_bytes_total; /* part of the budget that holds bases                */
  int64_t basis_bytes_used;  /* held by the running systems                        */
  int systems_running;
  int max_systems;
  int64_t queued;            /* submitted, not yet admitted                        */
  int64_t completions_pending; /* finished, not yet returned by ascg_server_step   */
  int64_t steps;             /* blocks landed, all size classes                    */
  int64_t launches;          /* kernels launched so far                            */
} ascg_server_stats;

/* Creates a server. opts: as for ascg_solve_batch (an s-step method, the
 * MONOMIAL basis; s_seq is copied), history buffers NULL; eps_target is per
 * request. hbm_budget: device bytes the server may hold for running
 * systems. A system of n rows holds (2 s_max + 1) 8 round_up(n, 1024) bytes
 * of basis (a row range of one shared matrix) plus (2 s_max + 1)(s_max + 1)
 * 8 bytes of Gram partials per FP64 Gram item (1024 to 8192 rows, about n/16
 * as a power of two) and per tensor-core Gram item (8192 rows). The basis
 * matrix takes the budget less the partials' share and is allocated here;
 * the partial and row-table buffers (about 16 bytes per 256 rows) grow on
 * demand within that share.
 * max_systems: most systems running at once (1 .. 2^20). cuda_stream: the
 * caller's stream, which orders submissions after the caller's work; the
 * server runs its blocks on streams of its own. The operators are the
 * caller's and are not counted. */
ascg_status ascg_server_create(const ascg_options* opts, int64_t hbm_budget, int max_systems,
                               void* cuda_stream, ascg_server* out);

/* Queues a request A x = b. op: an operator on the current device; b, x:
 * device double[n]; x holds x_1 and is updated in place while the system
 * runs, so b, x and op must stay valid and untouched until its completion is
 * returned. Work already queued on the server's stream (cuda_stream of
 * ascg_server_create) when this is called, such as the writes of b and x_1,
 * is done before the system starts. eps_target: relative target (eps* =
 * eps_target ||b||). tag: returned in the completion. ASCG_ERR_INVALID if
 * the system could never fit the budget. Launches nothing. */
ascg_status ascg_server_submit(ascg_server srv, ascg_op op, const double* b, double* x, double eps_target,
                               int64_t tag);

/* Advances the server until at least one block has landed (or there is no
 * work): completes the systems that finished (true residual computed, memory
 * freed), admits waiting requests, and starts the next block of every size
 * class that is idle and has running systems. Admission goes in submission
 * order; a request whose size class is in the middle of a block waits for
 * it while later requests of idle classes may go ahead, and the first
 * request that finds no free slot or no memory stops the scan (nothing
 * overtakes it). Writes up to cap completions to done (host) and their
 * number to *ndone; the rest wait for the next call. *nactive: systems
 * running; *npending: requests not yet admitted plus completions not yet
 * returned (the server is idle when both are 0). The blocks it starts may
 * still run on the GPU when it returns. */
ascg_status ascg_server_step(ascg_server srv, ascg_completion* done, int cap, int* ndone, int* nactive,
                             int* npending);

/* Admission policy of a server. */
typedef enum {
  ASCG_ADMIT_FIFO = 0,            /* the scan visits requests in submission order
                                     (the default)                               */
  ASCG_ADMIT_SHORTEST_FIRST = 1   /* in increasing estimated work: rows times the
                                     decimal digits of the target (n *
                                     max(1, -log10 eps_target)); ties in
                                     submission order                            */
} ascg_admit_order;

/* Sets the server's scheduling policy (host; takes effect at the next
 * ascg_server_step). admit_order: ascg_admit_order. large_class_cap > 0: at
 * most that many systems run at once in the largest size class (n >= 2^19),
 * whose kernels cover the whole GPU by themselves, so that running more of
 * them at once only shares the GPU among them; 0: no cap. yield_large != 0:
 * the largest class starts no block while a smaller class has systems
 * running, so that small and medium requests get the whole GPU (large
 * requests wait meanwhile: their latency grows). The other rules of
 * ascg_server_step stay: a class in the middle of a block admits nothing,
 * and the first request that finds no slot or no memory stops the scan. A
 * system's arithmetic does not depend on the policy. ASCG_ERR_INVALID for an
 * unknown order or a negative cap. */
ascg_status ascg_server_set_policy(ascg_server srv, int admit_order, int large_class_cap, int yield_large);

/* Counters of the server (host). */
ascg_status ascg_server_info(ascg_server srv, ascg_server_stats* stats);

/* Waits for the server's work on the GPU and frees the server. Requests not
 * yet completed are dropped (their x holds whatever iterate was reached).
 * NULL is accepted. */
ascg_status ascg_server_destroy(ascg_server srv);

/* Autotuner of the batched Gram schedule. For w = 2 s_max + 1 and sizes
 * n = 2^12, 2^13, ..., 2^22, times on this GPU the Gram of one system of n
 * rows (random basis) in the FP64 item launch and in the tensor-core item
 * launch (column exponents, kernel, finalize), each the median of several
 * runs. In a batch each launch covers all its systems and fills the GPU, so
 * a system costs the per-row rate at full load (taken at the largest size)
 * times the rows read: n in FP64, round_up(n, 1024) on the tensor cores.
 * Writes to *tc_lane_rows the smallest power of two >= 256 from which the
 * tensor cores cost less at every larger size (or -1 if they never do), for
 * ascg_options.tc_lane_rows. table (host, may be NULL): up to table_cap rows
 * of (n, FP64 us, tensor-core us). *rows: rows written. 1 <= s_max <= 16.
 * Uses about (2 s_max + 1) x 32 MB of device memory while it runs.
 * Synchronises the stream. */
ascg_status ascg_tune_gram_schedule(int s_max, int64_t* tc_lane_rows, double* table, int table_cap, int* rows,
                                    void* cuda_stream);

/* Message of the last error on this thread ("" if none). */
const char* ascg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ASCG_H */
