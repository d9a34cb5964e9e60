// Shared device helpers and kernel declarations of libascg.
//
// Arithmetic is IEEE double throughout. On GB300 the FP64 pipe retires one
// warp-wide DFMA per ~20 SM cycles (about 1.0 TFLOP/s per GPU), and an
// instruction costs the same with 1 or 32 active lanes. Kernels therefore
// keep every lane busy and count FP64 instructions, not bytes.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/ascg.h"

namespace ascg {

constexpr int kMaxS = ASCG_MAX_S;
constexpr int kMaxW = ASCG_MAX_W;                 // 33
constexpr int kMaxPairs = kMaxW * (kMaxW + 1) / 2;  // 561
constexpr double kEps = 1.1102230246251565e-16;   // 2^-53

// Sparse matrix on the device in sliced ELL form, slices of 32 rows (one warp
// per slice). Entry j of row 32 s + l sits at val[ptr[s] + 32 j + l]; a
// slice's width is its longest row, and shorter rows are padded with value 0
// and their own column index. Every load of a warp is then one contiguous
// 256-byte (values) or 128-byte (columns) segment. No shared-memory staging
// is needed, and the padding costs no more than the divergence that a
// thread-per-row CSR loop pays for the warp's longest row.
constexpr int kSlice = 32;
struct DevSell {
  int64_t n;
  const int64_t* ptr;   // ceil(n/32) + 1 element offsets
  const int32_t* col;
  const double* val;
};

// Rows (threads) per CTA of the SpMV-based kernels.
constexpr int kSpmvRows = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (devices 0..63; others every call). The device's
// flag is set only after the attribute call succeeded, so a caller that sees
// it may launch; two threads may both make the call, which is harmless.
template <typename K>
inline cudaError_t smem_limit_once(std::atomic<uint64_t>& done, K* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t)1 << dev : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel in the stream is still finishing, and waits for it (all its
// memory operations visible) with pdl_wait() before touching anything that
// kernel wrote. pdl_release() lets the next such kernel be scheduled as soon
// as every CTA of this one has started. Without the launch attribute both are
// no-ops, so the kernels stay correct under any launch. Every kernel launched
// this way calls pdl_wait() at entry: a kernel that returned before its
// predecessor finished would let its own successor overtake that predecessor.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  return launch_pdl_ex(kernel, dim3((unsigned)grid), dim3((unsigned)block), 0, s, args...);
}

// Number of blocks for a grid-stride kernel over n items.
inline int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Launchers (defined in the kernel .cu files). Each returns the CUDA error of
// the launch.
// ---------------------------------------------------------------------------

// y = A x
cudaError_t launch_spmv(const DevSell& A, const double* x, double* y, cudaStream_t s);
// r = b - A x; also writes p = r when p != nullptr
cudaError_t launch_residual(const DevSell& A, const double* b, const double* x, double* r,
                            double* p, cudaStream_t s);
// out[0] = sum_i u_i v_i over n, deterministic two-stage reduction.
// partials: device double[kRedBlocks], counter: device unsigned (zero on entry, left zero).
constexpr int kRedBlocks = 304;
cudaError_t launch_dot(const double* u, const double* v, int64_t n, double* out, double* partials,
                       unsigned* counter, cudaStream_t s);

// A split as D + O for the matrix powers kernel: O is the off-diagonal part in
// sliced ELL form (diagonal removed), D the diagonal.
struct DevSplit {
  DevSell O;
  int64_t o_len;        // elements of O's value array (padding included)
  const double* diag;
};

// Operator of one matrix powers step j (eq. polybasiscg) after folding the
// basis coefficients into the matrix:
//   rho_{j+1} = (Dt_j + Ot_j) rho_j - sig_j rho_{j-1},
//   Dt_j = (D - theta_j) / gamma_j,  Ot_j = O / gamma_j,  sig_j = sigma_{j-1} / gamma_j.
// One multiply for the diagonal, one FMA per off-diagonal nonzero and one FMA for
// the sigma term per row: nnz_row + 1 FP64 instructions instead of nnz_row + 3,
// and nnz_row when sig_j = 1 (the negated rho_{j-1} starts the sum).
struct StepOp {
  const double* oval;   // values of Ot_j (O's sliced ELL layout)
  const double* dtil;   // Dt_j, n values
  double sig;           // sig_j (0 for j = 0)
};
// Forms column 2(j+1) from 2j, 2(j-1), and column 2(j+1)+1 from 2j+1, 2j-1 if do_r.
// do_p must be 1 (cudaErrorInvalidValue otherwise): every step forms the P column.
// emax_part (device int[kMaxW * emax_ld] or nullptr, emax_ld >= ceil(n/32), a
// multiple of 4, entries past ceil(n/32) zero):
// per warp of 32 rows, the largest biased exponent of each column written (for
// j = 0 also of columns 0 and 1), at [col * emax_ld + warp].
// gate (device int, or nullptr): every kernel of a solver block takes the
// block's flag, and returns at once when it is 0 (a block enqueued ahead of the
// host's reading of the previous one, which ended the solve).
cudaError_t launch_mpk_split_step(const DevSplit& O, const StepOp& op, double* Y, int64_t ldY, int j, int do_p,
                                  int do_r, int* emax_part, int64_t emax_ld, cudaStream_t s,
                                  const int* gate = nullptr);
// col_emax[c] = max_k emax_part[c * emax_ld + k] for c < w, k < ceil(n/32).
cudaError_t launch_emax_reduce(const int* emax_part, int64_t emax_ld, int64_t n, int w, int* col_emax,
                               cudaStream_t s, const int* gate = nullptr);
// dst[i] = (src[i] - theta) * scale, for i < n
cudaError_t launch_shift_scale(const double* src, int64_t n, double theta, double scale, double* dst,
                               cudaStream_t s);

// Gram partials: per CTA, the upper triangle (row-major pair order) of Y^T Y.
int gram_grid();                // CTAs per launch at most (the SM count)
int gram_parts(int64_t n);      // CTAs (= partials) used for n rows
cudaError_t launch_gram_partial(int64_t n, int w, const double* Y, int64_t ldY, double* partials,
                                cudaStream_t s, const int* gate = nullptr);
// Sum the partials in a fixed order; G row-major w x w, both halves.
cudaError_t launch_gram_finalize(int w, const double* partials, int nparts, double* G, cudaStream_t s,
                                 const int* gate = nullptr);

// Batched solves: one Gram item = rows [row0, row0 + nrows) of system sys.
struct GramItem {
  int64_t row0;
  int nrows;
  int sys;
};
// Rows per Gram item of a system of n rows: about n/16 as a power of two,
// within [1024, 8192]. It depends on the system's own size only.
inline int64_t gram_item_rows(int64_t n) {
  int64_t r = 1024;
  while (r < 8192 && r * 16 < n) r *= 2;
  return r;
}
constexpr int kGramItemRowsMin = 1024;
// FP64 partials (W columns, W odd <= 33) of every item, rows read from the
// item's system (descs[sys].Y); items of systems with sys_w 0 are skipped.
// The pairs of each item are split over pair_groups CTAs (1 .. 65535), which
// changes no result. partials: nitems x W(W+1)/2.
struct SysDesc;
cudaError_t launch_gram_items(int W, const SysDesc* descs, const GramItem* items, int nitems, const int* sys_w,
                              double* partials, int pair_groups, bool moments, cudaStream_t s);
// G of each active system q (w_q = sys_w[q] x w_q, stride w_q) at G + q * g_stride.
cudaError_t launch_gram_items_finalize(int W, const double* partials, const int* sys_item0, const int* sys_nitems,
                                       const int* sys_w, int count, double* G, int64_t g_stride, bool moments,
                                       cudaStream_t s);
// Hankel-moment Gram of the monomial basis (interleaved columns P_j = 2j,
// R_j = 2j + 1, w = 2s + 1 odd >= 3): the 6s dot products
// mu_pp[k] = <P_floor(k/2), P_ceil(k/2)>, mu_pr[k] = <P_ceil(k/2), R_floor(k/2)>,
// mu_rr[k] = <R_floor(k/2), R_ceil(k/2)>, each in the FP64 kernel's fixed
// order, and G = [mu_(ab)[i + j]]. Partials: kMomSlots per CTA (or per item
// with moments = true above); slot = family * kMomFam + k.
constexpr int kMomFam = 2 * kMaxS + 1;
constexpr int kMomSlots = 3 * kMomFam;
cudaError_t launch_gram_moments(int64_t n, int w, const double* Y, int64_t ldY, double* partials, int* nparts,
                                cudaStream_t s, const int* gate = nullptr);
cudaError_t launch_gram_moment_finalize(int w, const double* partials, int nparts, double* G, cudaStream_t s,
                                        const int* gate = nullptr);

// Tensor-core Gram (split-bf16 operands, exact integer sums) for
// kGramTcMinW <= w <= kMaxW. Below that width the FP64 kernel is faster.
constexpr int kGramTcMinW = 9;
int gram_tc_parts(int64_t n);   // CTAs (= partials) of the tensor-core Gram
bool gram_tc_applies(int w);
// The tensor-core Gram needs 16-byte aligned columns: Y 16-byte aligned, ldY even.
bool gram_tc_aligned(const double* Y, int64_t ldY);
// Every mbarrier wait of the tensor-core Gram is bounded. A wait that runs out
// makes the CTA give up: it lets the copies and MMAs it already issued land,
// frees its tensor memory, writes NaN partials and, when err is given, sets
// *err = ASCG_ERR_TIMEOUT (device int). stall_stage >= 0 is the stall test:
// CTA 0 never issues the copy of that stage, so a wait runs out by
// construction; wait_limit is then a few milliseconds.
struct TcGuard {
  long long wait_limit;
  int stall_stage;
  int* err;
  const int* gate;  // see launch_mpk_split_step
};
// col_emax: device int[kMaxW], the largest biased exponent of each column;
// computed here unless emax_ready (then it already holds them, e.g. from the
// matrix powers kernel). partials as for launch_gram_partial. err: as in
// TcGuard (may be nullptr); stall_test: run the stall test (see TcGuard).
cudaError_t launch_gram_tc(int64_t n, int w, const double* Y, int64_t ldY, int* col_emax, bool emax_ready,
                           double* partials, cudaStream_t s, int* err = nullptr, bool stall_test = false,
                           const int* gate = nullptr);
// True when the tensor-core Gram can take n rows (at most 2^31 - 1 rows and
// 2048 chunks of 1024 rows per CTA); larger bases take the FP64 kernel.
bool gram_tc_fits(int64_t n);
// Partials of G with the kernel for this width (FP64 when force_fp64); returns
// the number of partials through *nparts.
// Tensor-core Gram of many systems whose bases are row ranges of one matrix
// Y (rows x w used, leading dimension ldY, rows a multiple of 1024): items
// are whole 1024-row chunks of one system each (GramItem rows in Y, nrows a
// multiple of 1024, at most 8 chunks); items of systems with sys_w 0 skip.
// Each item gets its system's column exponents (emax_all: nsys x 33 ints,
// zeroed and filled here) and writes w(w+1)/2 partials.
cudaError_t launch_gram_tc_items(int w, const double* Y, int64_t ldY, int64_t rows, const GramItem* items,
                                 int nitems, const int* sys_w, int nsys, int* emax_all, double* partials,
                                 cudaStream_t s);
// Recovery (eq. coords) on the tensor cores: x += Y x', r = Y r', p = Y p' in
// one pass, with the Gram's digit split of Y (col_emax: the Gram's column
// exponents, device int[kMaxW]) and coefficients (coords: device double[3w],
// x', r', p'). Each result is the FP64 rounding of a fixed-point sum, within a
// normwise bound (kernels_gram_tc.cu). kGramTcMinW <= w <= kMaxW, Y aligned
// as for the tensor-core Gram; r and p may be columns 1 and 0 of Y. err and
// gate: as in TcGuard.
cudaError_t launch_recover_tc(int64_t n, int w, const double* Y, int64_t ldY, const int* col_emax,
                              const double* coords, double* x, double* r, double* p, cudaStream_t s,
                              int* err = nullptr, const int* gate = nullptr);
// The largest biased exponent of each column into col_emax (device int[kMaxW]).
cudaError_t launch_col_exponents(int64_t n, int w, const double* Y, int64_t ldY, int* col_emax, cudaStream_t s);
cudaError_t launch_gram_any(int64_t n, int w, const double* Y, int64_t ldY, bool force_fp64, int* col_emax,
                            bool emax_ready, double* partials, int* nparts, cudaStream_t s, int* err = nullptr,
                            bool stall_test = false, const int* gate = nullptr);

// Many systems in lockstep (kernels_batch.cu): a device table of per-system
// descriptors and row items of one system each (up to kRowItem rows starting
// on a 32-row slice).
struct SysDesc {
  int64_t n;
  const int64_t* o_ptr;   // O (off-diagonal part of A) in sliced ELL form
  const int32_t* o_col;
  const double* o_val;
  const double* diag;     // D
  double* Y;              // basis, column 0 = p, column 1 = r
  int64_t ldY;
  double* x;
  const double* b;
};
constexpr int kRowItem = 256;
struct RowItem {
  int sys;
  int row0;
  int nrows;
  int pad_;
};
// Matrix powers step j (monomial basis) of every system q with j < sys_steps[q].
cudaError_t launch_mpk_items(const SysDesc* descs, const RowItem* items, int nitems, const int* sys_steps, int j,
                             cudaStream_t s);
// b - A x of the systems with sel[q] != 0: into Y columns 1 and 0, or into column 2.
cudaError_t launch_residual_items(const SysDesc* descs, const RowItem* items, int nitems, const int* sel,
                                  int into_col2, cudaStream_t s);
// out[q] = sum of squares (fixed order) of b (which 0) or Y column `which` of the systems in list.
cudaError_t launch_seg_sumsq(const SysDesc* descs, const int* list, int nlist, int which, double* out,
                             cudaStream_t s);
// count values in [-1, 1) from a hash of (seed, index) (timing data).
cudaError_t launch_fill_uniform(double* v, int64_t count, uint64_t seed, cudaStream_t s);
// Recovery of every system with w_q = sys_w[q] > 0 (W >= max w_q), coordinates at coords + q * c_stride.
cudaError_t launch_recover_items(int W, const SysDesc* descs, const RowItem* items, int nitems, const int* sys_w,
                                 const double* coords, int64_t c_stride, cudaStream_t s);

// Recovery (eq. coords).
cudaError_t launch_recover(int64_t n, int w, const double* Y, int64_t ldY, const double* coords,
                           double* x, double* r, double* p, cudaStream_t s);
// The recovery in two parts with the same bits: r = Y r', p = Y p' (r and p
// must not alias Y), and x += Y x' on `ctas` CTAs of which no two share an SM
// and none shares an SM with a kernel holding more than ~6 KB of shared
// memory.
cudaError_t launch_recover_rp(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* r,
                              double* p, cudaStream_t s, const int* gate = nullptr);
cudaError_t launch_recover_x(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* x,
                             int ctas, cudaStream_t s, const int* gate = nullptr);

// Block controller state shared by the controller kernels and the host driver.
struct BlockState {
  // inputs set by the host before the block
  int sbar;
  int method;          // ASCG_ADAPTIVE or ASCG_FIXED_S
  int check_in_loop;
  int max_steps;
  int m;               // iterations before this block
  int k;               // block index
  double eps_star;
  double c;            // c_{k,j} when c_step is 0
  double c_step;       // > 0: c_{k,j} = c_step * j, and c_step * c_smax in eq. (condy)
  int c_smax;
  int pad2_;
  double bnorm;
  double sqrt_n;       // sqrt(length of the basis vectors)
  int active;          // batched solves: 0 skips this system's block (single solves: 1)
  int pad_;
  // outputs
  int stilde;
  int s_k;
  int stop;
  int converged;
  int status;          // ascg_status of the device side
  double rnorm;
  double threshold;
  double gamma;
  double rel_res;      // sqrt(max(r'Gr',0)) / bnorm after the last step
  double sqrt_kappa[kMaxS];
};

// The block after its Gram matrix G (w x w, w = 2 sbar + 1, row-major): the
// condition estimates kappa(G_{k,i}), i = 1..sbar (adaptive only), the choice
// of s~ (eq. condy), B (eq. AVVB) and the inner loop with eq. (check); writes
// st's outputs, coords[3w] (x', r', p') and the histories. theta/sigma/gamma:
// device double[kMaxS]. hist: device double[3 * kMaxS] per block (alpha,
// beta, rel res) or nullptr; res_hist: device array indexed by iteration,
// capacity res_cap (entries m+1 .. m+s_k written), or nullptr. spec: device
// scratch of kSpecDoubles; counter: device unsigned, zero on entry and left
// zero. adaptive: st->method == ASCG_ADAPTIVE.
constexpr int kSpecDoubles = kMaxS * (3 * kMaxW + 3) + 1;
cudaError_t launch_block_ctrl(const double* G, const double* theta, const double* sigma, const double* gamma,
                              BlockState* st, int sbar, int adaptive, double* coords, double* hist, double* res_hist,
                              int res_cap, double* ab_hist, int ab_cap, double* spec, unsigned* counter,
                              cudaStream_t s);
// The same for `count` systems (shared theta/sigma/gamma): system q uses
// G + q * g_stride, st + q (its own sbar <= max_sbar), coords + q * c_stride,
// res_hist + q * res_cap, ab_hist + q * 2 * ab_cap (histories may be nullptr),
// spec + q * kSpecDoubles and counters + q; inactive systems skip.
cudaError_t launch_block_ctrl_batch(const double* G, int64_t g_stride, const double* theta, const double* sigma,
                                    const double* gamma, BlockState* st, int count, int max_sbar, int adaptive,
                                    double* coords, int64_t c_stride, double* res_hist, int res_cap, double* ab_hist,
                                    int ab_cap, double* spec, unsigned* counters, cudaStream_t s);

// Block j+1 of a single solve from block j's record (m, k, iteration budget,
// and the flag that gates every kernel of block j+1).
cudaError_t launch_block_advance(const BlockState* prev, BlockState* cur, int max_iters, cudaStream_t s);

// Newton shifts: Ritz values of the CG tridiagonal, Leja order. alphas, betas:
// device; shifts: device double[k].
cudaError_t launch_newton_shifts(const double* alphas, const double* betas, int k, double* shifts,
                                 cudaStream_t s);

// Classical CG (Alg. 1). State lives on the device.
struct CGState {
  double rr;        // r^T r
  double pAp;
  double alpha;
  double beta;
  double eps_star;
  double bnorm;
  int iter;         // iterations completed
  int max_iters;
  int done;         // 1 once converged or capped
  int converged;
  int active;       // 1 if the current iteration runs (set by the SpMV kernel)
  int breakdown;    // 1 once p^T A p was not positive and finite (the solve stops)
};
// q = A p, state.pAp; the last CTA sets alpha. nnz: A's nonzeros (a large A
// is streamed past L2, see sell_row).
cudaError_t launch_cg_spmv_dot(const DevSell& A, int64_t nnz, const double* p, double* q, CGState* st,
                               double* partials, unsigned* counter, cudaStream_t s);
// r -= alpha q, rr_new; the last CTA sets beta, records histories, tests
// convergence.
cudaError_t launch_cg_update(int64_t n, double* r, const double* q, CGState* st, double* partials,
                             unsigned* counter, double* res_hist, int res_cap, double* alpha_hist, double* beta_hist,
                             int ab_cap, cudaStream_t s);
// x += alpha p (the iteration's p), then p = r + beta p
cudaError_t launch_cg_pupdate(int64_t n, double* x, const double* r, double* p, const CGState* st, cudaStream_t s);
// CG state init from rr = r^T r computed into st->rr.
cudaError_t launch_cg_init(CGState* st, double eps_star, double bnorm, int max_iters, int iter0,
                           double* res_hist, int res_cap, cudaStream_t s);

// Basis size sbar_k of block k: s_max (Alg. 2), s_seq[min(k, len - 1)]
// (Alg. 3), s0 then min(s_{k-1} + f, s_max) (Alg. 4).
inline int block_sbar(const ascg_options& o, int k, int s_prev) {
  if (o.method == ASCG_FIXED_S) return o.s_max;
  if (o.method == ASCG_VARIABLE_S) return o.s_seq[k < o.s_seq_len ? k : o.s_seq_len - 1];
  return k == 0 ? o.s0 : (s_prev + o.f < o.s_max ? s_prev + o.f : o.s_max);
}

// Sets the message that ascg_last_error() returns on this thread.
void set_last_error(const std::string& msg);
// Batched solves on the lockstep engine (lockstep.cu).
ascg_status lockstep_solve_batch(int count, const ascg_op* ops, const double* const* b, double* const* x,
                                 const double* eps_target, const ascg_options& o, ascg_result* results,
                                 cudaStream_t s);

}  // namespace ascg
