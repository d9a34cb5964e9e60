// Host side of the libascg C ABI (include/ascg.h): operator, workspace and the
// solve drivers for Alg. 1 (classical CG), Alg. 2 (fixed s) and Alg. 4
// (adaptive s).
//
// Per block the device runs, in stream order: s matrix powers steps, the Gram
// partials and their fixed-order sum (the block's single grid-wide
// reduction, Sec. 2.1), the condition estimates, the controller, and the
// recovery. The host reads back one small status record per block, since the
// next block's basis size sbar_k = min(s_{k-1} + f, s_max) depends on it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ascg_common.cuh"

using namespace ascg;

namespace {

thread_local std::string g_err;

ascg_status fail(ascg_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define ASCG_CUDA(call)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? ASCG_ERR_OOM : ASCG_ERR_CUDA,              \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

#define ASCG_TRY(expr)              \
  do {                              \
    ascg_status s_ = (expr);        \
    if (s_ != ASCG_OK) return s_;   \
  } while (0)

template <class T>
ascg_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(ASCG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return ASCG_OK;
}

template <class T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Records of the blocks in flight: block j uses slot j % kRing.
constexpr int kRing = 4;

// Device workspace owned by an operator; grows on demand.
struct Workspace {
  int64_t n = 0;
  int wcols = 0;
  int64_t ldY = 0;
  double* Y = nullptr;
  double* Y2 = nullptr;     // second basis buffer: blocks alternate, so x += Y x' can run late
  double* b = nullptr;      // for host-buffer solves
  double* x = nullptr;      // for host-buffer solves
  double* q = nullptr;      // classical CG: A p; also a scratch vector
  double* partials = nullptr;
  int64_t partials_cap = 0;
  int* expp = nullptr;      // column exponents of the tensor-core Gram, gram_grid() x kMaxW
  int* emax_part = nullptr; // per-warp column exponents from the matrix powers steps, kMaxW x emax_ld
  int64_t emax_ld = 0;
  unsigned* counter = nullptr;
  double* G = nullptr;      // kMaxW^2
  double* coords = nullptr; // 3 kMaxW
  double* params = nullptr; // theta, sigma, gamma: 3 kMaxS
  double* scal = nullptr;   // 4 scalars
  double* spec = nullptr;   // speculative coordinate steps of a block (kSpecDoubles)
  double* shifts = nullptr; // 32
  BlockState* bst = nullptr;
  CGState* cgs = nullptr;
  double* res_hist = nullptr;
  int res_cap = 0;
  double* ab_hist = nullptr;  // alpha[ab_cap], beta[ab_cap]
  int ab_cap = 0;
  double* dtils = nullptr;      // folded diagonals Dt_j, kMaxS x n
  double* oscaled[2] = {};      // O / gamma for up to two gamma != 1
  bool steps_ready = false;
  // pinned host mirrors
  BlockState* h_bst = nullptr;
  CGState* h_cgs = nullptr;
  double* h_scal = nullptr;
  cudaEvent_t ev[8] = {};
  cudaEvent_t ev_blk[kRing][5] = {};  // per record slot: the phase boundaries of a block (timing)
  cudaEvent_t ev_rec[kRing] = {};     // per record slot: the block's record is on the host
  bool events = false;
  cudaStream_t side = nullptr;  // x += Y x' of the previous block
  cudaEvent_t ev_gram = nullptr, ev_x[2] = {};

  void release() {
    dev_free(Y); dev_free(Y2); dev_free(b); dev_free(x); dev_free(q); dev_free(partials); dev_free(expp); dev_free(emax_part); dev_free(counter);
    dev_free(G); dev_free(coords); dev_free(params); dev_free(scal); dev_free(spec); dev_free(shifts);
    dev_free(bst); dev_free(cgs); dev_free(res_hist); dev_free(ab_hist);
    dev_free(dtils); dev_free(oscaled[0]); dev_free(oscaled[1]);
    steps_ready = false;
    if (h_bst) cudaFreeHost(h_bst);
    if (h_cgs) cudaFreeHost(h_cgs);
    if (h_scal) cudaFreeHost(h_scal);
    h_bst = nullptr; h_cgs = nullptr; h_scal = nullptr;
    if (events) {
      for (auto& e : ev) cudaEventDestroy(e);
      for (auto& row : ev_blk)
        for (auto& e : row) cudaEventDestroy(e);
      for (auto& e : ev_rec) cudaEventDestroy(e);
      cudaEventDestroy(ev_gram);
      for (auto& e : ev_x) cudaEventDestroy(e);
      if (side) cudaStreamDestroy(side);
    }
    events = false;
    side = nullptr;
    ev_gram = nullptr;
    ev_x[0] = ev_x[1] = nullptr;
    n = 0; wcols = 0; ldY = 0; partials_cap = 0; res_cap = 0; ab_cap = 0; emax_ld = 0;
  }
};

}  // namespace

struct ascg_op_s {
  int64_t n = 0, nnz = 0;
  int device = 0;
  int max_row_nnz = 0;  // N_A (Sec. 3.1): most nonzeros in a row of A
  // A in sliced ELL form (SpMV, residual, classical CG)
  int64_t* a_ptr = nullptr;
  int32_t* a_col = nullptr;
  double* a_val = nullptr;
  // A = D + O for the matrix powers kernel, O in sliced ELL form
  int64_t o_len = 0;
  int64_t* o_ptr = nullptr;
  int32_t* o_col = nullptr;
  double* o_val = nullptr;
  double* diag = nullptr;
  Workspace ws;
  DevSell sell() const { return DevSell{n, a_ptr, a_col, a_val}; }
  DevSplit split() const { return DevSplit{DevSell{n, o_ptr, o_col, o_val}, o_len, diag}; }
  void free_device() {
    dev_free(a_ptr); dev_free(a_col); dev_free(a_val);
    dev_free(o_ptr); dev_free(o_col); dev_free(o_val); dev_free(diag);
  }
};

namespace {

// Host construction of a sliced ELL matrix (see DevSell) from CSR. With
// drop_diag, diagonal entries are summed into diag[] and left out.
struct HostSell {
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

HostSell build_sell(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, bool drop_diag,
                    std::vector<double>* diag) {
  const int64_t nsl = (n + kSlice - 1) / kSlice;
  HostSell h;
  h.ptr.assign(nsl + 1, 0);
  for (int64_t s = 0; s < nsl; ++s) {
    int64_t width = 0;
    for (int64_t i = s * kSlice; i < std::min<int64_t>(n, (s + 1) * kSlice); ++i) {
      int64_t len = 0;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) len += !(drop_diag && ci[k] == i);
      width = std::max(width, len);
    }
    h.ptr[s + 1] = h.ptr[s] + width * kSlice;
  }
  h.col.assign(h.ptr[nsl], 0);
  h.val.assign(h.ptr[nsl], 0.0);
  for (int64_t s = 0; s < nsl; ++s) {
    const int64_t width = (h.ptr[s + 1] - h.ptr[s]) / kSlice;
    for (int l = 0; l < kSlice; ++l) {
      const int64_t i = s * kSlice + l;
      int64_t j = 0;
      if (i < n) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
          if (drop_diag && ci[k] == i) {
            (*diag)[i] += va[k];
            continue;
          }
          h.col[h.ptr[s] + j * kSlice + l] = ci[k];
          h.val[h.ptr[s] + j * kSlice + l] = va[k];
          ++j;
        }
      }
      for (; j < width; ++j)  // padding: value 0, a valid column (the row itself)
        h.col[h.ptr[s] + j * kSlice + l] = (int32_t)std::min<int64_t>(i, n - 1);
    }
  }
  return h;
}

template <class T>
ascg_status upload(T** dst, const std::vector<T>& src) {
  ASCG_TRY(dev_alloc(dst, src.size()));
  if (!src.empty()) ASCG_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return ASCG_OK;
}

}  // namespace

namespace {

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Products n w(w+1)/2 from which a single solve's Gram runs on the tensor
// cores by default (measured on GB300: the tensor-core kernel costs about
// 40 us at n = 1024, w = 17, where the FP64 kernel takes a few).
constexpr double kTcSolveProducts = 33554432.0;  // 2^25

// Ensures the workspace can hold n rows, wcols basis columns and histories of
// res_cap entries.
ascg_status ensure(ascg_op op, int wcols, int res_cap) {
  Workspace& w = op->ws;
  const int64_t n = op->n;
  if (!w.counter) {
    ASCG_TRY(dev_alloc(&w.counter, 2));  // [0]: reductions, [1]: the block controller's ticket
    ASCG_CUDA(cudaMemset(w.counter, 0, 2 * sizeof(unsigned)));
    ASCG_TRY(dev_alloc(&w.spec, kSpecDoubles));
    ASCG_TRY(dev_alloc(&w.G, kMaxW * kMaxW));
    ASCG_TRY(dev_alloc(&w.coords, 6 * kMaxW));  // two blocks' x', r', p'  
    ASCG_TRY(dev_alloc(&w.params, 3 * kMaxS));
    ASCG_TRY(dev_alloc(&w.scal, 4));
    ASCG_TRY(dev_alloc(&w.shifts, 32));
    ASCG_TRY(dev_alloc(&w.bst, kRing));
    ASCG_TRY(dev_alloc(&w.cgs, 1));
    ASCG_CUDA(cudaMallocHost((void**)&w.h_bst, 2 * kRing * sizeof(BlockState)));
    ASCG_CUDA(cudaMallocHost((void**)&w.h_cgs, sizeof(CGState)));
    ASCG_CUDA(cudaMallocHost((void**)&w.h_scal, 4 * sizeof(double)));
    for (auto& e : w.ev) ASCG_CUDA(cudaEventCreate(&e));
    for (auto& row : w.ev_blk)
      for (auto& e : row) ASCG_CUDA(cudaEventCreate(&e));
    for (auto& e : w.ev_rec) ASCG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ASCG_CUDA(cudaEventCreateWithFlags(&w.ev_gram, cudaEventDisableTiming));
    for (auto& e : w.ev_x) ASCG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ASCG_CUDA(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
    w.events = true;
  }
  if (w.n != n || w.wcols < wcols) {
    dev_free(w.Y); dev_free(w.Y2); dev_free(w.q);
    const int64_t ld = round_up(n, 32);  // 256-byte aligned columns
    const int cols = wcols > 2 ? wcols : 2;
    ASCG_TRY(dev_alloc(&w.Y, (size_t)(cols * ld)));
    if (wcols > 2) ASCG_TRY(dev_alloc(&w.Y2, (size_t)(cols * ld)));
    ASCG_TRY(dev_alloc(&w.q, (size_t)n));
    w.ldY = ld;
    w.wcols = cols;
    w.n = n;
  }
  const int64_t spmv_blocks = (n + kSpmvRows - 1) / kSpmvRows;
  const int64_t pcap = std::max<int64_t>(std::max<int64_t>(spmv_blocks, kRedBlocks),
                                         (int64_t)gram_grid() * kMaxPairs);
  if (w.partials_cap < pcap) {
    dev_free(w.partials);
    ASCG_TRY(dev_alloc(&w.partials, (size_t)pcap));
    w.partials_cap = pcap;
  }
  if (!w.expp) ASCG_TRY(dev_alloc(&w.expp, (size_t)gram_grid() * kMaxW));
  if (wcols > 2 && w.emax_ld < round_up((n + 31) / 32, 4)) {
    dev_free(w.emax_part);
    w.emax_ld = round_up((n + 31) / 32, 4);  // int4 rows; entries past the warp count stay zero
    ASCG_TRY(dev_alloc(&w.emax_part, (size_t)kMaxW * w.emax_ld));
    ASCG_CUDA(cudaMemset(w.emax_part, 0, sizeof(int) * kMaxW * w.emax_ld));
  }
  if (wcols > 2 && !w.dtils) {
    ASCG_TRY(dev_alloc(&w.dtils, (size_t)kMaxS * n));
    ASCG_TRY(dev_alloc(&w.oscaled[0], (size_t)op->o_len));
    ASCG_TRY(dev_alloc(&w.oscaled[1], (size_t)op->o_len));
  }
  if (w.res_cap < res_cap) {
    dev_free(w.res_hist); dev_free(w.ab_hist);
    ASCG_TRY(dev_alloc(&w.res_hist, (size_t)res_cap));
    ASCG_TRY(dev_alloc(&w.ab_hist, (size_t)2 * res_cap));
    w.res_cap = res_cap;
    w.ab_cap = res_cap;
  }
  return ASCG_OK;
}

// ||B_{k,s}||_2 of eq. (AVVB) for the basis coefficients th, sg, gm. B is
// block diagonal; its R block is a submatrix of its P block (the same
// coefficients, one column fewer), so the norm is that of the P block:
// (s+1) x (s+1), column j < s holding sg[j-1] above, th[j] on and gm[j]
// below the diagonal. The largest eigenvalue of P^T P comes from cyclic
// Jacobi rotations (a standard dense symmetric eigenvalue method).
double norm_B(int s, const double* th, const double* sg, const double* gm) {
  const int m = s + 1;
  double Bp[kMaxS + 1][kMaxS + 1] = {};
  for (int j = 0; j < s; ++j) {
    Bp[j][j] = th[j];
    Bp[j + 1][j] = gm[j];
    if (j >= 1) Bp[j - 1][j] = sg[j - 1];
  }
  double M[kMaxS + 1][kMaxS + 1];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      double acc = 0.0;
      for (int r = 0; r < m; ++r) acc += Bp[r][a] * Bp[r][b];
      M[a][b] = acc;
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int a = 0; a < m; ++a) {
      diag += M[a][a] * M[a][a];
      for (int b = a + 1; b < m; ++b) off += M[a][b] * M[a][b];
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        if (M[p][q] == 0.0) continue;
        const double theta = (M[q][q] - M[p][p]) / (2.0 * M[p][q]);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < m; ++r) {  // M <- M J
          const double mp = M[r][p], mq = M[r][q];
          M[r][p] = c * mp - sn * mq;
          M[r][q] = sn * mp + c * mq;
        }
        for (int r = 0; r < m; ++r) {  // M <- J^T M
          const double mp = M[p][r], mq = M[q][r];
          M[p][r] = c * mp - sn * mq;
          M[q][r] = sn * mp + c * mq;
        }
      }
  }
  double lmax = 0.0;
  for (int a = 0; a < m; ++a) lmax = std::max(lmax, M[a][a]);
  return std::sqrt(lmax);
}

ascg_status check_opts(const ascg_options& o) {
  if (o.method != ASCG_CLASSICAL && o.method != ASCG_FIXED_S && o.method != ASCG_ADAPTIVE &&
      o.method != ASCG_VARIABLE_S)
    return fail(ASCG_ERR_INVALID, "unknown method");
  if (o.method == ASCG_VARIABLE_S) {
    if (!o.s_seq || o.s_seq_len < 1) return fail(ASCG_ERR_INVALID, "ASCG_VARIABLE_S needs s_seq and s_seq_len >= 1");
    for (int i = 0; i < o.s_seq_len; ++i)
      if (o.s_seq[i] < 1 || o.s_seq[i] > o.s_max) return fail(ASCG_ERR_INVALID, "s_seq entries must be in 1..s_max");
  }
  if (o.method != ASCG_CLASSICAL) {
    if (o.s_max < 1 || o.s_max > ASCG_MAX_S) return fail(ASCG_ERR_INVALID, "s_max must be in 1..16");
    if (o.s0 < 1 || o.s0 > o.s_max) return fail(ASCG_ERR_INVALID, "s0 must be in 1..s_max");
    if (o.f < 1) return fail(ASCG_ERR_INVALID, "f must be >= 1");
    if (o.basis != ASCG_MONOMIAL && o.basis != ASCG_NEWTON && o.basis != ASCG_CHEBYSHEV)
      return fail(ASCG_ERR_INVALID, "unknown basis");
    if (o.basis == ASCG_CHEBYSHEV && !(o.lambda_max > o.lambda_min))
      return fail(ASCG_ERR_INVALID, "Chebyshev basis needs lambda_max > lambda_min");
    if (o.basis == ASCG_NEWTON) {
      const int nw = o.newton_warmup > 0 ? o.newton_warmup : 2 * o.s_max;
      if (nw < o.s_max || nw > 32) return fail(ASCG_ERR_INVALID, "newton_warmup must be in s_max..32");
    }
  }
  if ((o.flags & ASCG_FLAG_GRAM_TC) && (o.flags & (ASCG_FLAG_GRAM_FP64 | ASCG_FLAG_MOMENT_GRAM)))
    return fail(ASCG_ERR_INVALID, "ASCG_FLAG_GRAM_TC excludes ASCG_FLAG_GRAM_FP64 and ASCG_FLAG_MOMENT_GRAM");
  if ((o.flags & ASCG_FLAG_MOMENT_GRAM) && (o.method == ASCG_CLASSICAL || o.basis != ASCG_MONOMIAL))
    return fail(ASCG_ERR_INVALID, "ASCG_FLAG_MOMENT_GRAM needs an s-step method with the monomial basis");
  if (o.flags & ASCG_FLAG_C_FORMULA) {
    if (o.method != ASCG_ADAPTIVE) return fail(ASCG_ERR_INVALID, "ASCG_FLAG_C_FORMULA needs ASCG_ADAPTIVE");
    if (!(o.kappa_A >= 1.0 && std::isfinite(o.kappa_A)) || !(o.norm_A > 0.0 && std::isfinite(o.norm_A)))
      return fail(ASCG_ERR_INVALID, "ASCG_FLAG_C_FORMULA needs finite kappa_A >= 1 and norm_A > 0");
  }
  if (!(o.eps_target >= 0.0)) return fail(ASCG_ERR_INVALID, "eps_target must be >= 0");
  if (!(o.c > 0.0)) return fail(ASCG_ERR_INVALID, "c must be > 0");
  if (o.max_iters < 0) return fail(ASCG_ERR_INVALID, "max_iters must be >= 0");
  return ASCG_OK;
}

// theta, sigma, gamma of eq. (polybasiscg) for monomial and Chebyshev bases.
void basis_params(const ascg_options& o, double* th, double* sg, double* gm) {
  for (int j = 0; j < kMaxS; ++j) {
    th[j] = 0.0;
    sg[j] = 0.0;
    gm[j] = 1.0;
  }
  if (o.basis == ASCG_CHEBYSHEV) {
    // rho_j(z) = T_j((z - c)/h): theta_j = c, gamma_0 = h, gamma_j = h/2, sigma_j = h/2
    const double c = (o.lambda_max + o.lambda_min) / 2, h = (o.lambda_max - o.lambda_min) / 2;
    for (int j = 0; j < kMaxS; ++j) {
      th[j] = c;
      sg[j] = h / 2;
      gm[j] = j == 0 ? h : h / 2;
    }
  }
}

// Runs classical CG iterations (Alg. 1) on the device until the CG state says
// done. x, r, p, q are device vectors. Returns the iterations done by this call.
// Per-step operators of the matrix powers recurrence with theta, sigma and gamma
// folded in (see StepOp). dtils: n x s doubles; oscaled: two arrays of o_len
// doubles (used when gamma != 1; at most two distinct gamma values, which covers
// the monomial, Chebyshev and Newton bases).
ascg_status prepare_steps(ascg_op op, const double* th, const double* sg, const double* gm, int s, double* dtils,
                          double* const oscaled[2], StepOp* out, cudaStream_t st, int* launches) {
  double gam_of[2] = {0.0, 0.0};
  int ng = 0;
  for (int j = 0; j < s; ++j) {
    if (!(gm[j] != 0.0) || !std::isfinite(gm[j]) || !std::isfinite(th[j]))
      return fail(ASCG_ERR_INVALID, "basis coefficients must be finite with gamma != 0");
    const double inv = 1.0 / gm[j];
    const double* ov = op->o_val;
    if (gm[j] != 1.0) {
      int slot = -1;
      for (int q = 0; q < ng; ++q)
        if (gam_of[q] == gm[j]) slot = q;
      if (slot < 0) {
        if (ng == 2) return fail(ASCG_ERR_INVALID, "at most two distinct gamma != 1 are supported");
        slot = ng++;
        gam_of[slot] = gm[j];
        ASCG_CUDA(launch_shift_scale(op->o_val, op->o_len, 0.0, inv, oscaled[slot], st));
        ++*launches;
      }
      ov = oscaled[slot];
    }
    const double* dt = nullptr;
    if (th[j] == 0.0 && gm[j] == 1.0) dt = op->diag;
    for (int q = 0; q < j && !dt; ++q)
      if (th[q] == th[j] && gm[q] == gm[j]) dt = out[q].dtil;
    if (!dt) {
      double* dst = dtils + (int64_t)j * op->n;
      ASCG_CUDA(launch_shift_scale(op->diag, op->n, th[j], inv, dst, st));
      ++*launches;
      dt = dst;
    }
    // sig_j = sigma_{j-1} / gamma_j, exactly 1 when the two are equal (Chebyshev)
    const double sj = j < 1 ? 0.0 : (sg[j - 1] == gm[j] ? 1.0 : sg[j - 1] * inv);
    out[j] = StepOp{ov, dt, sj};
  }
  return ASCG_OK;
}

ascg_status run_classical(ascg_op op, double* x, double* r, double* p, double eps_star, double bnorm,
                          int max_iters, int iter0, cudaStream_t s, ascg_result* res, bool timing) {
  Workspace& w = op->ws;
  const int64_t n = op->n;
  const DevSell A = op->sell();
  ASCG_CUDA(launch_dot(r, r, n, &w.cgs->rr, w.partials, w.counter, s));
  ASCG_CUDA(launch_cg_init(w.cgs, eps_star, bnorm, max_iters, iter0, w.res_hist, w.res_cap, s));
  res->launches += 2;
  res->grid_reductions += 1;
  if (timing) ASCG_CUDA(cudaEventRecord(w.ev[6], s));
  int batch = 8;
  for (;;) {
    for (int i = 0; i < batch; ++i) {
      ASCG_CUDA(launch_cg_spmv_dot(A, op->nnz, p, w.q, w.cgs, w.partials, w.counter, s));
      ASCG_CUDA(launch_cg_update(n, r, w.q, w.cgs, w.partials, w.counter, w.res_hist, w.res_cap, w.ab_hist,
                                 w.ab_hist + w.ab_cap, w.ab_cap, s));
      ASCG_CUDA(launch_cg_pupdate(n, x, r, p, w.cgs, s));
    }
    res->launches += 3 * batch;
    ASCG_CUDA(cudaMemcpyAsync(w.h_cgs, w.cgs, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    ASCG_CUDA(cudaStreamSynchronize(s));
    if (w.h_cgs->done) break;
    if (batch < 64) batch *= 2;
  }
  if (timing) {
    ASCG_CUDA(cudaEventRecord(w.ev[7], s));
    ASCG_CUDA(cudaEventSynchronize(w.ev[7]));
    float ms = 0.f;
    ASCG_CUDA(cudaEventElapsedTime(&ms, w.ev[6], w.ev[7]));
    res->t_cg_ms += ms;
  }
  res->grid_reductions += 2 * (w.h_cgs->iter - iter0);
  return ASCG_OK;
}

ascg_status solve_device(ascg_op op, const double* b, double* x, const ascg_options& o, ascg_result* res,
                         cudaStream_t s) {
  Workspace& w = op->ws;
  const int64_t n = op->n;
  const DevSell A = op->sell();
  const bool sstep = o.method != ASCG_CLASSICAL;
  const int wmax = sstep ? 2 * o.s_max + 1 : 2;
  ASCG_TRY(ensure(op, wmax, o.max_iters + 2));
  const bool timing = (o.flags & ASCG_FLAG_TIMING) != 0;
  const bool gram_fp64 = (o.flags & ASCG_FLAG_GRAM_FP64) != 0;
  const bool gram_tc_force = (o.flags & ASCG_FLAG_GRAM_TC) != 0;
  const bool gram_mom = (o.flags & ASCG_FLAG_MOMENT_GRAM) != 0;
  const bool rec_fp64 = (o.flags & ASCG_FLAG_RECOVER_FP64) != 0;
  const bool stall_test = (o.flags & ASCG_FLAG_TEST_GRAM_STALL) != 0;
  if (timing) ASCG_CUDA(cudaEventRecord(w.ev[0], s));

  // ||b||, r_1 = b - A x_1, p_1 = r_1 (Alg. 1/4 first line). p = column 0 and
  // r = column 1 of the basis buffer.
  double* p = w.Y;
  double* r = w.Y + w.ldY;
  ASCG_CUDA(launch_dot(b, b, n, &w.scal[0], w.partials, w.counter, s));
  ASCG_CUDA(launch_residual(A, b, x, r, p, s));
  res->launches += 2;
  res->grid_reductions += 1;
  ASCG_CUDA(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  ASCG_CUDA(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(w.h_scal[0]);
  res->bnorm = bnorm;
  if (!(bnorm > 0.0) || !std::isfinite(bnorm)) {
    if (bnorm == 0.0) {  // b = 0: x = 0 is the solution
      ASCG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
      ASCG_CUDA(cudaStreamSynchronize(s));
      res->status = ASCG_OK;
      return ASCG_OK;
    }
    return fail(ASCG_ERR_INVALID, "b is not finite");
  }
  const double eps_star = o.eps_target * bnorm;
  int m = 0;
  ascg_status final_status = ASCG_OK;

  if (!sstep) {
    ASCG_TRY(run_classical(op, x, r, p, eps_star, bnorm, o.max_iters, 0, s, res, timing));
    m = w.h_cgs->iter;
    final_status = w.h_cgs->converged ? ASCG_OK : ASCG_NOT_CONVERGED;
    if (w.h_cgs->breakdown) {
      final_status = ASCG_ERR_BREAKDOWN;
      g_err = "breakdown: p^T A p was not positive and finite";
    }
    res->rel_res_updated = std::sqrt(std::max(w.h_cgs->rr, 0.0)) / bnorm;
  } else {
    double th[kMaxS], sg[kMaxS], gm[kMaxS];
    basis_params(o, th, sg, gm);
    bool done = false;
    // the residual history entry for i = 1 (m = 0)
    ASCG_CUDA(launch_dot(r, r, n, &w.scal[1], w.partials, w.counter, s));
    ASCG_CUDA(cudaMemcpyAsync(w.h_scal + 1, w.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    ASCG_CUDA(cudaStreamSynchronize(s));
    res->launches += 1;
    res->grid_reductions += 1;
    double r0 = std::sqrt(std::max(w.h_scal[1], 0.0));
    {
      const double rel = r0 / bnorm;
      ASCG_CUDA(cudaMemcpyAsync(w.res_hist, &rel, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    res->rel_res_updated = r0 / bnorm;
    if (r0 <= eps_star) done = true;
    if (!done && o.basis == ASCG_NEWTON) {
      // 2 s_max classical steps; the Ritz values of their Lanczos tridiagonal,
      // in Leja order, are the shifts theta_j of the Newton basis.
      const int nw = o.newton_warmup > 0 ? o.newton_warmup : 2 * o.s_max;
      const int cap = std::min(nw, o.max_iters);
      ASCG_TRY(run_classical(op, x, r, p, eps_star, bnorm, cap, 0, s, res, timing));
      m = w.h_cgs->iter;
      res->rel_res_updated = std::sqrt(std::max(w.h_cgs->rr, 0.0)) / bnorm;
      if (w.h_cgs->converged) done = true;
      if (!done && w.h_cgs->breakdown) {
        done = true;
        final_status = ASCG_ERR_BREAKDOWN;
        g_err = "breakdown: p^T A p was not positive and finite in the Newton warm-up";
      }
      if (!done && m >= o.max_iters) {
        done = true;
        final_status = ASCG_NOT_CONVERGED;
      }
      if (!done) {
        if (m < o.s_max) return fail(ASCG_ERR_BREAKDOWN, "Newton warm-up ended early");
        ASCG_CUDA(launch_newton_shifts(w.ab_hist, w.ab_hist + w.ab_cap, m, w.shifts, s));
        res->launches += 1;
        double sh[32];
        ASCG_CUDA(cudaMemcpyAsync(sh, w.shifts, m * sizeof(double), cudaMemcpyDeviceToHost, s));
        ASCG_CUDA(cudaStreamSynchronize(s));
        for (int j = 0; j < kMaxS; ++j) th[j] = j < o.s_max ? sh[j] : 0.0;
      }
    }
    double hp[3 * kMaxS];
    std::memcpy(hp, th, sizeof(th));
    std::memcpy(hp + kMaxS, sg, sizeof(sg));
    std::memcpy(hp + 2 * kMaxS, gm, sizeof(gm));
    ASCG_CUDA(cudaMemcpyAsync(w.params, hp, sizeof(hp), cudaMemcpyHostToDevice, s));
    StepOp steps[kMaxS];
    if (!done) {
      int nl = 0;
      ASCG_TRY(prepare_steps(op, th, sg, gm, o.s_max, w.dtils, w.oscaled, steps, s, &nl));
      res->launches += nl;
    }
    const DevSplit Asplit = op->split();
    const double sqrt_n = std::sqrt((double)n);
    // ASCG_FLAG_C_FORMULA: c_{k,j} = 6 N_k j kappa(A), N_k = 7 + 2 N_A + 14 ||B_k|| / ||A||
    double c_step_of[kMaxS + 1] = {};
    if (o.flags & ASCG_FLAG_C_FORMULA)
      for (int sb = 1; sb <= o.s_max; ++sb)
        c_step_of[sb] = 6.0 * (7.0 + 2.0 * op->max_row_nnz + 14.0 * norm_B(sb, th, sg, gm) / o.norm_A) * o.kappa_A;
    int k = 0, s_prev = 0;
    int nb_info = 0;
    // Blocks alternate between two basis buffers. Block k recovers r and p
    // into the other buffer; its x += Y x' waits until block k+1's Gram is
    // done and then runs on the side stream beside block k+1's condition
    // estimates and controller, which leave most SMs idle. Block k+1's own
    // recovery overwrites columns 0 and 1 of block k's buffer, so it waits for
    // that update first.
    double* Ybuf[2] = {w.Y, w.Y2};
    double* cbuf[2] = {w.coords, w.coords + 3 * kMaxW};
    bool x_out[2] = {false, false};  // an x update reading buffer b is queued on the side stream
    // the x update runs beside the controller, whose CTAs (one per condition
    // estimate plus one for the steps: s_max + 1 at most) keep their SMs; the
    // x update takes every other SM, one CTA each
    const int x_ctas = std::max(1, gram_grid() - (o.method == ASCG_ADAPTIVE ? o.s_max + 1 : 1));
    // Block j uses basis buffer j & 1, coordinates cbuf[j & 1] and record slot
    // j % kRing (device w.bst[slot], pinned host w.h_bst[slot] going in and
    // w.h_bst[kRing + slot] coming back). When block j+1's basis size does not
    // depend on block j's outcome (Alg. 2, Alg. 3, and Alg. 4 with f >= s_max - 1,
    // where sbar_k = s_max for every k >= 1), block j+1 is enqueued before the
    // host reads block j's record: the GPU never waits for the host between
    // blocks. A device kernel carries m, k and the iteration budget from
    // block to block and clears block j+1's flag when block j ended the solve;
    // every kernel of a block then returns at once.
    const bool ahead = o.method == ASCG_FIXED_S || o.method == ASCG_VARIABLE_S ||
                       (o.method == ASCG_ADAPTIVE && o.f >= o.s_max - 1);
    int wb_of[kRing] = {};
    bool rec_tc_of[kRing] = {};  // the block's recovery ran on the tensor cores (x included)
    int sbar_of[kRing] = {};
    auto enqueue = [&](int j, int sbar) -> ascg_status {
      const int slot = j % kRing, cur = j & 1;
      const int wb = 2 * sbar + 1;
      double* const Yc = Ybuf[cur];
      BlockState* const dst = w.bst + slot;
      const int* const gate = &dst->active;
      BlockState& hb = w.h_bst[slot];
      std::memset(&hb, 0, sizeof(hb));
      hb.sbar = sbar;
      hb.method = o.method;
      hb.check_in_loop = o.check_in_loop;
      hb.max_steps = o.max_iters - m;  // block 0; later blocks: set on the device
      hb.m = m;
      hb.k = j;
      hb.eps_star = eps_star;
      hb.c = o.c;
      hb.c_step = c_step_of[sbar];
      hb.c_smax = o.s_max;
      hb.bnorm = bnorm;
      hb.sqrt_n = sqrt_n;
      hb.active = 1;
      ASCG_CUDA(cudaMemcpyAsync(dst, &hb, sizeof(BlockState), cudaMemcpyHostToDevice, s));
      if (j > 0) {
        ASCG_CUDA(launch_block_advance(w.bst + (j - 1) % kRing, dst, o.max_iters, s));
        res->launches += 1;
      }
      wb_of[slot] = wb;
      sbar_of[slot] = sbar;
      cudaEvent_t* ev = w.ev_blk[slot];
      // matrix powers: P columns 1..sbar, R columns 1..sbar-1 (eq. cg-krylovbasis)
      if (timing) ASCG_CUDA(cudaEventRecord(ev[0], s));
      // The tensor cores take the Gram when its FP64 work, n w(w+1)/2 products,
      // is large enough to pay for the kernel's fixed cost (tensor memory,
      // barriers, pipeline fill: about 40 us on GB300, against about 1 us per
      // 2^20 products in FP64), or when ASCG_FLAG_GRAM_TC asks for them. The
      // matrix powers steps then also record each column's largest exponent.
      const bool tc_big = gram_tc_force || (double)n * wb * (wb + 1) / 2.0 >= kTcSolveProducts;
      const bool tc_gram = !gram_fp64 && !gram_mom && tc_big && gram_tc_applies(wb) && gram_tc_aligned(Yc, w.ldY) &&
                           gram_tc_fits(n);
      for (int q = 0; q < sbar; ++q) {
        ASCG_CUDA(launch_mpk_split_step(Asplit, steps[q], Yc, w.ldY, q, 1, q < sbar - 1,
                                        tc_gram ? w.emax_part : nullptr, w.emax_ld, s, gate));
      }
      if (tc_gram) {
        ASCG_CUDA(launch_emax_reduce(w.emax_part, w.emax_ld, n, wb, w.expp, s, gate));
        res->launches += 1;
      }
      res->launches += sbar;
      if (timing) ASCG_CUDA(cudaEventRecord(ev[1], s));
      // Gram: the block's one grid-wide reduction
      int nparts = 0;
      if (gram_mom)
        ASCG_CUDA(launch_gram_moments(n, wb, Yc, w.ldY, w.partials, &nparts, s, gate));
      else
        ASCG_CUDA(launch_gram_any(n, wb, Yc, w.ldY, !tc_gram, w.expp, tc_gram, w.partials, &nparts, s,
                                  &dst->status, stall_test && j == 0, gate));
      if (timing) ASCG_CUDA(cudaEventRecord(ev[2], s));
      if (gram_mom)
        ASCG_CUDA(launch_gram_moment_finalize(wb, w.partials, nparts, w.G, s, gate));
      else
        ASCG_CUDA(launch_gram_finalize(wb, w.partials, nparts, w.G, s, gate));
      res->launches += 2;
      if (j > 0 && !rec_tc_of[(j - 1) % kRing]) {  // block j-1's x += Y x', beside this block's controller
        const int ps = (j - 1) % kRing;
        ASCG_CUDA(cudaEventRecord(w.ev_gram, s));
        ASCG_CUDA(cudaStreamWaitEvent(w.side, w.ev_gram, 0));
        ASCG_CUDA(launch_recover_x(n, wb_of[ps], Ybuf[cur ^ 1], w.ldY, cbuf[cur ^ 1], x, x_ctas, w.side,
                                   &w.bst[ps].active));
        ASCG_CUDA(cudaEventRecord(w.ev_x[cur ^ 1], w.side));
        x_out[cur ^ 1] = true;
        res->launches += 1;
      }
      ASCG_CUDA(launch_block_ctrl(w.G, w.params, w.params + kMaxS, w.params + 2 * kMaxS, dst, sbar,
                                  o.method == ASCG_ADAPTIVE, cbuf[cur], nullptr, w.res_hist, w.res_cap, w.ab_hist,
                                  w.ab_cap, w.spec, w.counter + 1, s));
      if (timing) ASCG_CUDA(cudaEventRecord(ev[3], s));
      // r and p into columns 1 and 0 of the other buffer, once the update that reads it is done
      if (x_out[cur ^ 1]) {
        ASCG_CUDA(cudaStreamWaitEvent(s, w.ev_x[cur ^ 1], 0));
        x_out[cur ^ 1] = false;
      }
      // A block whose Gram took the tensor cores recovers x, r and p on them in
      // one pass (its column exponents are in w.expp); otherwise r and p here
      // and x during the next block.
      const bool tc_rec = tc_gram && !rec_fp64;
      rec_tc_of[slot] = tc_rec;
      if (tc_rec)
        ASCG_CUDA(launch_recover_tc(n, wb, Yc, w.ldY, w.expp, cbuf[cur], x, Ybuf[cur ^ 1] + w.ldY, Ybuf[cur ^ 1], s,
                                    &dst->status, gate));
      else
        ASCG_CUDA(launch_recover_rp(n, wb, Yc, w.ldY, cbuf[cur], Ybuf[cur ^ 1] + w.ldY, Ybuf[cur ^ 1], s, gate));
      res->launches += 2;
      if (timing) ASCG_CUDA(cudaEventRecord(ev[4], s));
      ASCG_CUDA(cudaMemcpyAsync(w.h_bst + kRing + slot, dst, sizeof(BlockState), cudaMemcpyDeviceToHost, s));
      ASCG_CUDA(cudaEventRecord(w.ev_rec[slot], s));
      return ASCG_OK;
    };
    // block sizes known without the previous block's outcome
    auto sbar_ahead = [&](int j, int* sbar) {
      if (!ahead || j == 0) return false;
      *sbar = o.method == ASCG_ADAPTIVE ? o.s_max : block_sbar(o, j, 1);
      return true;
    };
    int enq = 0;  // blocks enqueued
    if (!done) {
      ASCG_TRY(enqueue(0, block_sbar(o, 0, 0)));
      enq = 1;
    }
    while (!done) {
      int sb_next = 0;
      if (enq == k + 1 && sbar_ahead(k + 1, &sb_next)) {
        ASCG_TRY(enqueue(k + 1, sb_next));
        enq = k + 2;
      }
      const int slot = k % kRing;
      const int sbar = sbar_of[slot];
      const int wb = wb_of[slot];
      ASCG_CUDA(cudaEventSynchronize(w.ev_rec[slot]));
      if (timing) {
        cudaEvent_t* ev = w.ev_blk[slot];
        float a = 0.f, b2 = 0.f, c2 = 0.f, d2 = 0.f;
        ASCG_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
        ASCG_CUDA(cudaEventElapsedTime(&b2, ev[1], ev[2]));
        ASCG_CUDA(cudaEventElapsedTime(&c2, ev[2], ev[3]));
        ASCG_CUDA(cudaEventElapsedTime(&d2, ev[3], ev[4]));
        res->t_mpk_ms += a;
        res->t_gram_ms += b2;
        res->t_ctrl_ms += c2;
        res->t_recover_ms += d2;
        res->gram_launches += 1;
        res->mpk_launches += sbar;
        res->gram_flops += 2.0 * (gram_mom ? 3.0 * (wb - 1) : (double)wb * (wb + 1) / 2.0) * (double)n;
        res->gram_bytes += 8.0 * (double)wb * (double)n;
        // per step and chain: the SpMV's 2 nnz flops (the folded shift, scale and
        // sigma terms are not counted)
        const double nchains = 2.0 * sbar - 1.0;
        res->mpk_flops += nchains * 2.0 * (double)op->nnz;
        res->mpk_bytes += (double)sbar * (12.0 * op->nnz + 4.0 * (n + 1)) + nchains * 16.0 * n + 8.0 * n;
        // the timed part: r = Y r', p = Y p', and x += Y x' on the tensor-core
        // path (the FP64 path's x update runs later, on the side stream)
        const double nvec = rec_tc_of[slot] ? 3.0 : 2.0;
        res->recover_flops += 2.0 * nvec * wb * (double)n;
        res->recover_bytes += 8.0 * wb * (double)n + (rec_tc_of[slot] ? 32.0 : 16.0) * n;
      }
      const BlockState& out = w.h_bst[kRing + slot];
      res->grid_reductions += 1;
      if (o.block_hist && nb_info < o.block_hist_cap) {
        ascg_block_info& bi = o.block_hist[nb_info];
        std::memset(&bi, 0, sizeof(bi));
        bi.sbar = sbar;
        bi.stilde = out.stilde;
        bi.s_k = out.s_k;
        bi.stop = out.stop;
        bi.m = m;
        bi.rnorm = out.rnorm;
        bi.threshold = out.threshold;
        bi.gamma = out.gamma;
        for (int i = 0; i < sbar; ++i) bi.sqrt_kappa[i] = o.method == ASCG_ADAPTIVE ? out.sqrt_kappa[i] : 0.0;
      }
      ++nb_info;
      res->wasted_vecs += 2 * (sbar - out.s_k);
      if (out.status == ASCG_ERR_TIMEOUT) {
        // a bounded wait of the tensor-core Gram ran out; its CTA gave up
        // cleanly and the block's G is NaN, so no step was taken
        final_status = ASCG_ERR_TIMEOUT;
        g_err = "timeout: a bounded wait of the tensor-core Gram ran out";
        break;
      }
      if (out.s_k == 0) {
        final_status = ASCG_ERR_BREAKDOWN;
        g_err = "breakdown: a block could not take an inner step";
        break;
      }
      res->rel_res_updated = out.rel_res;
      m += out.s_k;
      s_prev = out.s_k;
      ++k;
      if (out.converged) break;
      if (m >= o.max_iters) {
        final_status = ASCG_NOT_CONVERGED;
        break;
      }
      if (enq == k) {
        ASCG_TRY(enqueue(k, block_sbar(o, k, s_prev)));
        enq = k + 1;
      }
    }
    // the x update of the last block enqueued (block enq-1: it returns at once
    // if that block was enqueued ahead and had nothing to do), after any still
    // on the side stream
    for (int bq = 0; bq < 2; ++bq)
      if (x_out[bq]) ASCG_CUDA(cudaStreamWaitEvent(s, w.ev_x[bq], 0));
    if (enq > 0 && !rec_tc_of[(enq - 1) % kRing]) {
      const int last = enq - 1, ls = last % kRing;
      ASCG_CUDA(launch_recover_x(n, wb_of[ls], Ybuf[last & 1], w.ldY, cbuf[last & 1], x, x_ctas, s,
                                 &w.bst[ls].active));
      res->launches += 1;
    }
    res->blocks = k;
  }
  res->iters = m;
  // true residual ||b - A x|| / ||b||
  ASCG_CUDA(launch_residual(A, b, x, w.q, nullptr, s));
  ASCG_CUDA(launch_dot(w.q, w.q, n, &w.scal[2], w.partials, w.counter, s));
  res->launches += 2;
  if (timing) ASCG_CUDA(cudaEventRecord(w.ev[7], s));
  ASCG_CUDA(cudaMemcpyAsync(w.h_scal + 2, w.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  ASCG_CUDA(cudaStreamSynchronize(s));
  res->rel_res_true = std::sqrt(w.h_scal[2]) / bnorm;
  if (timing) {
    float ms = 0.f;
    ASCG_CUDA(cudaEventElapsedTime(&ms, w.ev[0], w.ev[7]));
    res->t_total_ms = ms;
  }
  // histories to the caller
  const int nh = m + 1;
  if (o.res_hist && o.res_hist_cap > 0)
    ASCG_CUDA(cudaMemcpy(o.res_hist, w.res_hist, sizeof(double) * std::min(nh, o.res_hist_cap),
                         cudaMemcpyDeviceToHost));
  if (o.alpha_hist && o.coef_hist_cap > 0 && m > 0)
    ASCG_CUDA(cudaMemcpy(o.alpha_hist, w.ab_hist, sizeof(double) * std::min(m, o.coef_hist_cap),
                         cudaMemcpyDeviceToHost));
  if (o.beta_hist && o.coef_hist_cap > 0 && m > 0)
    ASCG_CUDA(cudaMemcpy(o.beta_hist, w.ab_hist + w.ab_cap, sizeof(double) * std::min(m, o.coef_hist_cap),
                         cudaMemcpyDeviceToHost));
  res->status = final_status;
  return final_status;
}


void zero_result(ascg_result* r) {
  if (r) std::memset(r, 0, sizeof(*r));
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

ascg_status ascg_options_default(ascg_options* o) {
  if (!o) return fail(ASCG_ERR_INVALID, "options pointer is NULL");
  std::memset(o, 0, sizeof(*o));
  o->method = ASCG_ADAPTIVE;
  o->basis = ASCG_MONOMIAL;
  o->s_max = 8;
  o->s0 = 8;
  o->f = 8;
  o->newton_warmup = 0;
  o->max_iters = 100000;
  o->check_in_loop = 1;
  o->eps_target = 1e-10;
  o->c = 1.0;
  return ASCG_OK;
}

ascg_status ascg_op_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
                               const double* val, int on_device, ascg_op* out) {
  g_err.clear();
  if (!out) return fail(ASCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1) return fail(ASCG_ERR_INVALID, "n must be >= 1");
  if (nnz < 0 || nnz >= (int64_t)1 << 31) return fail(ASCG_ERR_INVALID, "nnz must be in [0, 2^31)");
  if (n >= (int64_t)1 << 31) return fail(ASCG_ERR_INVALID, "n must be < 2^31");
  if (!rowptr || (nnz > 0 && (!colind || !val))) return fail(ASCG_ERR_INVALID, "NULL CSR array");
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
  const int64_t* hrp = rowptr;
  const int32_t* hci = colind;
  const double* hva = val;
  if (on_device) {
    rp.resize(n + 1);
    ci.resize(nnz);
    va.resize(nnz);
    ASCG_CUDA(cudaMemcpy(rp.data(), rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
    if (nnz) {
      ASCG_CUDA(cudaMemcpy(ci.data(), colind, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
      ASCG_CUDA(cudaMemcpy(va.data(), val, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    }
    hrp = rp.data();
    hci = ci.data();
    hva = va.data();
  }
  if (hrp[0] != 0 || hrp[n] != nnz) return fail(ASCG_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] = nnz");
  for (int64_t i = 0; i < n; ++i)  // all of rowptr first, so rows below index only [0, nnz)
    if (hrp[i + 1] < hrp[i] || hrp[i + 1] > nnz) return fail(ASCG_ERR_INVALID, "rowptr is not non-decreasing");
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t k = hrp[i]; k < hrp[i + 1]; ++k) {
      const int32_t c = hci[k];
      if (c < 0 || c >= n) return fail(ASCG_ERR_INVALID, "column index out of range");
      if (!std::isfinite(hva[k])) return fail(ASCG_ERR_INVALID, "non-finite matrix entry");
      if (c == i) {
        if (!(hva[k] > 0.0)) return fail(ASCG_ERR_NOT_SPD, "diagonal entry is not positive");
        diag = true;
      }
    }
    if (!diag) return fail(ASCG_ERR_NOT_SPD, "a row has no diagonal entry");
  }
  std::vector<double> dg(n, 0.0);
  const HostSell ha = build_sell(n, hrp, hci, hva, false, nullptr);
  const HostSell ho = build_sell(n, hrp, hci, hva, true, &dg);
  ascg_op op = new ascg_op_s();
  op->n = n;
  op->nnz = nnz;
  for (int64_t i = 0; i < n; ++i) op->max_row_nnz = std::max<int>(op->max_row_nnz, (int)(hrp[i + 1] - hrp[i]));
  op->o_len = (int64_t)ho.val.size();
  cudaGetDevice(&op->device);
  ascg_status st = upload(&op->a_ptr, ha.ptr);
  if (st == ASCG_OK) st = upload(&op->a_col, ha.col);
  if (st == ASCG_OK) st = upload(&op->a_val, ha.val);
  if (st == ASCG_OK) st = upload(&op->o_ptr, ho.ptr);
  if (st == ASCG_OK) st = upload(&op->o_col, ho.col);
  if (st == ASCG_OK) st = upload(&op->o_val, ho.val);
  if (st == ASCG_OK) st = upload(&op->diag, dg);
  if (st != ASCG_OK) {
    op->free_device();
    delete op;
    return st;
  }
  *out = op;
  return ASCG_OK;
}

ascg_status ascg_op_destroy(ascg_op op) {
  if (!op) return ASCG_OK;
  op->ws.release();
  op->free_device();
  delete op;
  return ASCG_OK;
}

ascg_status ascg_op_size(ascg_op op, int64_t* n, int64_t* nnz) {
  if (!op) return fail(ASCG_ERR_INVALID, "op is NULL");
  if (n) *n = op->n;
  if (nnz) *nnz = op->nnz;
  return ASCG_OK;
}

ascg_status ascg_solve(ascg_op op, const double* b, double* x, const ascg_options* opts, ascg_result* result,
                       void* cuda_stream) {
  g_err.clear();
  ascg_result local;
  ascg_result* res = result ? result : &local;
  zero_result(res);
  ascg_options o;
  if (opts)
    o = *opts;
  else
    ascg_options_default(&o);
  auto finish = [&](ascg_status st) {
    res->status = st;
    return st;
  };
  if (!op || !b || !x) return finish(fail(ASCG_ERR_INVALID, "NULL op, b or x"));
  ascg_status st = check_opts(o);
  if (st != ASCG_OK) return finish(st);
  st = solve_device(op, b, x, o, res, (cudaStream_t)cuda_stream);
  return finish(st);
}

ascg_status ascg_solve_host(ascg_op op, const double* b, double* x, const ascg_options* opts,
                            ascg_result* result, void* cuda_stream) {
  g_err.clear();
  ascg_result local;
  ascg_result* res = result ? result : &local;
  zero_result(res);
  auto finish = [&](ascg_status st) {
    res->status = st;
    return st;
  };
  if (!op || !b || !x) return finish(fail(ASCG_ERR_INVALID, "NULL op, b or x"));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Workspace& w = op->ws;
  if (!w.b || w.n != op->n) {
    dev_free(w.b);
    dev_free(w.x);
    ascg_status a = dev_alloc(&w.b, (size_t)op->n);
    if (a == ASCG_OK) a = dev_alloc(&w.x, (size_t)op->n);
    if (a != ASCG_OK) return finish(a);
  }
  cudaError_t e = cudaMemcpyAsync(w.b, b, sizeof(double) * op->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.x, x, sizeof(double) * op->n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return finish(fail(ASCG_ERR_CUDA, std::string("H2D: ") + cudaGetErrorString(e)));
  // solve_device may reallocate the basis buffers but keeps b and x
  double* db = w.b;
  double* dx = w.x;
  ascg_status st = ascg_solve(op, db, dx, opts, res, cuda_stream);
  e = cudaMemcpyAsync(x, dx, sizeof(double) * op->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return finish(fail(ASCG_ERR_CUDA, std::string("D2H: ") + cudaGetErrorString(e)));
  return finish(st);
}

ascg_status ascg_solve_batch(int count, const ascg_op* ops, const double* const* b, double* const* x,
                             const double* eps_target, const ascg_options* opts, ascg_result* results,
                             void* cuda_stream) {
  g_err.clear();
  if (count < 1 || !ops || !b || !x || !opts) return fail(ASCG_ERR_INVALID, "bad argument");
  const ascg_options o = *opts;
  ASCG_TRY(check_opts(o));
  if (o.method == ASCG_CLASSICAL) return fail(ASCG_ERR_INVALID, "batched solves run an s-step method");
  if (o.flags & ASCG_FLAG_C_FORMULA)
    return fail(ASCG_ERR_INVALID, "ASCG_FLAG_C_FORMULA needs one system's kappa(A) and ||A||: use ascg_solve");
  if (o.basis != ASCG_MONOMIAL) return fail(ASCG_ERR_INVALID, "batched solves use the monomial basis");
  if ((o.res_hist && o.res_hist_cap < 1) || (o.block_hist && o.block_hist_cap < 1))
    return fail(ASCG_ERR_INVALID, "history capacities must be >= 1");
  try {
    return lockstep_solve_batch(count, ops, b, x, eps_target, o, results, (cudaStream_t)cuda_stream);
  } catch (const std::bad_alloc&) {
    return fail(ASCG_ERR_OOM, "host allocation failed");
  }
}

ascg_status ascg_spmv(ascg_op op, const double* x, double* y, void* cuda_stream) {
  g_err.clear();
  if (!op || !x || !y) return fail(ASCG_ERR_INVALID, "NULL argument");
  ASCG_CUDA(launch_spmv(op->sell(), x, y, (cudaStream_t)cuda_stream));
  return ASCG_OK;
}

ascg_status ascg_matrix_powers(ascg_op op, int s, const double* theta, const double* sigma, const double* gamma,
                               double* Y, int64_t ldY, void* cuda_stream) {
  g_err.clear();
  if (!op || !theta || !sigma || !gamma || !Y) return fail(ASCG_ERR_INVALID, "NULL argument");
  if (s < 1 || s > ASCG_MAX_S) return fail(ASCG_ERR_INVALID, "s must be in 1..16");
  if (ldY < op->n) return fail(ASCG_ERR_INVALID, "ldY < n");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* dtils = nullptr;
  double* osc[2] = {nullptr, nullptr};
  ascg_status rs = dev_alloc(&dtils, (size_t)s * op->n);
  if (rs == ASCG_OK) rs = dev_alloc(&osc[0], (size_t)op->o_len);
  if (rs == ASCG_OK) rs = dev_alloc(&osc[1], (size_t)op->o_len);
  StepOp steps[kMaxS];
  int nl = 0;
  if (rs == ASCG_OK) rs = prepare_steps(op, theta, sigma, gamma, s, dtils, osc, steps, st, &nl);
  cudaError_t e = cudaSuccess;
  for (int j = 0; rs == ASCG_OK && j < s && e == cudaSuccess; ++j)
    e = launch_mpk_split_step(op->split(), steps[j], Y, ldY, j, 1, j < s - 1, nullptr, 0, st);
  if (e == cudaSuccess && rs == ASCG_OK) e = cudaStreamSynchronize(st);
  cudaFree(dtils);
  cudaFree(osc[0]);
  cudaFree(osc[1]);
  if (rs != ASCG_OK) return rs;
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("matrix powers: ") + cudaGetErrorString(e));
  return ASCG_OK;
}

ascg_status ascg_gram(int64_t n, int w, const double* Y, int64_t ldY, double* G, void* cuda_stream) {
  g_err.clear();
  if (!Y || !G || n < 1 || w < 1 || w > ASCG_MAX_W || ldY < n) return fail(ASCG_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* partials = nullptr;
  int* expp = nullptr;
  int parts = 0;
  ASCG_TRY(dev_alloc(&partials, (size_t)gram_grid() * kMaxPairs));
  // column exponents, then one error word of the tensor-core kernel
  const size_t nexp = (size_t)gram_grid() * kMaxW;
  ascg_status rs = dev_alloc(&expp, nexp + 1);
  if (rs != ASCG_OK) {
    cudaFree(partials);
    return rs;
  }
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(expp + nexp, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_gram_any(n, w, Y, ldY, false, expp, false, partials, &parts, s, expp + nexp);
  if (e == cudaSuccess) e = launch_gram_finalize(w, partials, parts, G, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, expp + nexp, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(partials);
  cudaFree(expp);
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("gram: ") + cudaGetErrorString(e));
  if (herr == ASCG_ERR_TIMEOUT) return fail(ASCG_ERR_TIMEOUT, "gram: a bounded wait of the tensor-core kernel ran out");
  return ASCG_OK;
}

ascg_status ascg_gram_moments(int64_t n, int s_, const double* Y, int64_t ldY, double* G, void* cuda_stream) {
  g_err.clear();
  if (!Y || !G || n < 1 || s_ < 1 || s_ > ASCG_MAX_S || ldY < n) return fail(ASCG_ERR_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* partials = nullptr;
  ASCG_TRY(dev_alloc(&partials, (size_t)gram_grid() * kMomSlots));
  int parts = 0;
  const int w = 2 * s_ + 1;
  cudaError_t e = launch_gram_moments(n, w, Y, ldY, partials, &parts, s);
  if (e == cudaSuccess) e = launch_gram_moment_finalize(w, partials, parts, G, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(partials);
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("gram moments: ") + cudaGetErrorString(e));
  return ASCG_OK;
}

ascg_status ascg_block_step(int sbar, const double* G, int method, const double* theta, const double* sigma,
                            const double* gamma, int64_t nrows, double eps_star, double c, int check_in_loop,
                            int max_steps, double bnorm, double* coords, ascg_block_info* info, double* hist,
                            void* cuda_stream) {
  g_err.clear();
  if (sbar < 1 || sbar > ASCG_MAX_S || !G || !theta || !sigma || !gamma || !coords || !info)
    return fail(ASCG_ERR_INVALID, "bad argument");
  if (method != ASCG_ADAPTIVE && method != ASCG_FIXED_S) return fail(ASCG_ERR_INVALID, "method");
  if (!(bnorm > 0.0) || !(c > 0.0) || nrows < 1 || max_steps < 0) return fail(ASCG_ERR_INVALID, "bad scalar");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  BlockState* bst = nullptr;
  double* dpar = nullptr;
  double* dhist = nullptr;
  double* dspec = nullptr;
  unsigned* dcnt = nullptr;
  ASCG_TRY(dev_alloc(&bst, 1));
  ascg_status st = dev_alloc(&dpar, 3 * kMaxS);
  if (st == ASCG_OK) st = dev_alloc(&dhist, 3 * kMaxS);
  if (st == ASCG_OK) st = dev_alloc(&dspec, kSpecDoubles);
  if (st == ASCG_OK) st = dev_alloc(&dcnt, 1);
  if (st != ASCG_OK) {
    cudaFree(bst);
    cudaFree(dpar);
    cudaFree(dhist);
    cudaFree(dspec);
    return st;
  }
  BlockState hb;
  std::memset(&hb, 0, sizeof(hb));
  hb.sbar = sbar;
  hb.method = method;
  hb.check_in_loop = check_in_loop;
  hb.max_steps = max_steps;
  hb.eps_star = eps_star;
  hb.c = c;
  hb.bnorm = bnorm;
  hb.sqrt_n = std::sqrt((double)nrows);
  hb.active = 1;
  double hp[3 * kMaxS];
  for (int j = 0; j < kMaxS; ++j) {
    hp[j] = j < sbar ? theta[j] : 0.0;
    hp[kMaxS + j] = j < sbar ? sigma[j] : 0.0;
    hp[2 * kMaxS + j] = j < sbar ? gamma[j] : 1.0;
  }
  double hh[3 * kMaxS];
  cudaError_t e = cudaMemcpyAsync(bst, &hb, sizeof(hb), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dpar, hp, sizeof(hp), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dcnt, 0, sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = launch_block_ctrl(G, dpar, dpar + kMaxS, dpar + 2 * kMaxS, bst, sbar, method == ASCG_ADAPTIVE, coords, dhist,
                          nullptr, 0, nullptr, 0, dspec, dcnt, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bst, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hh, dhist, sizeof(hh), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bst);
  cudaFree(dpar);
  cudaFree(dhist);
  cudaFree(dspec);
  cudaFree(dcnt);
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("block step: ") + cudaGetErrorString(e));
  std::memset(info, 0, sizeof(*info));
  info->sbar = sbar;
  info->stilde = hb.stilde;
  info->s_k = hb.s_k;
  info->stop = hb.stop;
  info->rnorm = hb.rnorm;
  info->threshold = hb.threshold;
  info->gamma = hb.gamma;
  for (int i = 0; i < sbar; ++i) info->sqrt_kappa[i] = method == ASCG_ADAPTIVE ? hb.sqrt_kappa[i] : 0.0;
  if (hist) std::memcpy(hist, hh, sizeof(double) * 3 * std::max(hb.s_k, 0));
  return ASCG_OK;
}

ascg_status ascg_recover(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* x, double* r,
                         double* p, void* cuda_stream) {
  g_err.clear();
  if (!Y || !coords || !x || !r || !p || n < 1 || w < 1 || w > ASCG_MAX_W || (w % 2) == 0 || ldY < n)
    return fail(ASCG_ERR_INVALID, "bad argument");
  ASCG_CUDA(launch_recover(n, w, Y, ldY, coords, x, r, p, (cudaStream_t)cuda_stream));
  return ASCG_OK;
}

ascg_status ascg_recover_tc(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* x,
                            double* r, double* p, void* cuda_stream) {
  g_err.clear();
  if (!Y || !coords || !x || !r || !p || n < 1 || n > 0x7fffffffll || w < kGramTcMinW || w > ASCG_MAX_W || ldY < n)
    return fail(ASCG_ERR_INVALID, "bad argument");
  if (!gram_tc_aligned(Y, ldY)) return fail(ASCG_ERR_INVALID, "Y must be 16-byte aligned with an even ldY");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* expp = nullptr;  // column exponents, then the kernel's error word
  ASCG_TRY(dev_alloc(&expp, (size_t)kMaxW + 1));
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(expp + kMaxW, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_col_exponents(n, w, Y, ldY, expp, s);
  if (e == cudaSuccess) e = launch_recover_tc(n, w, Y, ldY, expp, coords, x, r, p, s, expp + kMaxW);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, expp + kMaxW, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(expp);
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("recover_tc: ") + cudaGetErrorString(e));
  if (herr == ASCG_ERR_TIMEOUT) return fail(ASCG_ERR_TIMEOUT, "recover_tc: a bounded wait of the kernel ran out");
  return ASCG_OK;
}

ascg_status ascg_newton_shifts(const double* alphas, const double* betas, int k, int s, double* shifts,
                               void* cuda_stream) {
  g_err.clear();
  if (!alphas || (k > 1 && !betas) || !shifts || k < 1 || k > 32 || s < 1 || s > k)
    return fail(ASCG_ERR_INVALID, "bad argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* d = nullptr;
  ASCG_TRY(dev_alloc(&d, 96));
  double h[96] = {0};
  for (int j = 0; j < k; ++j) h[j] = alphas[j];
  for (int j = 0; j + 1 < k; ++j) h[32 + j] = betas[j];
  cudaError_t e = cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_newton_shifts(d, d + 32, k, d + 64, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d + 64, sizeof(double) * 32, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return fail(ASCG_ERR_CUDA, std::string("newton shifts: ") + cudaGetErrorString(e));
  for (int j = 0; j < s; ++j) shifts[j] = h[j];
  return ASCG_OK;
}

const char* ascg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace ascg {
void set_last_error(const std::string& msg) { g_err = msg; }

ascg_status check_options(const ascg_options& o) { return check_opts(o); }

ascg_status op_split_desc(ascg_op op, SysDesc* d, int* device) {
  if (!op) return fail(ASCG_ERR_INVALID, "op is NULL");
  std::memset(d, 0, sizeof(*d));
  d->n = op->n;
  d->o_ptr = op->o_ptr;
  d->o_col = op->o_col;
  d->o_val = op->o_val;
  d->diag = op->diag;
  *device = op->device;
  return ASCG_OK;
}
}  // namespace ascg
