// Lockstep engine: many independent SPD systems, each running Alg. 4 (or
// Alg. 2, Alg. 3) on its own operator, advance one block at a time together.
// It is the engine behind ascg_solve_batch and the solve server
// (ascg_server_*).
//
// Every system sits in a lane. A lane holds the system's descriptor (its
// operator, its basis Y, x and b), its controller state and its Gram and
// coordinate slots. One "super-block" runs one block of every active lane:
//   sbar_max matrix powers steps  (mpk_items_kernel, one row item per CTA)
//   Gram: tensor-core lanes in one launch (gram_tc_items_kernel), the other
//         lanes in one FP64 launch (gram_items_kernel), fixed-order sums
//   condition estimates and coordinate steps  (block_ctrl_kernel, per lane)
//   recovery  (recover_items_kernel)
// so a super-block is the same dozen launches for any number of systems,
// replayed as one captured graph while its shape stays the same. The host
// reads back one BlockState per lane, since the next block's basis size
// sbar_k = min(s_{k-1} + f, s_max) depends on it (Alg. 4).
//
// Each lane's arithmetic reads that lane's data only, in an order fixed by
// its own size: a system's result is bitwise the same alone and in any mix,
// whichever lane it lands in and whoever else is running.
//
// The bases are row ranges of one shared matrix (first-fit over 1024-row
// chunks) owned by the caller of the engine: admitting and retiring systems
// allocates nothing from CUDA, and one tensor map covers every lane.
//
// Gram schedule per lane, fixed by the lane's own size: lanes of at least
// tc_lane_rows rows (default 1024) with w >= 9 take the tensor-core launch;
// the others the FP64 one.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <string>
#include <vector>

#include "ascg_common.cuh"

namespace ascg {

// Defined in ascg_api.cu.
ascg_status check_options(const ascg_options& o);
ascg_status op_split_desc(ascg_op op, SysDesc* d, int* device);

namespace {

ascg_status lfail(ascg_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

#define LS_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return lfail(e_ == cudaErrorMemoryAllocation ? ASCG_ERR_OOM : ASCG_ERR_CUDA,             \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

#define LS_TRY(expr)                \
  do {                              \
    ascg_status s_ = (expr);        \
    if (s_ != ASCG_OK) return s_;   \
  } while (0)

template <class T>
ascg_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return lfail(ASCG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return ASCG_OK;
}

template <class T>
ascg_status halloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocHost((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return lfail(ASCG_ERR_OOM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  }
  return ASCG_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <class T>
void hfree(T*& p) {
  if (p) cudaFreeHost(p);
  p = nullptr;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// The bases of all held systems are row ranges of one matrix of wcols
// columns and R rows (column-major, leading dimension R): a system of n rows
// holds rows [r0, r0 + round_up(n, 1024)) of every column. One leading
// dimension for all lets one tensor map, and so one tensor-core Gram launch,
// cover every system. First-fit over row ranges; a freed range merges with
// its free neighbours. Ranges start and end on 1024-row boundaries, the
// chunks of the tensor-core Gram.
class Arena {
 public:
  static constexpr int64_t kRowAlign = 1024;
  ~Arena() { dfree(base_); }
  ascg_status init(int wcols, int64_t rows) {
    wcols_ = wcols;
    rows_ = rows > 0 ? round_up(rows, kRowAlign) : 0;
    if (rows_ > 0) {
      LS_TRY(dalloc(&base_, (size_t)wcols * rows_));
      free_[0] = rows_;
    }
    return ASCG_OK;
  }
  static int64_t rounded(int64_t n) { return round_up(n > 0 ? n : 1, kRowAlign); }
  bool take(int64_t n, int64_t* r0) {
    const int64_t need = rounded(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      *r0 = it->first;
      const int64_t rest = it->second - need, next = it->first + need;
      free_.erase(it);
      if (rest) free_[next] = rest;
      live_[*r0] = need;
      used_ += need;
      return true;
    }
    return false;
  }
  void give(int64_t r0) {
    auto l = live_.find(r0);
    if (l == live_.end()) return;
    int64_t len = l->second;
    live_.erase(l);
    used_ -= len;
    auto nx = free_.lower_bound(r0);
    if (nx != free_.end() && nx->first == r0 + len) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == r0) {
        pv->second += len;
        return;
      }
    }
    free_[r0] = len;
  }
  double* row(int64_t r0) const { return base_ + r0; }  // column 0 at row r0
  double* base() const { return base_; }
  int64_t ld() const { return rows_; }
  size_t bytes_total() const { return (size_t)wcols_ * rows_ * sizeof(double); }
  size_t bytes_used() const { return (size_t)wcols_ * used_ * sizeof(double); }

 private:
  double* base_ = nullptr;
  int wcols_ = 0;
  int64_t rows_ = 0, used_ = 0;
  std::map<int64_t, int64_t> free_, live_;  // first row -> rows
};

}  // namespace

// One system: what the caller handed in, and its progress.
struct LaneSys {
  ascg_op op = nullptr;
  SysDesc d{};
  double eps_target = 0.0;
  int64_t tag = 0;
  int64_t off = 0;   // first row of the system's range in the shared basis matrix
  size_t bytes = 0;  // basis bytes: (2 s_max + 1) 8 round_up(n, 1024)
  int m = 0, kb = 0, s_prev = 0, nb_info = 0, wasted = 0, sbar = 0;
  double bnorm = 0.0, eps_star = 0.0, rel_upd = 0.0, rnorm0 = 0.0, rel_true = 0.0;
  bool active = false, done = false;
  ascg_status status = ASCG_OK;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int64_t step_admit = 0, step_done = 0;
  cudaEvent_t ready = nullptr;  // server: b and x_1 written on the caller's stream
};

// Rows from which a lane's Gram runs on the tensor cores (all such lanes in
// one launch over the shared basis matrix) by default; below it the lane
// joins the FP64 item launch: a tensor-core lane reads whole 1024-row chunks,
// so a very small system costs less in FP64. The options can set another
// value (ascg_tune_gram_schedule measures one).
constexpr int64_t kTcLaneRows = (int64_t)1 << 10;

// A lane's running state on the device, for batched solves whose block loop
// runs on the GPU (Lockstep::run_on_device): the fields the host loop keeps
// in LaneSys, updated from each block's record exactly as complete_block
// does on the host.
struct LaneRun {
  int active, started, m, kb, s_prev, wasted, status, tc_ok;
  double rel_upd, eps_star, bnorm, sqrt_n;
};
struct LoopParams {
  int method, s_max, s0, f, check_in_loop, max_iters, seq_len, iter_cap;
  double c;
  const int* seq;
};

// One CTA: for every lane, the outcome of its last block (as complete_block),
// then its next block's record and table entries (as launch_block), or zeros
// when it has finished; then the loop's condition: another block while any
// lane runs and fewer than iter_cap blocks have been taken. Every block takes
// at least one step of every running lane or ends it, so the loop ends within
// max_iters + 1 blocks; iter_cap bounds it in any case.
__global__ void __launch_bounds__(1024) lanes_advance_kernel(BlockState* __restrict__ bst, LaneRun* __restrict__ run,
                                                             int nl, int* __restrict__ steps, int* __restrict__ w,
                                                             int* __restrict__ wi, int* __restrict__ wtc,
                                                             const LoopParams P, int* __restrict__ iter,
                                                             cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int q = threadIdx.x; q < nl; q += blockDim.x) {
    LaneRun R = run[q];
    BlockState& B = bst[q];
    if (R.active && R.started) {
      R.wasted += 2 * (B.sbar - B.s_k);
      if (B.s_k == 0) {
        R.status = ASCG_ERR_BREAKDOWN;
        R.active = 0;
      } else {
        R.rel_upd = B.rel_res;
        R.m += B.s_k;
        R.s_prev = B.s_k;
        ++R.kb;
        if (B.converged) {
          R.active = 0;
        } else if (R.m >= P.max_iters) {
          R.status = ASCG_NOT_CONVERGED;
          R.active = 0;
        }
      }
    }
    R.started = 1;
    int sb = 0;
    if (R.active) {
      if (P.method == ASCG_FIXED_S)
        sb = P.s_max;
      else if (P.method == ASCG_VARIABLE_S)
        sb = P.seq[R.kb < P.seq_len ? R.kb : P.seq_len - 1];
      else
        sb = R.kb == 0 ? P.s0 : (R.s_prev + P.f < P.s_max ? R.s_prev + P.f : P.s_max);
      BlockState nb;
      memset(&nb, 0, sizeof(nb));
      nb.sbar = sb;
      nb.method = P.method;
      nb.check_in_loop = P.check_in_loop;
      nb.max_steps = P.max_iters - R.m;
      nb.m = R.m;
      nb.k = R.kb;
      nb.eps_star = R.eps_star;
      nb.c = P.c;
      nb.bnorm = R.bnorm;
      nb.sqrt_n = R.sqrt_n;
      nb.active = 1;
      B = nb;
    } else {
      B.active = 0;
    }
    const int ww = sb > 0 ? 2 * sb + 1 : 0;
    const bool tc = R.tc_ok && ww >= kGramTcMinW;
    steps[q] = sb;
    w[q] = ww;
    wi[q] = tc ? 0 : ww;
    wtc[q] = tc ? ww : 0;
    run[q] = R;
    any |= R.active;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int it = ++*iter;
    cudaGraphSetConditional(cond, (any && it <= P.iter_cap) ? 1u : 0u);
  }
}

class Lockstep {
 public:
  ~Lockstep() { release(); }

  // lanes: most systems held at once; gitems, ritems: initial Gram and row
  // item capacities (they grow on demand); rcap, abcap: history capacities
  // per lane (0: none). All work is ordered on stream s.
  ascg_status init(const ascg_options& o, int lanes, int64_t gitems, int64_t ritems, int rcap, int abcap,
                   double* basis, int64_t basis_ld, cudaStream_t s) {
    o_ = o;
    ybase_ = basis;
    yld_ = basis_ld;
    if (o.method == ASCG_VARIABLE_S) {  // keep a copy: the caller's array may go
      seq_.assign(o.s_seq, o.s_seq + o.s_seq_len);
      o_.s_seq = seq_.data();
    }
    s_ = s;
    lanes_ = lanes;
    rcap_ = rcap;
    abcap_ = abcap;
    wcols_ = 2 * o.s_max + 1;
    moments_ = (o.flags & ASCG_FLAG_MOMENT_GRAM) != 0;
    tc_rows_ = o.tc_lane_rows == 0 ? kTcLaneRows : (o.tc_lane_rows < 0 ? INT64_MAX : o.tc_lane_rows);
    tcnp_ = wcols_ * (wcols_ + 1) / 2;
    npw_ = (int)partials_per_item(o.s_max, moments_);
    LS_TRY(dalloc(&d_desc_, lanes));
    LS_TRY(dalloc(&d_bst_, lanes));
    LS_TRY(dalloc(&d_G_, (size_t)lanes * kGStride));
    LS_TRY(dalloc(&d_coords_, (size_t)lanes * kCStride));
    LS_TRY(dalloc(&d_int_, (size_t)kIntArrays * lanes));
    LS_TRY(dalloc(&d_sums_, (size_t)2 * lanes));
    LS_TRY(dalloc(&d_params_, (size_t)3 * kMaxS));
    LS_TRY(dalloc(&d_spec_, (size_t)lanes * kSpecDoubles));
    LS_TRY(dalloc(&d_emax_, (size_t)lanes * kMaxW));
    LS_TRY(dalloc(&d_tickets_, (size_t)lanes));
    if (rcap_) LS_TRY(dalloc(&d_res_hist_, (size_t)lanes * rcap_));
    if (abcap_) LS_TRY(dalloc(&d_ab_hist_, (size_t)lanes * 2 * abcap_));
    LS_TRY(halloc(&h_desc_, lanes));
    LS_TRY(halloc(&h_bst_, lanes));
    LS_TRY(halloc(&h_int_, (size_t)kIntArrays * lanes));
    LS_TRY(halloc(&h_sums_, (size_t)2 * lanes));
    LS_TRY(grow_items(ritems, gitems));
    std::memset(h_desc_, 0, sizeof(SysDesc) * lanes);
    std::memset(h_bst_, 0, sizeof(BlockState) * lanes);
    std::memset(h_int_, 0, sizeof(int) * kIntArrays * lanes);
    LS_CUDA(cudaMemsetAsync(d_coords_, 0, sizeof(double) * lanes * kCStride, s_));
    LS_CUDA(cudaMemsetAsync(d_bst_, 0, sizeof(BlockState) * lanes, s_));
    LS_CUDA(cudaMemsetAsync(d_tickets_, 0, sizeof(unsigned) * lanes, s_));
    double hp[3 * kMaxS];  // monomial basis: theta = sigma = 0, gamma = 1
    for (int j = 0; j < kMaxS; ++j) {
      hp[j] = 0.0;
      hp[kMaxS + j] = 0.0;
      hp[2 * kMaxS + j] = 1.0;
    }
    LS_CUDA(cudaMemcpyAsync(d_params_, hp, sizeof(hp), cudaMemcpyHostToDevice, s_));
    LS_CUDA(cudaStreamSynchronize(s_));
    lane_.assign(lanes, LaneSys());
    used_.assign(lanes, 0);
    return ASCG_OK;
  }

  static int64_t gram_items_of(int64_t n) { return (n + gram_item_rows(n) - 1) / gram_item_rows(n); }
  static int64_t row_items_of(int64_t n) { return (n + kRowItem - 1) / kRowItem; }
  // Tensor-core Gram items: up to kTcItemRows rows (whole 1024-row chunks) each.
  static constexpr int64_t kTcItemRows = 8192;
  static int64_t tc_items_of(int64_t n) { return (Arena::rounded(n) + kTcItemRows - 1) / kTcItemRows; }
  // Basis bytes of a system of n rows: 2 s_max + 1 columns of round_up(n, 1024).
  static size_t basis_bytes(int s_max, int64_t n) {
    return (size_t)(2 * s_max + 1) * Arena::rounded(n) * sizeof(double);
  }
  // Gram partials per item: the pairs' upper triangle, or the moment slots.
  static int64_t partials_per_item(int s_max, bool moments) {
    const int64_t w = 2 * s_max + 1, np = w * (w + 1) / 2;
    return moments ? std::max<int64_t>(kMomSlots, np) : np;
  }
  // Device bytes one system holds while it runs: its basis and its Gram partials.
  static size_t footprint(int s_max, int64_t n, bool moments) {
    const int64_t w = 2 * s_max + 1;
    return basis_bytes(s_max, n) + (size_t)gram_items_of(n) * partials_per_item(s_max, moments) * sizeof(double) +
           (size_t)tc_items_of(n) * (w * (w + 1) / 2) * sizeof(double);
  }

  // Validates a system and fills its descriptor (all but Y).
  static ascg_status prepare(int s_max, ascg_op op, const double* b, double* x, double eps_target, int64_t tag,
                             LaneSys* out) {
    if (!op || !b || !x) return lfail(ASCG_ERR_INVALID, "op, b and x must be non-NULL");
    if (!(eps_target >= 0.0 && std::isfinite(eps_target)))
      return lfail(ASCG_ERR_INVALID, "eps_target must be finite and >= 0");
    int dev = 0, cur = 0;
    LS_TRY(op_split_desc(op, &out->d, &dev));
    LS_CUDA(cudaGetDevice(&cur));
    if (dev != cur) return lfail(ASCG_ERR_INVALID, "every operator must live on the current device");
    out->op = op;
    out->d.b = b;
    out->d.x = x;
    out->d.ldY = 0;  // set at admission: the shared basis matrix's leading dimension
    out->eps_target = eps_target;
    out->tag = tag;
    out->bytes = basis_bytes(s_max, out->d.n);
    return ASCG_OK;
  }

  int free_lanes() const { return lanes_ - nused_; }
  int active_lanes() const { return nused_; }

  // Admits systems whose basis Y the caller has placed (each into the lowest
  // free lane; the caller checks free_lanes()), computes ||b||, r_1 = b - A x_1
  // into Y columns 1 and 0 and ||r_1||. Systems that need no block (b = 0, r_1
  // already small enough, max_iters = 0) come out done. lanes_out: their lanes.
  ascg_status admit(const std::vector<LaneSys>& sys, std::vector<int>* lanes_out) {
    std::vector<int> fresh;
    for (const LaneSys& S : sys) {
      int q = 0;
      while (used_[q]) ++q;
      lane_[q] = S;
      used_[q] = 1;
      ++nused_;
      hi_ = std::max(hi_, q + 1);
      h_desc_[q] = S.d;
      fresh.push_back(q);
    }
    if (lanes_out) *lanes_out = fresh;
    if (fresh.empty()) return ASCG_OK;
    // rows n .. round_up(n, 1024) of every column are zero: the tensor-core
    // Gram reads whole 1024-row chunks
    for (int q : fresh) {
      const LaneSys& L = lane_[q];
      const int64_t pad = Arena::rounded(L.d.n) - L.d.n;
      if (pad > 0)
        LS_CUDA(cudaMemset2DAsync(L.d.Y + L.d.n, (size_t)L.d.ldY * sizeof(double), 0, (size_t)pad * sizeof(double),
                                  (size_t)wcols_, s_));
    }
    LS_TRY(rebuild_tables());
    int* h_sel = h_int_ + kSel * lanes_;
    int* h_list = h_int_ + kList * lanes_;
    for (int q = 0; q < hi_; ++q) h_sel[q] = 0;
    for (size_t i = 0; i < fresh.size(); ++i) {
      h_sel[fresh[i]] = 1;
      h_list[i] = fresh[i];
    }
    int* d_sel = d_int_ + kSel * lanes_;
    int* d_list = d_int_ + kList * lanes_;
    LS_CUDA(cudaMemcpyAsync(d_sel, h_sel, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
    LS_CUDA(cudaMemcpyAsync(d_list, h_list, sizeof(int) * fresh.size(), cudaMemcpyHostToDevice, s_));
    LS_CUDA(launch_seg_sumsq(d_desc_, d_list, (int)fresh.size(), 0, d_sums_, s_));
    LS_CUDA(launch_residual_items(d_desc_, d_ritems_, (int)ritems_.size(), d_sel, 0, s_));
    LS_CUDA(launch_seg_sumsq(d_desc_, d_list, (int)fresh.size(), 1, d_sums_ + lanes_, s_));
    LS_CUDA(cudaMemcpyAsync(h_sums_, d_sums_, sizeof(double) * 2 * lanes_, cudaMemcpyDeviceToHost, s_));
    LS_CUDA(cudaStreamSynchronize(s_));
    launches_ += 3;
    for (int q : fresh) {
      LaneSys& L = lane_[q];
      L.bnorm = std::sqrt(h_sums_[q]);
      L.rnorm0 = std::sqrt(std::max(h_sums_[lanes_ + q], 0.0));
      if (!std::isfinite(L.bnorm) || !std::isfinite(L.rnorm0)) {
        L.status = ASCG_ERR_INVALID;
        L.done = true;
        continue;
      }
      L.eps_star = L.eps_target * L.bnorm;
      L.rel_upd = L.bnorm > 0.0 ? L.rnorm0 / L.bnorm : 0.0;
      const bool need = L.bnorm > 0.0 && L.rnorm0 > L.eps_star;
      L.active = need && o_.max_iters > 0;
      if (need && o_.max_iters == 0) L.status = ASCG_NOT_CONVERGED;
      L.done = !L.active;
      if (rcap_) {
        const double rel = L.rel_upd;
        LS_CUDA(cudaMemcpyAsync(d_res_hist_ + (int64_t)q * rcap_, &rel, sizeof(double), cudaMemcpyHostToDevice, s_));
      }
    }
    return ASCG_OK;
  }

  bool any_active() const {
    for (int q = 0; q < hi_; ++q)
      if (used_[q] && lane_[q].active) return true;
    return false;
  }

  // Enqueues one block of every active lane and the read-back of their
  // states; *launched = false when no lane is active. The host must call
  // complete_block() once the stream has reached this point.
  ascg_status launch_block(bool* launched) {
    *launched = false;
    int* h_steps = h_int_ + kSteps * lanes_;
    int* h_w = h_int_ + kW * lanes_;
    int* h_wi = h_int_ + kWItems * lanes_;
    int* h_wtc = h_int_ + kWTc * lanes_;
    int max_sbar = 0, n_tc = 0;
    for (int q = 0; q < hi_; ++q) {
      BlockState& hb = h_bst_[q];
      std::memset(&hb, 0, sizeof(hb));
      LaneSys& L = lane_[q];
      if (!used_[q] || !L.active) {
        h_steps[q] = 0;
        h_w[q] = 0;
        h_wi[q] = 0;
        h_wtc[q] = 0;
        continue;
      }
      const int sbar = block_sbar(o_, L.kb, L.s_prev);
      L.sbar = sbar;
      hb.sbar = sbar;
      hb.method = o_.method;
      hb.check_in_loop = o_.check_in_loop;
      hb.max_steps = o_.max_iters - L.m;
      hb.m = L.m;
      hb.k = L.kb;
      hb.eps_star = L.eps_star;
      hb.c = o_.c;
      hb.bnorm = L.bnorm;
      hb.sqrt_n = std::sqrt((double)L.d.n);
      hb.active = 1;
      const int w = 2 * sbar + 1;
      h_steps[q] = sbar;
      h_w[q] = w;
      const bool tc = !moments_ && L.d.n >= tc_rows_ && gram_tc_applies(w) && gram_tc_aligned(L.d.Y, L.d.ldY);
      h_wi[q] = tc ? 0 : w;
      h_wtc[q] = tc ? w : 0;
      n_tc += tc;
      max_sbar = std::max(max_sbar, sbar);
    }
    if (max_sbar == 0) return ASCG_OK;
    int* d_steps = d_int_ + kSteps * lanes_;
    int* d_w = d_int_ + kW * lanes_;
    int* d_wi = d_int_ + kWItems * lanes_;
    int* d_item0 = d_int_ + kItem0 * lanes_;
    int* d_nitems = d_int_ + kNItems * lanes_;
    int* d_wtc = d_int_ + kWTc * lanes_;
    int* d_tc0 = d_int_ + kTcItem0 * lanes_;
    int* d_tcn = d_int_ + kTcNItems * lanes_;
    const int nr = (int)ritems_.size(), ng = (int)gitems_.size(), nt = (int)titems_.size();
    const bool item_gram = n_tc < count_active();
    const bool tc_gram = n_tc > 0;
    const int Wb = 2 * max_sbar + 1;
    int nl = max_sbar + 2 + (item_gram ? 2 : 0) + (tc_gram ? 3 : 0);
    // The block's work: the state records in, the matrix powers steps, the
    // Gram (item launch and tensor-core lanes), the controller, the recovery,
    // the state records out. The host fills the pinned records before each
    // launch; a captured graph reads them when it runs.
    auto enqueue = [&]() -> ascg_status {
      LS_CUDA(cudaMemcpyAsync(d_bst_, h_bst_, sizeof(BlockState) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_steps, h_steps, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_w, h_w, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_wi, h_wi, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_wtc, h_wtc, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_TRY(block_kernels(max_sbar, item_gram, tc_gram));
      LS_CUDA(cudaMemcpyAsync(h_bst_, d_bst_, sizeof(BlockState) * hi_, cudaMemcpyDeviceToHost, s_));
      return ASCG_OK;
    };
    // A block of the same shape (tables, sbar_max, Gram schedule) replays a
    // captured graph: one launch instead of about twenty calls.
    const std::vector<int> key = {tables_version_, max_sbar, item_gram ? 1 : 0, tc_gram ? 1 : 0};
    cudaGraphExec_t exec = nullptr;
    auto it = graphs_.find(key);
    if (it != graphs_.end()) {
      exec = it->second;
    } else if (capturable_) {
      if (cudaStreamBeginCapture(s_, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const ascg_status st = enqueue();
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s_, &g);
        if (st != ASCG_OK || e != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          if (st != ASCG_OK) return st;
          return lfail(ASCG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        LS_CUDA(ei);
        if (graphs_.size() >= kMaxGraphs) drop_graphs();
        graphs_[key] = exec;
      } else {
        cudaGetLastError();
        capturable_ = false;  // e.g. the legacy default stream: launch directly
      }
    }
    if (exec)
      LS_CUDA(cudaGraphLaunch(exec, s_));
    else
      LS_TRY(enqueue());
    launches_ += nl;
    *launched = true;
    return ASCG_OK;
  }

  // The kernels of one block of every lane whose table entries (steps, w,
  // wi, wtc) and record are set: the matrix powers steps, the Gram (item
  // launch and tensor-core lanes), the controller, the recovery.
  ascg_status block_kernels(int max_sbar, bool item_gram, bool tc_gram) {
    int* d_steps = d_int_ + kSteps * lanes_;
    int* d_w = d_int_ + kW * lanes_;
    int* d_wi = d_int_ + kWItems * lanes_;
    int* d_item0 = d_int_ + kItem0 * lanes_;
    int* d_nitems = d_int_ + kNItems * lanes_;
    int* d_wtc = d_int_ + kWTc * lanes_;
    int* d_tc0 = d_int_ + kTcItem0 * lanes_;
    int* d_tcn = d_int_ + kTcNItems * lanes_;
    const int nr = (int)ritems_.size(), ng = (int)gitems_.size(), nt = (int)titems_.size();
    const int Wb = 2 * max_sbar + 1;
    for (int j = 0; j < max_sbar; ++j) LS_CUDA(launch_mpk_items(d_desc_, d_ritems_, nr, d_steps, j, s_));
    if (item_gram) {
      // pair groups: enough CTAs to cover the SMs twice
      const int groups = std::max(1, std::min(16, (2 * gram_grid() + ng - 1) / std::max(ng, 1)));
      LS_CUDA(launch_gram_items(Wb, d_desc_, d_gitems_, ng, d_wi, d_partials_, groups, moments_, s_));
      LS_CUDA(launch_gram_items_finalize(Wb, d_partials_, d_item0, d_nitems, d_wi, hi_, d_G_, kGStride, moments_, s_));
    }
    if (tc_gram) {  // every tensor-core lane in one launch over the shared basis matrix
      LS_CUDA(launch_gram_tc_items(Wb, ybase_, yld_, yld_, d_titems_, nt, d_wtc, hi_, d_emax_, d_tpart_, s_));
      LS_CUDA(launch_gram_items_finalize(Wb, d_tpart_, d_tc0, d_tcn, d_wtc, hi_, d_G_, kGStride, false, s_));
    }
    LS_CUDA(launch_block_ctrl_batch(d_G_, kGStride, d_params_, d_params_ + kMaxS, d_params_ + 2 * kMaxS, d_bst_,
                                    hi_, max_sbar, o_.method == ASCG_ADAPTIVE, d_coords_, kCStride, d_res_hist_,
                                    rcap_, d_ab_hist_, abcap_, d_spec_, d_tickets_, s_));
    LS_CUDA(launch_recover_items(Wb, d_desc_, d_ritems_, nr, d_w, d_coords_, kCStride, s_));
    return ASCG_OK;
  }

  // The whole block loop of the held lanes as one launch: a graph whose
  // while-node body is lanes_advance_kernel (which decides, on the device,
  // each lane's next block or its end, and whether to go on) followed by the
  // block's kernels for s_max steps (lanes with fewer steps skip the rest, as
  // in a host-driven block with a larger s of another lane). The host takes
  // no part between blocks and reads each lane's outcome once at the end.
  // Each lane's arithmetic is the same as in the host-driven loop. *ran =
  // false (nothing done) when the stream cannot be captured or the graph
  // cannot be built, and the caller then drives the blocks from the host.
  ascg_status run_on_device(bool* ran) {
    *ran = false;
    if (!capturable_ || hi_ == 0) return ASCG_OK;
    if (!d_run_) {
      LS_TRY(dalloc(&d_run_, (size_t)lanes_));
      LS_TRY(dalloc(&d_iter_, 1));
      LS_TRY(dalloc(&d_seq_, (size_t)std::max<size_t>(seq_.size(), 1)));
    }
    std::vector<LaneRun> hr(hi_);
    bool any_tc = false;
    for (int q = 0; q < hi_; ++q) {
      const LaneSys& L = lane_[q];
      LaneRun& R = hr[q];
      std::memset(&R, 0, sizeof(R));
      R.active = used_[q] && L.active;
      R.m = L.m;
      R.kb = L.kb;
      R.s_prev = L.s_prev;
      R.wasted = L.wasted;
      R.status = L.status;
      R.tc_ok = used_[q] && !moments_ && L.d.n >= tc_rows_ && gram_tc_aligned(L.d.Y, L.d.ldY);
      R.rel_upd = L.rel_upd;
      R.eps_star = L.eps_star;
      R.bnorm = L.bnorm;
      R.sqrt_n = std::sqrt((double)L.d.n);
      any_tc = any_tc || (R.active && R.tc_ok && gram_tc_applies(2 * o_.s_max + 1));
    }
    LS_CUDA(cudaMemcpyAsync(d_run_, hr.data(), sizeof(LaneRun) * hi_, cudaMemcpyHostToDevice, s_));
    LS_CUDA(cudaMemsetAsync(d_iter_, 0, sizeof(int), s_));
    if (!seq_.empty())
      LS_CUDA(cudaMemcpyAsync(d_seq_, seq_.data(), sizeof(int) * seq_.size(), cudaMemcpyHostToDevice, s_));
    LoopParams lp;
    lp.method = o_.method;
    lp.s_max = o_.s_max;
    lp.s0 = o_.s0;
    lp.f = o_.f;
    lp.check_in_loop = o_.check_in_loop;
    lp.max_iters = o_.max_iters;
    lp.seq_len = (int)seq_.size();
    lp.iter_cap = o_.max_iters + 2;
    lp.c = o_.c;
    lp.seq = d_seq_;
    // the graph: one while node whose body is captured from the stream
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto fail_build = [&](cudaError_t e) {
      if (exec) cudaGraphExecDestroy(exec);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      (void)e;
      return ASCG_OK;  // *ran stays false: the host loop takes over
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return fail_build(e);
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail_build(e);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) return fail_build(e);
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s_, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail_build(e);
    int* d_steps = d_int_ + kSteps * lanes_;
    int* d_w = d_int_ + kW * lanes_;
    int* d_wi = d_int_ + kWItems * lanes_;
    int* d_wtc = d_int_ + kWTc * lanes_;
    lanes_advance_kernel<<<1, 1024, 0, s_>>>(d_bst_, d_run_, hi_, d_steps, d_w, d_wi, d_wtc, lp, d_iter_, cond);
    ascg_status st = cudaGetLastError() == cudaSuccess ? ASCG_OK : ASCG_ERR_CUDA;
    if (st == ASCG_OK) st = block_kernels(o_.s_max, true, any_tc);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(s_, &captured);
    if (st != ASCG_OK || e != cudaSuccess) return fail_build(e);
    e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) return fail_build(e);
    int iters = 0;
    e = cudaGraphLaunch(exec, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), d_run_, sizeof(LaneRun) * hi_, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&iters, d_iter_, sizeof(int), cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(g);
    LS_CUDA(e);
    for (int q = 0; q < hi_; ++q) {
      if (!used_[q]) continue;
      LaneSys& L = lane_[q];
      const LaneRun& R = hr[q];
      L.m = R.m;
      L.kb = R.kb;
      L.s_prev = R.s_prev;
      L.wasted = R.wasted;
      L.status = (ascg_status)R.status;
      L.rel_upd = R.rel_upd;
      if (R.active) {  // the block cap ended the loop (cannot happen: each block advances every lane)
        L.status = ASCG_NOT_CONVERGED;
      }
      L.active = false;
      L.done = true;
    }
    super_blocks_ += std::max(iters - 1, 0);  // the last pass found no lane running
    launches_ += 1;
    *ran = true;
    return ASCG_OK;
  }

  // Reads the block's outcome per lane (after the stream reached the end of
  // launch_block's work). Lanes whose system finished are marked done.
  void complete_block(ascg_block_info* block_hist, int block_hist_cap) {
    ++super_blocks_;
    for (int q = 0; q < hi_; ++q) {
      LaneSys& L = lane_[q];
      if (!used_[q] || !L.active) continue;
      const BlockState& out = h_bst_[q];
      const int sbar = L.sbar;
      if (block_hist && L.nb_info < block_hist_cap) {
        ascg_block_info& bi = block_hist[(int64_t)q * block_hist_cap + L.nb_info];
        std::memset(&bi, 0, sizeof(bi));
        bi.sbar = sbar;
        bi.stilde = out.stilde;
        bi.s_k = out.s_k;
        bi.stop = out.stop;
        bi.m = L.m;
        bi.rnorm = out.rnorm;
        bi.threshold = out.threshold;
        bi.gamma = out.gamma;
        for (int i = 0; i < sbar; ++i) bi.sqrt_kappa[i] = o_.method == ASCG_ADAPTIVE ? out.sqrt_kappa[i] : 0.0;
      }
      ++L.nb_info;
      L.wasted += 2 * (sbar - out.s_k);
      if (out.s_k == 0) {
        L.status = ASCG_ERR_BREAKDOWN;
        L.active = false;
        L.done = true;
        continue;
      }
      L.rel_upd = out.rel_res;
      L.m += out.s_k;
      L.s_prev = out.s_k;
      ++L.kb;
      if (out.converged) {
        L.active = false;
      } else if (L.m >= o_.max_iters) {
        L.status = ASCG_NOT_CONVERGED;
        L.active = false;
      }
      L.done = !L.active;
    }
  }

  // One block of every active lane, waiting for it.
  ascg_status super_block(ascg_block_info* block_hist, int block_hist_cap) {
    bool launched = false;
    LS_TRY(launch_block(&launched));
    if (!launched) return ASCG_OK;
    LS_CUDA(cudaStreamSynchronize(s_));
    complete_block(block_hist, block_hist_cap);
    return ASCG_OK;
  }

  // Lanes held and done (finished, not yet retired).
  std::vector<int> done_lanes() const {
    std::vector<int> v;
    for (int q = 0; q < hi_; ++q)
      if (used_[q] && lane_[q].done) v.push_back(q);
    return v;
  }

  // True residuals ||b - A x|| / ||b|| of done lanes that are still held
  // (into Y column 2), and x = 0 for b = 0. Fills rel_true. Synchronises.
  ascg_status finish(const std::vector<int>& lanes) {
    if (lanes.empty()) return ASCG_OK;
    int* h_sel = h_int_ + kSel * lanes_;
    int* h_list = h_int_ + kList * lanes_;
    for (int q = 0; q < hi_; ++q) h_sel[q] = 0;
    for (size_t i = 0; i < lanes.size(); ++i) {
      h_sel[lanes[i]] = 1;
      h_list[i] = lanes[i];
    }
    int* d_sel = d_int_ + kSel * lanes_;
    int* d_list = d_int_ + kList * lanes_;
    LS_CUDA(cudaMemcpyAsync(d_sel, h_sel, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
    LS_CUDA(cudaMemcpyAsync(d_list, h_list, sizeof(int) * lanes.size(), cudaMemcpyHostToDevice, s_));
    LS_CUDA(launch_residual_items(d_desc_, d_ritems_, (int)ritems_.size(), d_sel, 1, s_));
    LS_CUDA(launch_seg_sumsq(d_desc_, d_list, (int)lanes.size(), 2, d_sums_, s_));
    LS_CUDA(cudaMemcpyAsync(h_sums_, d_sums_, sizeof(double) * lanes_, cudaMemcpyDeviceToHost, s_));
    launches_ += 2;
    for (int q : lanes)
      if (lane_[q].bnorm == 0.0) LS_CUDA(cudaMemsetAsync(lane_[q].d.x, 0, sizeof(double) * lane_[q].d.n, s_));
    LS_CUDA(cudaStreamSynchronize(s_));
    for (int q : lanes) {
      LaneSys& L = lane_[q];
      L.rel_true = L.bnorm > 0.0 ? std::sqrt(std::max(h_sums_[q], 0.0)) / L.bnorm : 0.0;
    }
    return ASCG_OK;
  }

  // Frees the lanes; the caller takes back their bases. Tables are rebuilt
  // before the next block.
  void retire(const std::vector<int>& lanes) {
    for (int q : lanes) {
      if (!used_[q]) continue;
      used_[q] = 0;
      --nused_;
      std::memset(&h_desc_[q], 0, sizeof(SysDesc));
      lane_[q] = LaneSys();
    }
    while (hi_ > 0 && !used_[hi_ - 1]) --hi_;
    dirty_ = true;
  }

  // Tables after retirements (admit rebuilds them itself).
  ascg_status refresh() { return dirty_ ? rebuild_tables() : ASCG_OK; }

  // Copies lane q's histories to the caller's row (batched solves).
  ascg_status copy_histories(int q, const ascg_options& o, int64_t row) {
    const LaneSys& L = lane_[q];
    if (o.res_hist && rcap_)
      LS_CUDA(cudaMemcpy(o.res_hist + row * o.res_hist_cap, d_res_hist_ + (int64_t)q * rcap_,
                         sizeof(double) * std::min(L.m + 1, o.res_hist_cap), cudaMemcpyDeviceToHost));
    if (abcap_ && L.m > 0) {
      const int na = std::min(L.m, o.coef_hist_cap);
      LS_CUDA(cudaMemcpy(o.alpha_hist + row * o.coef_hist_cap, d_ab_hist_ + (int64_t)q * 2 * abcap_,
                         sizeof(double) * na, cudaMemcpyDeviceToHost));
      LS_CUDA(cudaMemcpy(o.beta_hist + row * o.coef_hist_cap, d_ab_hist_ + (int64_t)q * 2 * abcap_ + abcap_,
                         sizeof(double) * na, cudaMemcpyDeviceToHost));
    }
    return ASCG_OK;
  }

  void fill_result(int q, ascg_result* r) const {
    const LaneSys& L = lane_[q];
    std::memset(r, 0, sizeof(*r));
    r->status = L.status;
    r->iters = L.m;
    r->blocks = L.kb;
    r->grid_reductions = L.kb;
    r->wasted_vecs = L.wasted;
    r->launches = (int)std::min<int64_t>(super_blocks_, 0x7fffffff);
    r->bnorm = L.bnorm;
    r->rel_res_updated = L.rel_upd;
    r->rel_res_true = L.rel_true;
  }

  LaneSys& lane(int q) { return lane_[q]; }
  int nused() const { return nused_; }
  int64_t launches() const { return launches_; }
  cudaStream_t stream() const { return s_; }

 private:
  static constexpr int64_t kGStride = (int64_t)kMaxW * kMaxW;
  static constexpr int64_t kCStride = 3 * kMaxW;
  // int arrays of lanes entries each, in d_int_ and h_int_
  enum { kSteps = 0, kW, kSel, kList, kItem0, kNItems, kWItems, kWTc, kTcItem0, kTcNItems, kIntArrays };

  int count_active() const {
    int c = 0;
    for (int q = 0; q < hi_; ++q) c += used_[q] && lane_[q].active;
    return c;
  }

  ascg_status grow_titems(int64_t titems) {
    if (titems > tcap_items_) {
      LS_CUDA(cudaStreamSynchronize(s_));
      dfree(d_titems_);
      dfree(d_tpart_);
      tcap_items_ = std::max<int64_t>(titems, 2 * tcap_items_);
      LS_TRY(dalloc(&d_titems_, (size_t)tcap_items_));
      LS_TRY(dalloc(&d_tpart_, (size_t)tcap_items_ * tcnp_));
    }
    return ASCG_OK;
  }

  ascg_status grow_items(int64_t ritems, int64_t gitems) {
    if (ritems > rcap_items_) {
      LS_CUDA(cudaStreamSynchronize(s_));
      dfree(d_ritems_);
      rcap_items_ = std::max<int64_t>(ritems, 2 * rcap_items_);
      LS_TRY(dalloc(&d_ritems_, (size_t)rcap_items_));
    }
    if (gitems > gcap_items_) {
      LS_CUDA(cudaStreamSynchronize(s_));
      dfree(d_gitems_);
      dfree(d_partials_);
      gcap_items_ = std::max<int64_t>(gitems, 2 * gcap_items_);
      LS_TRY(dalloc(&d_gitems_, (size_t)gcap_items_));
      LS_TRY(dalloc(&d_partials_, (size_t)gcap_items_ * npw_));
    }
    return ASCG_OK;
  }

  // Row items, Gram items and descriptors of the held lanes, in lane order.
  // The pinned tables are rewritten only after the stream has passed the
  // copies below (every caller synchronises, or waits for the block's end,
  // before it changes the lanes again).
  ascg_status rebuild_tables() {
    ritems_.clear();
    gitems_.clear();
    titems_.clear();
    int* h_item0 = h_int_ + kItem0 * lanes_;
    int* h_nitems = h_int_ + kNItems * lanes_;
    int* h_tc0 = h_int_ + kTcItem0 * lanes_;
    int* h_tcn = h_int_ + kTcNItems * lanes_;
    for (int q = 0; q < hi_; ++q) {
      h_item0[q] = (int)gitems_.size();
      h_nitems[q] = 0;
      h_tc0[q] = (int)titems_.size();
      h_tcn[q] = 0;
      if (!used_[q]) continue;
      {  // whole 1024-row chunks of the lane's range in the shared basis matrix
        const int64_t rows = Arena::rounded(lane_[q].d.n), first = lane_[q].off;
        for (int64_t r = 0; r < rows; r += kTcItemRows)
          titems_.push_back(GramItem{first + r, (int)std::min<int64_t>(kTcItemRows, rows - r), q});
        h_tcn[q] = (int)titems_.size() - h_tc0[q];
      }
      const int64_t n = lane_[q].d.n;
      for (int64_t r = 0; r < n; r += kRowItem)
        ritems_.push_back(RowItem{q, (int)r, (int)std::min<int64_t>(kRowItem, n - r), 0});
      const int64_t gr = gram_item_rows(n);
      for (int64_t r = 0; r < n; r += gr) gitems_.push_back(GramItem{r, (int)std::min<int64_t>(gr, n - r), q});
      h_nitems[q] = (int)gitems_.size() - h_item0[q];
    }
    LS_TRY(grow_items((int64_t)ritems_.size(), (int64_t)gitems_.size()));
    LS_TRY(grow_titems((int64_t)titems_.size()));
    if (!titems_.empty())
      LS_CUDA(cudaMemcpyAsync(d_titems_, titems_.data(), sizeof(GramItem) * titems_.size(), cudaMemcpyHostToDevice, s_));
    if (!ritems_.empty())
      LS_CUDA(cudaMemcpyAsync(d_ritems_, ritems_.data(), sizeof(RowItem) * ritems_.size(), cudaMemcpyHostToDevice, s_));
    if (!gitems_.empty())
      LS_CUDA(cudaMemcpyAsync(d_gitems_, gitems_.data(), sizeof(GramItem) * gitems_.size(), cudaMemcpyHostToDevice, s_));
    if (hi_ > 0) {
      LS_CUDA(cudaMemcpyAsync(d_desc_, h_desc_, sizeof(SysDesc) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_int_ + kItem0 * lanes_, h_item0, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_int_ + kNItems * lanes_, h_nitems, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_int_ + kTcItem0 * lanes_, h_tc0, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
      LS_CUDA(cudaMemcpyAsync(d_int_ + kTcNItems * lanes_, h_tcn, sizeof(int) * hi_, cudaMemcpyHostToDevice, s_));
    }
    dirty_ = false;
    ++tables_version_;
    if (graphs_.size() >= kMaxGraphs) drop_graphs();
    return ASCG_OK;
  }

  static constexpr size_t kMaxGraphs = 64;
  void drop_graphs() {
    for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
    graphs_.clear();
  }

  void release() {
    drop_graphs();
    dfree(d_desc_); dfree(d_bst_); dfree(d_G_); dfree(d_coords_); dfree(d_int_); dfree(d_sums_); dfree(d_params_);
    dfree(d_res_hist_); dfree(d_ab_hist_); dfree(d_ritems_); dfree(d_gitems_); dfree(d_partials_);
    dfree(d_titems_); dfree(d_tpart_); dfree(d_emax_); dfree(d_spec_); dfree(d_tickets_);
    dfree(d_run_); dfree(d_iter_); dfree(d_seq_);
    hfree(h_desc_); hfree(h_bst_); hfree(h_int_); hfree(h_sums_);
  }

  ascg_options o_{};
  std::vector<int> seq_;
  cudaStream_t s_ = nullptr;
  int lanes_ = 0, nused_ = 0, hi_ = 0, rcap_ = 0, abcap_ = 0, wcols_ = 0, npw_ = 0;
  bool dirty_ = true;
  bool moments_ = false;  // Hankel-moment Gram (monomial basis)
  bool capturable_ = true;
  int64_t tc_rows_ = kTcLaneRows;  // lanes of at least this many rows: tensor-core Gram
  int tables_version_ = 0;
  std::map<std::vector<int>, cudaGraphExec_t> graphs_;  // captured blocks by shape
  int64_t super_blocks_ = 0, launches_ = 0;
  std::vector<LaneSys> lane_;
  std::vector<char> used_;
  std::vector<RowItem> ritems_;
  std::vector<GramItem> gitems_;
  std::vector<GramItem> titems_;
  int64_t rcap_items_ = 0, gcap_items_ = 0;
  SysDesc* d_desc_ = nullptr;
  BlockState* d_bst_ = nullptr;
  double* d_G_ = nullptr;
  double* d_coords_ = nullptr;
  int* d_int_ = nullptr;
  double* d_sums_ = nullptr;
  double* d_params_ = nullptr;
  double* d_res_hist_ = nullptr;
  double* d_ab_hist_ = nullptr;
  RowItem* d_ritems_ = nullptr;
  GramItem* d_gitems_ = nullptr;
  double* d_partials_ = nullptr;
  double* ybase_ = nullptr;  // the shared basis matrix (leading dimension yld_)
  int64_t yld_ = 0;
  GramItem* d_titems_ = nullptr;  // tensor-core Gram items (row ranges in the shared matrix)
  double* d_tpart_ = nullptr;     // their partials, tcnp_ each
  int* d_emax_ = nullptr;         // per-lane column exponents, kMaxW each
  int64_t tcap_items_ = 0;
  int tcnp_ = 0;
  LaneRun* d_run_ = nullptr;      // device-driven block loop: the lanes' running state
  int* d_iter_ = nullptr;         // its block counter
  int* d_seq_ = nullptr;          // Alg. 3's block sizes
  double* d_spec_ = nullptr;      // speculative coordinate steps, kSpecDoubles per lane
  unsigned* d_tickets_ = nullptr;  // the block controller's ticket counters, one per lane
  SysDesc* h_desc_ = nullptr;
  BlockState* h_bst_ = nullptr;
  int* h_int_ = nullptr;
  double* h_sums_ = nullptr;
};

// Batched solves: every system admitted at once, blocks until none is
// active, then the true residuals.
namespace {
// A stream of the call's own (blocks on it can be captured as graphs, which
// the legacy default stream does not allow), ordered after the caller's
// stream on entry and before it on exit.
struct OwnStream {
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev = nullptr;
  ascg_status open(cudaStream_t u) {
    user = u;
    LS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    LS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    LS_CUDA(cudaEventRecord(ev, user));
    LS_CUDA(cudaStreamWaitEvent(s, ev, 0));
    return ASCG_OK;
  }
  ~OwnStream() {
    if (s) {
      if (ev && cudaEventRecord(ev, s) == cudaSuccess) cudaStreamWaitEvent(user, ev, 0);
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    if (ev) cudaEventDestroy(ev);
  }
};
}  // namespace

ascg_status lockstep_solve_batch(int count, const ascg_op* ops, const double* const* b, double* const* x,
                                 const double* eps_target, const ascg_options& o, ascg_result* results,
                                 cudaStream_t user_stream) {
  OwnStream own;
  LS_TRY(own.open(user_stream));
  const cudaStream_t s = own.s;
  std::vector<LaneSys> sys(count);
  int64_t y_rows = 0, gi = 0, ri = 0;
  for (int q = 0; q < count; ++q) {
    LS_TRY(Lockstep::prepare(o.s_max, ops[q], b[q], x[q], eps_target ? eps_target[q] : o.eps_target, q, &sys[q]));
    y_rows += Arena::rounded(sys[q].d.n);
    gi += Lockstep::gram_items_of(sys[q].d.n);
    ri += Lockstep::row_items_of(sys[q].d.n);
  }
  if (y_rows > 0x7fffffffll) return lfail(ASCG_ERR_INVALID, "the batch exceeds 2^31 rows");
  Arena arena;  // destroyed after the engine and its stream's work (declaration order)
  LS_TRY(arena.init(2 * o.s_max + 1, y_rows));
  for (int q = 0; q < count; ++q) {
    if (!arena.take(sys[q].d.n, &sys[q].off)) return lfail(ASCG_ERR_OOM, "the batch does not fit its own arena");
    sys[q].d.Y = arena.row(sys[q].off);
    sys[q].d.ldY = arena.ld();
  }
  const int rcap = o.res_hist ? std::max(o.res_hist_cap, 1) : 0;
  const int abcap = (o.alpha_hist && o.beta_hist) ? std::max(o.coef_hist_cap, 1) : 0;
  Lockstep eng;
  LS_TRY(eng.init(o, count, gi, ri, rcap, abcap, arena.base(), arena.ld(), s));
  LS_TRY(eng.admit(sys, nullptr));
  for (int q = 0; q < count; ++q)
    if (eng.lane(q).status == ASCG_ERR_INVALID) return lfail(ASCG_ERR_INVALID, "b or x_1 is not finite");
  // Without per-block records to return, the whole block loop runs on the
  // device as one graph launch; otherwise (or if the graph cannot be built)
  // the host drives it block by block.
  bool on_device = false;
  if (!o.block_hist && eng.any_active()) LS_TRY(eng.run_on_device(&on_device));
  while (!on_device && eng.any_active()) LS_TRY(eng.super_block(o.block_hist, o.block_hist_cap));
  std::vector<int> all(count);
  for (int q = 0; q < count; ++q) all[q] = q;
  LS_TRY(eng.finish(all));
  ascg_status worst = ASCG_OK;
  for (int q = 0; q < count; ++q) {
    LS_TRY(eng.copy_histories(q, o, q));
    if (results) eng.fill_result(q, &results[q]);
    const ascg_status st = eng.lane(q).status;
    if (st == ASCG_ERR_BREAKDOWN) worst = ASCG_ERR_BREAKDOWN;
    else if (st == ASCG_NOT_CONVERGED && worst == ASCG_OK) worst = ASCG_NOT_CONVERGED;
  }
  if (worst == ASCG_ERR_BREAKDOWN) set_last_error("breakdown in at least one system (see results[q].status)");
  return worst;
}

}  // namespace ascg

// ===========================================================================
// Solve server (continuous batching)
// ===========================================================================

using namespace ascg;

namespace {

// Size classes of the server, by rows: each runs its own lockstep engine on
// its own stream and steps as soon as its previous block has landed, so
// small systems are not held to the pace of the large ones' blocks.
constexpr int kGroups = 3;
constexpr int64_t kGroupEnd[kGroups] = {(int64_t)1 << 16, (int64_t)1 << 19, INT64_MAX};

int group_of(int64_t n) {
  int g = 0;
  while (n >= kGroupEnd[g]) ++g;
  return g;
}

struct Group {
  Lockstep eng;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
  int64_t seq = 0;  // launch order, to wait for the oldest block first
};

}  // namespace

struct ascg_server_s {
  ascg_options o{};
  size_t budget = 0;
  int max_systems = 0;
  int running = 0;
  int admit_order = ASCG_ADMIT_FIFO;
  int large_cap = 0;       // > 0: most systems running at once in the largest size class
  bool yield_large = false;  // the largest class starts no block while a smaller class has systems
  cudaStream_t user = nullptr;
  Arena arena;
  Group group[kGroups];
  std::deque<LaneSys> queue;
  std::deque<ascg_completion> ready;
  int64_t steps = 0, seq = 0, launches = 0;

  ~ascg_server_s() {
    for (Group& g : group) {
      if (g.stream) cudaStreamSynchronize(g.stream);
    }
    for (LaneSys& L : queue)
      if (L.ready) cudaEventDestroy(L.ready);
    for (Group& g : group) {
      if (g.done) cudaEventDestroy(g.done);
      if (g.stream) cudaStreamDestroy(g.stream);  // the engines free their buffers afterwards
    }
  }

  void complete(Group& g, int q) {
    LaneSys& L = g.eng.lane(q);
    ascg_completion c;
    std::memset(&c, 0, sizeof(c));
    c.tag = L.tag;
    g.eng.fill_result(q, &c.result);
    c.result.launches = (int)std::min<int64_t>(steps - L.step_admit, 0x7fffffff);
    c.queue_ms = L.t_admit - L.t_submit;
    c.latency_ms = L.t_done - L.t_submit;
    c.step_admitted = L.step_admit;
    c.step_done = L.step_done;
    ready.push_back(c);
  }

  // Finishes, reports and frees the done lanes of group g (its stream idle).
  ascg_status retire_done(Group& g) {
    std::vector<int> fin = g.eng.done_lanes();
    if (fin.empty()) return ASCG_OK;
    LS_TRY(g.eng.finish(fin));
    const double t = now_ms();
    for (int q : fin) {
      LaneSys& L = g.eng.lane(q);
      L.t_done = t;
      L.step_done = steps;
      complete(g, q);
      arena.give(L.off);
    }
    running -= (int)fin.size();
    g.eng.retire(fin);
    return ASCG_OK;
  }

  // Estimated work of a request: its rows times the decimal digits of
  // accuracy it asks for (CG iterations grow with both).
  static double work_of(const LaneSys& L) {
    const double digits = L.eps_target > 0.0 ? -std::log10(L.eps_target) : 16.0;
    return (double)L.d.n * (digits > 1.0 ? digits : 1.0);
  }

  // Admission scan, in submission order (ASCG_ADMIT_FIFO) or in increasing
  // estimated work (ASCG_ADMIT_SHORTEST_FIRST, ties in submission order). A
  // request whose size class is in the middle of a block waits for it (later
  // requests of idle classes may go ahead), as does one whose class is at its
  // cap; the first request that finds no slot or no memory stops the scan.
  ascg_status admit() {
    std::vector<LaneSys> pick[kGroups];
    int taken[kGroups] = {0, 0, 0};
    std::vector<size_t> order(queue.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    if (admit_order == ASCG_ADMIT_SHORTEST_FIRST)
      std::stable_sort(order.begin(), order.end(),
                       [&](size_t a, size_t b) { return work_of(queue[a]) < work_of(queue[b]); });
    std::vector<char> gone(queue.size(), 0);
    for (size_t k = 0; k < order.size(); ++k) {
      LaneSys& Q = queue[order[k]];
      const int gi = group_of(Q.d.n);
      Group& g = group[gi];
      if (g.in_flight || g.eng.free_lanes() - taken[gi] <= 0) continue;
      if (large_cap > 0 && gi == kGroups - 1 && g.eng.active_lanes() + taken[gi] >= large_cap) continue;
      if (running >= max_systems) break;
      int64_t off = 0;
      if (!arena.take(Q.d.n, &off)) break;
      LaneSys L = Q;
      L.off = off;
      L.d.Y = arena.row(off);
      L.d.ldY = arena.ld();
      if (L.ready) {
        LS_CUDA(cudaStreamWaitEvent(g.stream, L.ready, 0));
        cudaEventDestroy(L.ready);
        L.ready = nullptr;
      }
      pick[gi].push_back(L);
      ++taken[gi];
      ++running;
      gone[order[k]] = 1;
    }
    if (!order.empty()) {
      std::deque<LaneSys> rest;
      for (size_t i = 0; i < queue.size(); ++i)
        if (!gone[i]) rest.push_back(queue[i]);
      queue.swap(rest);
    }
    for (int gi = 0; gi < kGroups; ++gi) {
      if (pick[gi].empty()) continue;
      Group& g = group[gi];
      std::vector<int> lanes;
      LS_TRY(g.eng.admit(pick[gi], &lanes));
      const double t = now_ms();
      for (int q : lanes) {
        g.eng.lane(q).t_admit = t;
        g.eng.lane(q).step_admit = steps;
      }
      LS_TRY(retire_done(g));  // systems that needed no block
    }
    return ASCG_OK;
  }
};

extern "C" {

ascg_status ascg_server_create(const ascg_options* opts, int64_t hbm_budget, int max_systems, void* cuda_stream,
                               ascg_server* out) {
  set_last_error("");
  if (!out) return lfail(ASCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!opts) return lfail(ASCG_ERR_INVALID, "opts is NULL");
  const ascg_options o = *opts;
  LS_TRY(check_options(o));
  if (o.method == ASCG_CLASSICAL) return lfail(ASCG_ERR_INVALID, "the server runs an s-step method");
  if (o.flags & ASCG_FLAG_C_FORMULA)
    return lfail(ASCG_ERR_INVALID, "ASCG_FLAG_C_FORMULA needs one system's kappa(A) and ||A||: use ascg_solve");
  if (o.basis != ASCG_MONOMIAL) return lfail(ASCG_ERR_INVALID, "the server uses the monomial basis");
  if (o.res_hist || o.block_hist || o.alpha_hist || o.beta_hist)
    return lfail(ASCG_ERR_INVALID, "the server keeps no histories: the history buffers must be NULL");
  if (max_systems < 1 || max_systems > (1 << 20)) return lfail(ASCG_ERR_INVALID, "max_systems must be in 1..2^20");
  if (hbm_budget < 1) return lfail(ASCG_ERR_INVALID, "hbm_budget must be >= 1");
  ascg_server srv = nullptr;
  try {
    srv = new ascg_server_s();
  } catch (const std::bad_alloc&) {
    return lfail(ASCG_ERR_OOM, "host allocation failed");
  }
  srv->o = o;
  srv->budget = (size_t)hbm_budget;
  srv->max_systems = max_systems;
  srv->user = (cudaStream_t)cuda_stream;
  // The Gram partials take (2 s_max + 1)(s_max + 1) doubles per item of at
  // least 1024 rows against (2 s_max + 1) 1024 doubles of basis: set them
  // aside out of the budget for the most rows the budget can hold, plus one
  // item per system.
  const int64_t wcols = 2 * o.s_max + 1;
  const int64_t npw = Lockstep::partials_per_item(o.s_max, (o.flags & ASCG_FLAG_MOMENT_GRAM) != 0);
  const int64_t rows_max = hbm_budget / (wcols * (int64_t)sizeof(double));
  const int64_t gitems = rows_max / kGramItemRowsMin + max_systems;
  const int64_t titems = rows_max / Lockstep::kTcItemRows + max_systems;
  const int64_t part_bytes = (gitems * npw + titems * (wcols * (wcols + 1) / 2)) * (int64_t)sizeof(double);
  const int64_t y_rows = std::min<int64_t>(std::max<int64_t>(hbm_budget - part_bytes, 0) /
                                               (wcols * (int64_t)sizeof(double)) / Arena::kRowAlign *
                                               Arena::kRowAlign,
                                           0x7fffffffll / Arena::kRowAlign * Arena::kRowAlign);
  auto fail_free = [&](ascg_status st) {
    delete srv;
    return st;
  };
  ascg_status st = srv->arena.init((int)wcols, y_rows);
  if (st != ASCG_OK) return fail_free(st);
  // Stream priorities: the smallest class highest, so that as the CTAs of a
  // large class's kernels retire, the SMs go to waiting small-class CTAs first.
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (int gi = 0; gi < kGroups; ++gi) {
    Group& g = srv->group[gi];
    const int prio = std::min(prio_least, prio_greatest + gi);  // greatest is the numerically lowest
    cudaError_t e = cudaStreamCreateWithPriority(&g.stream, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_free(lfail(ASCG_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e)));
    st = g.eng.init(o, max_systems, gitems / kGroups + 1, 1024, 0, 0, srv->arena.base(), srv->arena.ld(), g.stream);
    if (st != ASCG_OK) return fail_free(st);
  }
  *out = srv;
  return ASCG_OK;
}

ascg_status ascg_server_set_policy(ascg_server srv, int admit_order, int large_class_cap, int yield_large) {
  set_last_error("");
  if (!srv) return lfail(ASCG_ERR_INVALID, "srv is NULL");
  if (admit_order != ASCG_ADMIT_FIFO && admit_order != ASCG_ADMIT_SHORTEST_FIRST)
    return lfail(ASCG_ERR_INVALID, "unknown admission order");
  if (large_class_cap < 0) return lfail(ASCG_ERR_INVALID, "large_class_cap must be >= 0");
  srv->admit_order = admit_order;
  srv->large_cap = large_class_cap;
  srv->yield_large = yield_large != 0;
  return ASCG_OK;
}

ascg_status ascg_server_destroy(ascg_server srv) {
  if (!srv) return ASCG_OK;
  delete srv;
  return ASCG_OK;
}

ascg_status ascg_server_submit(ascg_server srv, ascg_op op, const double* b, double* x, double eps_target,
                               int64_t tag) {
  set_last_error("");
  if (!srv) return lfail(ASCG_ERR_INVALID, "srv is NULL");
  LaneSys L;
  LS_TRY(Lockstep::prepare(srv->o.s_max, op, b, x, eps_target, tag, &L));
  if (Lockstep::footprint(srv->o.s_max, L.d.n, (srv->o.flags & ASCG_FLAG_MOMENT_GRAM) != 0) > srv->budget ||
      L.bytes > srv->arena.bytes_total())
    return lfail(ASCG_ERR_INVALID, "the system needs more device memory than the server's budget");
  LS_CUDA(cudaEventCreateWithFlags(&L.ready, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(L.ready, srv->user);
  if (e != cudaSuccess) {
    cudaEventDestroy(L.ready);
    return lfail(ASCG_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
  }
  L.t_submit = now_ms();
  try {
    srv->queue.push_back(L);
  } catch (const std::bad_alloc&) {
    cudaEventDestroy(L.ready);
    return lfail(ASCG_ERR_OOM, "host allocation failed");
  }
  return ASCG_OK;
}

ascg_status ascg_server_step(ascg_server srv, ascg_completion* done, int cap, int* ndone, int* nactive,
                             int* npending) {
  set_last_error("");
  if (!srv || (cap > 0 && !done) || cap < 0) return lfail(ASCG_ERR_INVALID, "bad argument");
  try {
    for (;;) {
      bool progressed = false;
      // 1. blocks that have landed
      for (Group& g : srv->group) {
        if (!g.in_flight) continue;
        const cudaError_t q = cudaEventQuery(g.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return lfail(ASCG_ERR_CUDA, std::string("block: ") + cudaGetErrorString(q));
        g.in_flight = false;
        g.eng.complete_block(nullptr, 0);
        ++srv->steps;
        progressed = true;
        LS_TRY(srv->retire_done(g));
      }
      // 2. admission
      const size_t before = srv->ready.size();
      if (!srv->queue.empty()) LS_TRY(srv->admit());
      progressed = progressed || srv->ready.size() > before;
      // 3. the next block of every idle group with work (the largest class
      // waits while a smaller one has systems, when it yields)
      bool in_flight = false, smaller_busy = false;
      for (int gi = 0; gi < kGroups; ++gi) {
        Group& g = srv->group[gi];
        const bool yield = srv->yield_large && gi == kGroups - 1 && smaller_busy;
        smaller_busy = smaller_busy || g.eng.active_lanes() > 0;
        if (!g.in_flight && !yield) {
          LS_TRY(g.eng.refresh());
          bool launched = false;
          LS_TRY(g.eng.launch_block(&launched));
          if (launched) {
            LS_CUDA(cudaEventRecord(g.done, g.stream));
            g.in_flight = true;
            g.seq = ++srv->seq;
          }
        }
        in_flight = in_flight || g.in_flight;
      }
      if (progressed || !in_flight) break;
      // 4. nothing landed yet: wait for the oldest block
      Group* oldest = nullptr;
      for (Group& g : srv->group)
        if (g.in_flight && (!oldest || g.seq < oldest->seq)) oldest = &g;
      LS_CUDA(cudaEventSynchronize(oldest->done));
    }
  } catch (const std::bad_alloc&) {
    return lfail(ASCG_ERR_OOM, "host allocation failed");
  }
  int nd = 0;
  while (nd < cap && !srv->ready.empty()) {
    done[nd++] = srv->ready.front();
    srv->ready.pop_front();
  }
  if (ndone) *ndone = nd;
  if (nactive) *nactive = srv->running;
  if (npending) *npending = (int)std::min<size_t>(srv->queue.size() + srv->ready.size(), 0x7fffffff);
  return ASCG_OK;
}

ascg_status ascg_tune_gram_schedule(int s_max, int64_t* tc_lane_rows, double* table, int table_cap, int* rows,
                                    void* cuda_stream) {
  set_last_error("");
  if (!tc_lane_rows || s_max < 1 || s_max > ASCG_MAX_S || table_cap < 0 || (table_cap > 0 && !table))
    return lfail(ASCG_ERR_INVALID, "bad argument");
  *tc_lane_rows = -1;
  if (rows) *rows = 0;
  const int w = 2 * s_max + 1;
  if (!gram_tc_applies(w)) return ASCG_OK;  // narrow bases always take the FP64 kernel
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  constexpr int kLogMin = 12, kLogMax = 22, kReps = 5;
  const int64_t ld = (int64_t)1 << kLogMax;
  struct Bufs {
    double *Y = nullptr, *G = nullptr, *part = nullptr, *tpart = nullptr;
    int *ints = nullptr, *emax = nullptr;
    SysDesc* desc = nullptr;
    GramItem *items = nullptr, *titems = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Bufs() {
      dfree(Y); dfree(G); dfree(part); dfree(tpart); dfree(ints); dfree(emax); dfree(desc); dfree(items);
      dfree(titems);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } B;
  const int64_t max_items = ld / kGramItemRowsMin + 1, max_titems = ld / Lockstep::kTcItemRows + 1;
  const int64_t np = (int64_t)w * (w + 1) / 2;
  LS_TRY(dalloc(&B.Y, (size_t)w * ld));
  LS_TRY(dalloc(&B.G, (size_t)kMaxW * kMaxW));
  LS_TRY(dalloc(&B.part, (size_t)max_items * np));
  LS_TRY(dalloc(&B.tpart, (size_t)max_titems * np));
  LS_TRY(dalloc(&B.emax, (size_t)kMaxW));
  LS_TRY(dalloc(&B.ints, 5));
  LS_TRY(dalloc(&B.desc, 1));
  LS_TRY(dalloc(&B.items, (size_t)max_items));
  LS_TRY(dalloc(&B.titems, (size_t)max_titems));
  LS_CUDA(cudaEventCreate(&B.e0));
  LS_CUDA(cudaEventCreate(&B.e1));
  LS_CUDA(launch_fill_uniform(B.Y, (int64_t)w * ld, 0x5eed5eedull, s));
  std::vector<double> t_fp(kLogMax + 1), t_tc(kLogMax + 1);
  int nrow = 0;
  for (int lg = kLogMin; lg <= kLogMax; ++lg) {
    const int64_t n = (int64_t)1 << lg;
    SysDesc d{};
    d.n = n;
    d.Y = B.Y;
    d.ldY = ld;
    std::vector<GramItem> items, titems;
    const int64_t gr = gram_item_rows(n);
    for (int64_t r = 0; r < n; r += gr) items.push_back(GramItem{r, (int)std::min<int64_t>(gr, n - r), 0});
    const int64_t padded = Arena::rounded(n);
    for (int64_t r = 0; r < padded; r += Lockstep::kTcItemRows)
      titems.push_back(GramItem{r, (int)std::min<int64_t>(Lockstep::kTcItemRows, padded - r), 0});
    const int ng = (int)items.size(), nt = (int)titems.size();
    const int ints[5] = {w, 0, ng, 0, nt};  // sys_w, item0, nitems, tc item0, tc nitems
    LS_CUDA(cudaMemcpyAsync(B.desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    LS_CUDA(cudaMemcpyAsync(B.items, items.data(), sizeof(GramItem) * ng, cudaMemcpyHostToDevice, s));
    LS_CUDA(cudaMemcpyAsync(B.titems, titems.data(), sizeof(GramItem) * nt, cudaMemcpyHostToDevice, s));
    LS_CUDA(cudaMemcpyAsync(B.ints, ints, sizeof(ints), cudaMemcpyHostToDevice, s));
    LS_CUDA(cudaStreamSynchronize(s));  // the host arrays above are locals
    const int groups = std::max(1, std::min(16, (2 * gram_grid() + ng - 1) / ng));
    std::vector<float> a(kReps), b(kReps);
    for (int rep = 0; rep < kReps + 1; ++rep) {  // the first run of each is a warm-up
      LS_CUDA(cudaEventRecord(B.e0, s));
      LS_CUDA(launch_gram_items(w, B.desc, B.items, ng, B.ints, B.part, groups, false, s));
      LS_CUDA(launch_gram_items_finalize(w, B.part, B.ints + 1, B.ints + 2, B.ints, 1, B.G, kMaxW * kMaxW, false, s));
      LS_CUDA(cudaEventRecord(B.e1, s));
      LS_CUDA(cudaEventSynchronize(B.e1));
      float ms = 0.f;
      LS_CUDA(cudaEventElapsedTime(&ms, B.e0, B.e1));
      if (rep > 0) a[rep - 1] = ms;
      LS_CUDA(cudaEventRecord(B.e0, s));
      LS_CUDA(launch_gram_tc_items(w, B.Y, ld, ld, B.titems, nt, B.ints, 1, B.emax, B.tpart, s));
      LS_CUDA(launch_gram_items_finalize(w, B.tpart, B.ints + 3, B.ints + 4, B.ints, 1, B.G, kMaxW * kMaxW, false, s));
      LS_CUDA(cudaEventRecord(B.e1, s));
      LS_CUDA(cudaEventSynchronize(B.e1));
      LS_CUDA(cudaEventElapsedTime(&ms, B.e0, B.e1));
      if (rep > 0) b[rep - 1] = ms;
    }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    t_fp[lg] = 1e3 * a[kReps / 2];
    t_tc[lg] = 1e3 * b[kReps / 2];
    if (nrow < table_cap) {
      table[3 * nrow] = (double)n;
      table[3 * nrow + 1] = t_fp[lg];
      table[3 * nrow + 2] = t_tc[lg];
      ++nrow;
    }
  }
  if (rows) *rows = nrow;
  // In a batch both kinds of Gram run as one launch over all lanes that fills
  // the GPU, so each costs its per-row rate at full load (taken at the largest
  // size) times the rows it reads: n for the FP64 items, round_up(n, 1024) for
  // the tensor cores. The threshold is the smallest power of two n >= 2^8 from
  // which the tensor cores cost less at every larger size.
  const double c_fp = t_fp[kLogMax] / (double)ld, c_tc = t_tc[kLogMax] / (double)ld;
  int from = 31;
  for (int lg = 30; lg >= 8; --lg) {
    const int64_t m = (int64_t)1 << lg;
    if (c_tc * (double)Arena::rounded(m) < c_fp * (double)m)
      from = lg;
    else
      break;
  }
  *tc_lane_rows = from <= 30 ? ((int64_t)1 << from) : -1;
  return ASCG_OK;
}

ascg_status ascg_server_info(ascg_server srv, ascg_server_stats* st) {
  if (!srv || !st) return lfail(ASCG_ERR_INVALID, "bad argument");
  std::memset(st, 0, sizeof(*st));
  st->budget_bytes = (int64_t)srv->budget;
  st->basis_bytes_used = (int64_t)srv->arena.bytes_used();
  st->basis_bytes_total = (int64_t)srv->arena.bytes_total();
  st->systems_running = srv->running;
  st->max_systems = srv->max_systems;
  st->queued = (int64_t)srv->queue.size();
  st->completions_pending = (int64_t)srv->ready.size();
  st->steps = srv->steps;
  int64_t l = 0;
  for (const Group& g : srv->group) l += g.eng.launches();
  st->launches = l;
  return ASCG_OK;
}

}  // extern "C"
