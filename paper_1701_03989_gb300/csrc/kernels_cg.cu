// SpMV, residual, dot products and classical CG (Alg. 1).
//
// SpMV layout: sliced ELL (see DevSell), one thread per row, one warp per
// 32-row slice. Each thread sums its row with sequential FMAs in stored column
// order, which is the fewest FP64 instructions per nonzero. Every load of a
// warp is one contiguous segment.
//
// Reductions are deterministic. Each CTA writes a partial sum; the last CTA
// to finish (by an atomic ticket) adds the partials in index order. There are
// no spin-waits.
#include "ascg_common.cuh"

namespace ascg {

namespace {

// sum_j a_ij x_j for row i (i < A.n) in stored order, starting from 0. With
// STREAM, the values and column indices of A, read once per pass, are loaded
// with the evict-first (streaming) policy, so that the vectors of an
// iteration, which every pass reads again, keep their place in L2: worth it
// when A does not fit in L2 beside them. A small A is better left in L2.
template <bool STREAM = false>
__device__ __forceinline__ double sell_row(const DevSell& A, int64_t i, const double* __restrict__ x) {
  const int64_t s = i >> 5;
  const int l = (int)(i & 31);
  const int64_t b = A.ptr[s];
  const int width = (int)((A.ptr[s + 1] - b) >> 5);
  const double* v = A.val + b + l;
  const int32_t* c = A.col + b + l;
  double t = 0.0;
  if (STREAM) {
    for (int j = 0; j < width; ++j) t = fma(__ldcs(v + kSlice * j), __ldg(x + __ldcs(c + kSlice * j)), t);
  } else {
    for (int j = 0; j < width; ++j) t = fma(__ldg(v + kSlice * j), __ldg(x + __ldg(c + kSlice * j)), t);
  }
  return t;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  // fixed-order CTA reduction: warp trees, then warp 0 adds the warp sums in order
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// Deterministic completion: writes partials[blockIdx.x] and returns true in the
// CTA that finishes last, which may then read every partial.
__device__ __forceinline__ bool last_block(double part, double* partials, unsigned* counter, int* flag) {
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *flag = (prev == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = *flag;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ double sum_partials(const double* partials, int np, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += __ldcg(partials + i);
  return block_sum(s, red);
}

// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kSpmvRows) spmv_kernel(DevSell A, const double* __restrict__ x,
                                                         double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  if (i < A.n) y[i] = sell_row(A, i, x);
}

__global__ void __launch_bounds__(kSpmvRows) residual_kernel(DevSell A, const double* __restrict__ b,
                                                             const double* __restrict__ x,
                                                             double* __restrict__ r, double* __restrict__ p) {
  const int64_t i = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  if (i < A.n) {
    const double v = b[i] - sell_row(A, i, x);
    r[i] = v;
    if (p) p[i] = v;
  }
}

__global__ void __launch_bounds__(256) dot_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                                  int64_t n, double* out, double* partials, unsigned* counter) {
  __shared__ double red[32];
  __shared__ int flag;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(u[i], v[i], s);
  s = block_sum(s, red);
  if (last_block(s, partials, counter, &flag)) {
    const double tot = sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      *out = tot;
      *counter = 0u;
    }
  }
}

// --- classical CG -----------------------------------------------------------

// Grid-stride over rows with a bounded grid: every CTA ends in one block
// reduction and one atomic ticket, so few CTAs keep that overhead small. Each
// warp-wide FP64 add costs a full FP64 issue slot, however few lanes need it.
template <bool STREAM>
__global__ void __launch_bounds__(kSpmvRows) cg_spmv_dot_kernel(DevSell A, const double* __restrict__ p,
                                                                double* __restrict__ q, CGState* st,
                                                                double* partials, unsigned* counter) {
  __shared__ double red[32];
  __shared__ int flag;
  pdl_wait();     // the previous kernel's p and state
  pdl_release();
  const int done = st->done;  // uniform: written by an earlier kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) st->active = !done;  // read by the next two kernels
  if (done) return;
  double part = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * kSpmvRows) {
    const double v = sell_row<STREAM>(A, i, p);
    q[i] = v;
    part = fma(p[i], v, part);
  }
  part = block_sum(part, red);
  if (last_block(part, partials, counter, &flag)) {
    const double pq = sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->pAp = pq;
      if (pq > 0.0 && isfinite(pq)) {
        st->alpha = st->rr / pq;  // Alg. 1: alpha_i = r^T r / p^T A p
      } else {
        // breakdown (A is not SPD, or the data is not finite): this iteration
        // is skipped and the solve stops with x, r and p as they were
        st->alpha = 0.0;
        st->breakdown = 1;
        st->done = 1;
        st->active = 0;
      }
      *counter = 0u;
    }
  }
}

// r -= alpha A p and r^T r. x is not needed until the iteration's end: its
// update x += alpha p (the same FMA) runs in cg_pupdate_kernel, which reads p
// anyway, one pass over x and p fewer per iteration.
__global__ void __launch_bounds__(256) cg_update_kernel(int64_t n, double* __restrict__ r,
                                                        const double* __restrict__ q, CGState* st,
                                                        double* partials, unsigned* counter, double* res_hist,
                                                        int res_cap, double* alpha_hist, double* beta_hist,
                                                        int ab_cap) {
  __shared__ double red[32];
  __shared__ int flag;
  pdl_wait();     // q and alpha from the SpMV
  pdl_release();
  if (!st->active) return;
  const double alpha = st->alpha;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = fma(-alpha, q[i], r[i]);  // r -= A q = alpha (A p)
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s, red);
  if (last_block(s, partials, counter, &flag)) {
    const double rr = sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      const double beta = rr / st->rr;       // beta_i = r_{i+1}^T r_{i+1} / r_i^T r_i
      const int it = st->iter;
      if (it < ab_cap) {
        if (alpha_hist) alpha_hist[it] = alpha;
        if (beta_hist) beta_hist[it] = beta;
      }
      st->beta = beta;
      st->rr = rr;
      st->iter = it + 1;
      const double rn = sqrt(rr);
      if (res_hist && it + 1 < res_cap) res_hist[it + 1] = rn / st->bnorm;
      const int conv = rn <= st->eps_star;
      st->converged = conv;
      // p is still updated for this iteration (cg_pupdate reads 'active')
      st->done = conv || (it + 1 >= st->max_iters);
      *counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(256) cg_pupdate_kernel(int64_t n, double* __restrict__ x,
                                                         const double* __restrict__ r, double* __restrict__ p,
                                                         const CGState* st) {
  pdl_wait();     // r and beta from the update
  pdl_release();
  if (!st->active) return;  // this iteration was skipped (solve already done)
  const double alpha = st->alpha, beta = st->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = fma(alpha, pi, x[i]);             // x += q, q = alpha p (the iteration's p)
    p[i] = fma(beta, pi, r[i]);              // p = r + beta p
  }
}

__global__ void cg_init_kernel(CGState* st, double eps_star, double bnorm, int max_iters, int iter0,
                               double* res_hist, int res_cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->eps_star = eps_star;
    st->bnorm = bnorm;
    st->iter = iter0;
    st->max_iters = max_iters;
    const double rn = sqrt(st->rr);
    if (res_hist && iter0 < res_cap) res_hist[iter0] = rn / bnorm;
    st->converged = rn <= eps_star;
    st->done = st->converged || iter0 >= max_iters;
    st->alpha = st->beta = st->pAp = 0.0;
    st->active = 0;
    st->breakdown = 0;
  }
}

}  // namespace

cudaError_t launch_spmv(const DevSell& A, const double* x, double* y, cudaStream_t s) {
  const int g = (int)((A.n + kSpmvRows - 1) / kSpmvRows);
  spmv_kernel<<<g, kSpmvRows, 0, s>>>(A, x, y);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevSell& A, const double* b, const double* x, double* r, double* p,
                            cudaStream_t s) {
  const int g = (int)((A.n + kSpmvRows - 1) / kSpmvRows);
  residual_kernel<<<g, kSpmvRows, 0, s>>>(A, b, x, r, p);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* u, const double* v, int64_t n, double* out, double* partials,
                       unsigned* counter, cudaStream_t s) {
  dot_kernel<<<grid_for(n, 256, kRedBlocks), 256, 0, s>>>(u, v, n, out, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_cg_spmv_dot(const DevSell& A, int64_t nnz, const double* p, double* q, CGState* st,
                               double* partials, unsigned* counter, cudaStream_t s) {
  const int g = grid_for(A.n, kSpmvRows, 152 * 8);
  // A's values and columns (12 bytes per entry) beyond a quarter of the 129 MB
  // L2: stream them past it
  if (12 * nnz > ((int64_t)32 << 20))
    return launch_pdl(cg_spmv_dot_kernel<true>, g, kSpmvRows, s, A, p, q, st, partials, counter);
  return launch_pdl(cg_spmv_dot_kernel<false>, g, kSpmvRows, s, A, p, q, st, partials, counter);
}

cudaError_t launch_cg_update(int64_t n, double* r, const double* q, CGState* st, double* partials,
                             unsigned* counter, double* res_hist, int res_cap, double* alpha_hist, double* beta_hist,
                             int ab_cap, cudaStream_t s) {
  // HBM-bound axpys: 8 CTAs per SM keep enough loads in flight (partials hold one
  // slot per 256-row block, so any grid up to n/256 fits)
  return launch_pdl(cg_update_kernel, grid_for(n, 256, 152 * 8), 256, s, n, r, q, st, partials, counter, res_hist,
                    res_cap, alpha_hist, beta_hist, ab_cap);
}

cudaError_t launch_cg_pupdate(int64_t n, double* x, const double* r, double* p, const CGState* st, cudaStream_t s) {
  return launch_pdl(cg_pupdate_kernel, grid_for(n, 256, 4096), 256, s, n, x, r, p, st);
}

cudaError_t launch_cg_init(CGState* st, double eps_star, double bnorm, int max_iters, int iter0,
                           double* res_hist, int res_cap, cudaStream_t s) {
  cg_init_kernel<<<1, 32, 0, s>>>(st, eps_star, bnorm, max_iters, iter0, res_hist, res_cap);
  return cudaGetLastError();
}

}  // namespace ascg
