// Batched solves: many independent SPD systems advance block by block in
// lockstep. Their rows are concatenated, each system padded to whole 32-row
// slices, so the stacked operator is block diagonal and one launch of a
// per-row kernel serves every system. A slice never mixes systems: a warp
// looks up its system once (slice_sys) and skips it when it is inactive.
// Per-row work depends only on the row's own system, so each system's result
// is the same alone and in any batch.
#include "ascg_common.cuh"

namespace ascg {
namespace {

// Matrix powers step j in the monomial basis (theta = sigma = 0, gamma = 1;
// eq. (polybasiscg)): column 2j+2 = A column 2j, and column 2j+3 = A column
// 2j+1 while j + 1 < sbar, with A = D + O. sys_steps[q] = sbar_q of this block
// (0 for an inactive system).
__global__ void __launch_bounds__(kSpmvRows) mpk_batch_step_kernel(DevSell O, const double* __restrict__ diag,
                                                                   const int* __restrict__ slice_sys,
                                                                   const int* __restrict__ sys_steps,
                                                                   double* __restrict__ Y, int64_t ldY, int j) {
  const int64_t row = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  if (row >= O.n) return;
  const int64_t sl = row >> 5;
  const int steps = sys_steps[slice_sys[sl]];
  if (j >= steps) return;  // uniform over the warp
  const double* pj = Y + (int64_t)(2 * j) * ldY;
  const double* rj = Y + (int64_t)(2 * j + 1) * ldY;
  const int l = (int)(row & 31);
  const int64_t b = O.ptr[sl];
  const int width = (int)((O.ptr[sl + 1] - b) >> 5);
  const double* v = O.val + b + l;
  const int32_t* c = O.col + b + l;
  const double dg = diag[row];
  double tp = dg * pj[row];
  if (j + 1 < steps) {
    double tr = dg * rj[row];
    for (int k = 0; k < width; ++k) {
      const double a = __ldg(v + kSlice * k);
      const int cc = __ldg(c + kSlice * k);
      tp = fma(a, __ldg(pj + cc), tp);
      tr = fma(a, __ldg(rj + cc), tr);
    }
    Y[(int64_t)(2 * j + 3) * ldY + row] = tr;
  } else {
    for (int k = 0; k < width; ++k) tp = fma(__ldg(v + kSlice * k), __ldg(pj + __ldg(c + kSlice * k)), tp);
  }
  Y[(int64_t)(2 * j + 2) * ldY + row] = tp;
}

// r = b - (D + O) x for every row; also p = r when p != nullptr.
__global__ void __launch_bounds__(kSpmvRows) batch_residual_kernel(DevSell O, const double* __restrict__ diag,
                                                                   const double* __restrict__ b,
                                                                   const double* __restrict__ x,
                                                                   double* __restrict__ r, double* __restrict__ p) {
  const int64_t row = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  if (row >= O.n) return;
  const int64_t sl = row >> 5;
  const int l = (int)(row & 31);
  const int64_t o = O.ptr[sl];
  const int width = (int)((O.ptr[sl + 1] - o) >> 5);
  double ax = diag[row] * x[row];
  for (int k = 0; k < width; ++k) ax = fma(__ldg(O.val + o + kSlice * k + l), x[__ldg(O.col + o + kSlice * k + l)], ax);
  const double rr = b[row] - ax;
  r[row] = rr;
  if (p) p[row] = rr;
}

// out[q] = sum of u_i^2 over the rows of system q (one CTA per system, fixed
// summation order: strided thread sums, then a fixed tree).
__global__ void __launch_bounds__(1024) seg_sumsq_kernel(const double* __restrict__ u,
                                                         const int64_t* __restrict__ sys_row0,
                                                         const int64_t* __restrict__ sys_n, double* __restrict__ out) {
  const int q = blockIdx.x;
  const double* v = u + sys_row0[q];
  const int64_t n = sys_n[q];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) s = fma(v[i], v[i], s);
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = warp_sum(red[threadIdx.x]);
    if (threadIdx.x == 0) out[q] = s;
  }
}

// x += Y x', r = Y r', p = Y p' (eq. (coords)) for every row of an active
// system: its coordinates sit at coords + q * c_stride as x'[w_q], r'[w_q],
// p'[w_q]. Each thread reads its whole row of Y before writing, so r and p may
// alias columns 1 and 0.
template <int W>
__global__ void __launch_bounds__(256) recover_batch_kernel(int64_t n, const double* Y, int64_t ldY,
                                                            const int* __restrict__ slice_sys,
                                                            const int* __restrict__ sys_w,
                                                            const double* __restrict__ coords, int64_t c_stride,
                                                            double* x, double* r, double* p) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int q = slice_sys[row >> 5];
  const int w = sys_w[q];
  if (w == 0) return;  // uniform over the warp
  const double* cq = coords + (int64_t)q * c_stride;
  double y[W];
#pragma unroll
  for (int c = 0; c < W; ++c) y[c] = c < w ? Y[(int64_t)c * ldY + row] : 0.0;
  double sx = 0.0, sr = 0.0, sp = 0.0;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    if (c < w) {
      sx = fma(y[c], __ldg(cq + c), sx);
      sr = fma(y[c], __ldg(cq + w + c), sr);
      sp = fma(y[c], __ldg(cq + 2 * w + c), sp);
    }
  }
  x[row] += sx;
  r[row] = sr;
  p[row] = sp;
}

__global__ void add_offset_i32_kernel(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n,
                                      int32_t off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + off;
}

__global__ void add_offset_i64_kernel(int64_t* __restrict__ dst, const int64_t* __restrict__ src, int64_t n,
                                      int64_t off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + off;
}

}  // namespace

cudaError_t launch_mpk_batch_step(const DevSell& O, const double* diag, const int* slice_sys, const int* sys_steps,
                                  double* Y, int64_t ldY, int j, cudaStream_t s) {
  const int64_t g = (O.n + kSpmvRows - 1) / kSpmvRows;
  if (g < 1) return cudaSuccess;
  mpk_batch_step_kernel<<<(int)g, kSpmvRows, 0, s>>>(O, diag, slice_sys, sys_steps, Y, ldY, j);
  return cudaGetLastError();
}

cudaError_t launch_batch_residual(const DevSell& O, const double* diag, const double* b, const double* x, double* r,
                                  double* p, cudaStream_t s) {
  const int64_t g = (O.n + kSpmvRows - 1) / kSpmvRows;
  if (g < 1) return cudaSuccess;
  batch_residual_kernel<<<(int)g, kSpmvRows, 0, s>>>(O, diag, b, x, r, p);
  return cudaGetLastError();
}

cudaError_t launch_seg_sumsq(const double* u, const int64_t* sys_row0, const int64_t* sys_n, int count, double* out,
                             cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  seg_sumsq_kernel<<<count, 1024, 0, s>>>(u, sys_row0, sys_n, out);
  return cudaGetLastError();
}

cudaError_t launch_recover_batch(int W, int64_t n, const double* Y, int64_t ldY, const int* slice_sys,
                                 const int* sys_w, const double* coords, int64_t c_stride, double* x, double* r,
                                 double* p, cudaStream_t s) {
  const int64_t g = (n + 255) / 256;
  if (g < 1) return cudaSuccess;
  switch (W) {
#define ASCG_RB(WW)                                                                                           \
  case WW:                                                                                                    \
    recover_batch_kernel<WW><<<(int)g, 256, 0, s>>>(n, Y, ldY, slice_sys, sys_w, coords, c_stride, x, r, p); \
    return cudaGetLastError();
    ASCG_RB(3) ASCG_RB(5) ASCG_RB(7) ASCG_RB(9) ASCG_RB(11) ASCG_RB(13) ASCG_RB(15) ASCG_RB(17) ASCG_RB(19)
    ASCG_RB(21) ASCG_RB(23) ASCG_RB(25) ASCG_RB(27) ASCG_RB(29) ASCG_RB(31) ASCG_RB(33)
#undef ASCG_RB
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_add_offset_i32(int32_t* dst, const int32_t* src, int64_t n, int32_t off, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  add_offset_i32_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(dst, src, n, off);
  return cudaGetLastError();
}

cudaError_t launch_add_offset_i64(int64_t* dst, const int64_t* src, int64_t n, int64_t off, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  add_offset_i64_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(dst, src, n, off);
  return cudaGetLastError();
}

}  // namespace ascg
