// Matrix powers (eq. polybasiscg / cg-krylovbasis) and recovery (eq. coords).
//
// Basis layout: Y is column-major with leading dimension ldY and interleaves
// the two Krylov bases: column 2j = rho_j(A) p, column 2j+1 = rho_j(A) r.
// Then every i-step sub-basis Y_{k,i} is the first 2i+1 columns.
//
// One matrix powers step j forms column 2(j+1) of P and column 2(j+1)+1 of R
// in the same pass over A. Each value and column index of O (sliced ELL, one
// warp per 32-row slice, coalesced) is loaded once and applied to both vectors,
// so A is read s times per block, not 2s-1.
// The GPU has no room to keep A on chip across steps for the large
// workloads. This step is FP64-bound on GB300, so re-reading A costs no time.
//
// The basis coefficients are folded into the operator beforehand. A is kept
// as D + O, and step j uses Dt_j = (D - theta_j)/gamma_j and O/gamma_j, so a
// row costs nnz_row + 1 FP64 instructions rather than nnz_row + 3. That spends
// HBM capacity, of which a GB300 has plenty, to save FP64 work, which it lacks.
#include "ascg_common.cuh"

namespace ascg {

namespace {

__global__ void __launch_bounds__(kSpmvRows) mpk_split_step_kernel(DevSell O, const double* __restrict__ oval,
                                                                   const double* __restrict__ dtil, double sig,
                                                                   int use_sig, double* __restrict__ Y, int64_t ldY,
                                                                   int j, int do_p, int do_r) {
  const int64_t row = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  if (row >= O.n) return;
  const double* pj = Y + (int64_t)(2 * j) * ldY;
  const double* rj = Y + (int64_t)(2 * j + 1) * ldY;
  const int64_t sl = row >> 5;
  const int l = (int)(row & 31);
  const int64_t b = O.ptr[sl];
  const int width = (int)((O.ptr[sl + 1] - b) >> 5);
  const double* v = oval + b + l;
  const int32_t* c = O.col + b + l;
  const double dt = dtil[row];
  double tp = dt * pj[row];
  if (do_r) {
    double tr = dt * rj[row];
    for (int k = 0; k < width; ++k) {
      const double a = __ldg(v + kSlice * k);
      const int cc = __ldg(c + kSlice * k);
      tp = fma(a, __ldg(pj + cc), tp);
      tr = fma(a, __ldg(rj + cc), tr);
    }
    // rho_{j+1} = (Dt_j + Ot_j) rho_j - sig_j rho_{j-1}
    if (use_sig) {  // integer test: a double compare would take an FP64 issue slot per row
      tp = fma(-sig, Y[(int64_t)(2 * j - 2) * ldY + row], tp);
      tr = fma(-sig, Y[(int64_t)(2 * j - 1) * ldY + row], tr);
    }
    Y[(int64_t)(2 * j + 3) * ldY + row] = tr;
  } else {
    for (int k = 0; k < width; ++k) tp = fma(__ldg(v + kSlice * k), __ldg(pj + __ldg(c + kSlice * k)), tp);
    if (use_sig) tp = fma(-sig, Y[(int64_t)(2 * j - 2) * ldY + row], tp);
  }
  if (do_p) Y[(int64_t)(2 * j + 2) * ldY + row] = tp;
}

__global__ void shift_scale_kernel(const double* __restrict__ src, int64_t n, double theta, double scale,
                                   double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (src[i] - theta) * scale;
}

// x += Y x', r = Y r', p = Y p' over the first w columns (eq. coords).
// Each thread reads its whole row of Y before writing, so r and p may alias
// columns 1 and 0 of Y.
template <int W>
__global__ void __launch_bounds__(256) recover_kernel(int64_t n, const double* Y, int64_t ldY,
                                                      const double* __restrict__ coords, double* x, double* r,
                                                      double* p) {
  __shared__ double cx[W], cr[W], cp[W];
  if (threadIdx.x < W) {
    cx[threadIdx.x] = coords[threadIdx.x];
    cr[threadIdx.x] = coords[W + threadIdx.x];
    cp[threadIdx.x] = coords[2 * W + threadIdx.x];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[W];
#pragma unroll
    for (int c = 0; c < W; ++c) y[c] = Y[(int64_t)c * ldY + i];
    double sx = 0.0, sr = 0.0, sp = 0.0;
#pragma unroll
    for (int c = 0; c < W; ++c) {
      sx = fma(y[c], cx[c], sx);
      sr = fma(y[c], cr[c], sr);
      sp = fma(y[c], cp[c], sp);
    }
    x[i] = x[i] + sx;
    r[i] = sr;
    p[i] = sp;
  }
}

template <int W>
cudaError_t recover_w(int64_t n, const double* Y, int64_t ldY, const double* coords, double* x, double* r,
                      double* p, cudaStream_t s) {
  recover_kernel<W><<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(n, Y, ldY, coords, x, r, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mpk_split_step(const DevSplit& O, const StepOp& op, double* Y, int64_t ldY, int j, int do_p,
                                  int do_r, cudaStream_t s) {
  const int g = (int)((O.O.n + kSpmvRows - 1) / kSpmvRows);
  const int use_sig = (op.sig != 0.0 && j >= 1) ? 1 : 0;
  mpk_split_step_kernel<<<g, kSpmvRows, 0, s>>>(O.O, op.oval, op.dtil, op.sig, use_sig, Y, ldY, j, do_p, do_r);
  return cudaGetLastError();
}

cudaError_t launch_shift_scale(const double* src, int64_t n, double theta, double scale, double* dst,
                               cudaStream_t s) {
  shift_scale_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(src, n, theta, scale, dst);
  return cudaGetLastError();
}

cudaError_t launch_recover(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* x,
                           double* r, double* p, cudaStream_t s) {
  switch (w) {
#define ASCG_RW(W) \
  case W:          \
    return recover_w<W>(n, Y, ldY, coords, x, r, p, s);
    ASCG_RW(1) ASCG_RW(3) ASCG_RW(5) ASCG_RW(7) ASCG_RW(9) ASCG_RW(11) ASCG_RW(13) ASCG_RW(15) ASCG_RW(17)
    ASCG_RW(19) ASCG_RW(21) ASCG_RW(23) ASCG_RW(25) ASCG_RW(27) ASCG_RW(29) ASCG_RW(31) ASCG_RW(33)
#undef ASCG_RW
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ascg
