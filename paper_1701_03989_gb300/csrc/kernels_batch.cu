// Many independent systems advancing block by block in lockstep (batched
// solves and the solve server). Each system keeps its own operator, basis,
// x and b; a device table of descriptors (SysDesc) points at them. Work is
// cut into row items of one system each (RowItem: up to 256 rows starting on
// a 32-row slice), so one launch serves every system and adding or retiring
// a system only changes the tables. A kernel reads nothing of the other
// systems, so each system's result is the same alone and in any mix.
#include "ascg_common.cuh"

namespace ascg {
namespace {

__device__ __forceinline__ bool item_row(const RowItem* items, int64_t* row, int* sys) {
  const RowItem it = items[blockIdx.x];
  if ((int)threadIdx.x >= it.nrows) return false;
  *row = it.row0 + threadIdx.x;
  *sys = it.sys;
  return true;
}

// Matrix powers step j in the monomial basis (theta = sigma = 0, gamma = 1;
// eq. (polybasiscg)) for every system q with j < sys_steps[q]: column 2j+2 =
// A column 2j and, while j + 1 < sbar_q, column 2j+3 = A column 2j+1, A = D + O.
__global__ void __launch_bounds__(kRowItem) mpk_items_kernel(const SysDesc* __restrict__ descs,
                                                             const RowItem* __restrict__ items,
                                                             const int* __restrict__ sys_steps, int j) {
  int64_t row;
  int q;
  if (!item_row(items, &row, &q)) return;
  const int steps = sys_steps[q];
  if (j >= steps) return;  // uniform over the CTA
  const SysDesc d = descs[q];
  const double* pj = d.Y + (int64_t)(2 * j) * d.ldY;
  const double* rj = d.Y + (int64_t)(2 * j + 1) * d.ldY;
  const int64_t sl = row >> 5;
  const int l = (int)(row & 31);
  const int64_t b = d.o_ptr[sl];
  const int width = (int)((d.o_ptr[sl + 1] - b) >> 5);
  const double* v = d.o_val + b + l;
  const int32_t* c = d.o_col + b + l;
  const double dg = d.diag[row];
  double tp = dg * pj[row];
  if (j + 1 < steps) {
    double tr = dg * rj[row];
    for (int k = 0; k < width; ++k) {
      const double a = __ldg(v + kSlice * k);
      const int cc = __ldg(c + kSlice * k);
      tp = fma(a, __ldg(pj + cc), tp);
      tr = fma(a, __ldg(rj + cc), tr);
    }
    d.Y[(int64_t)(2 * j + 3) * d.ldY + row] = tr;
  } else {
    for (int k = 0; k < width; ++k) tp = fma(__ldg(v + kSlice * k), __ldg(pj + __ldg(c + kSlice * k)), tp);
  }
  d.Y[(int64_t)(2 * j + 2) * d.ldY + row] = tp;
}

// Residual of the systems with sel[q] != 0: into columns 1 (r) and 0 (p) of Y
// (setup), or into column 2 (true residual at the end).
__global__ void __launch_bounds__(kRowItem) residual_items_kernel(const SysDesc* __restrict__ descs,
                                                                  const RowItem* __restrict__ items,
                                                                  const int* __restrict__ sel, int into_col2) {
  int64_t row;
  int q;
  if (!item_row(items, &row, &q)) return;
  if (!sel[q]) return;
  const SysDesc d = descs[q];
  const int64_t sl = row >> 5;
  const int l = (int)(row & 31);
  const int64_t o = d.o_ptr[sl];
  const int width = (int)((d.o_ptr[sl + 1] - o) >> 5);
  double ax = d.diag[row] * d.x[row];
  for (int k = 0; k < width; ++k)
    ax = fma(__ldg(d.o_val + o + kSlice * k + l), d.x[__ldg(d.o_col + o + kSlice * k + l)], ax);
  const double rr = d.b[row] - ax;
  if (into_col2) {
    d.Y[2 * d.ldY + row] = rr;
  } else {
    d.Y[d.ldY + row] = rr;
    d.Y[row] = rr;
  }
}

// out[q] = sum of squares of a vector of each selected system (one CTA per
// selected system; fixed order: strided thread sums, then a fixed tree).
// which: 0 = b, 1 = Y column 1 (r), 2 = Y column 2.
__global__ void __launch_bounds__(1024) seg_sumsq_kernel(const SysDesc* __restrict__ descs,
                                                         const int* __restrict__ list, int which,
                                                         double* __restrict__ out) {
  const int q = list[blockIdx.x];
  const SysDesc d = descs[q];
  const double* v = which == 0 ? d.b : d.Y + (int64_t)which * d.ldY;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < d.n; i += 1024) s = fma(v[i], v[i], s);
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = warp_sum(red[threadIdx.x]);
    if (threadIdx.x == 0) out[q] = s;
  }
}

// x += Y x', r = Y r', p = Y p' (eq. (coords)) for every active system
// (w_q = sys_w[q] > 0); its coordinates sit at coords + q * c_stride as x'[w_q],
// r'[w_q], p'[w_q]. A thread reads its whole row of Y before writing r and p
// into columns 1 and 0.
template <int W>
__global__ void __launch_bounds__(kRowItem) recover_items_kernel(const SysDesc* __restrict__ descs,
                                                                 const RowItem* __restrict__ items,
                                                                 const int* __restrict__ sys_w,
                                                                 const double* __restrict__ coords, int64_t c_stride) {
  int64_t row;
  int q;
  if (!item_row(items, &row, &q)) return;
  const int w = sys_w[q];
  if (w == 0) return;  // uniform over the CTA
  const SysDesc d = descs[q];
  const double* cq = coords + (int64_t)q * c_stride;
  double y[W];
#pragma unroll
  for (int c = 0; c < W; ++c) y[c] = c < w ? d.Y[(int64_t)c * d.ldY + row] : 0.0;
  double sx = 0.0, sr = 0.0, sp = 0.0;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    if (c < w) {
      sx = fma(y[c], __ldg(cq + c), sx);
      sr = fma(y[c], __ldg(cq + w + c), sr);
      sp = fma(y[c], __ldg(cq + 2 * w + c), sp);
    }
  }
  d.x[row] += sx;
  d.Y[d.ldY + row] = sr;
  d.Y[row] = sp;
}

// v[i] in [-1, 1) from a 64-bit mix of (seed, i) (the SplitMix64 finaliser of
// Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): synthetic data for the autotuner's timings.
__global__ void fill_uniform_kernel(double* __restrict__ v, int64_t count, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(int64_t)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

}  // namespace

cudaError_t launch_fill_uniform(double* v, int64_t count, uint64_t seed, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  fill_uniform_kernel<<<grid_for(count, 256, 152 * 16), 256, 0, s>>>(v, count, seed);
  return cudaGetLastError();
}

cudaError_t launch_mpk_items(const SysDesc* descs, const RowItem* items, int nitems, const int* sys_steps, int j,
                             cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  mpk_items_kernel<<<nitems, kRowItem, 0, s>>>(descs, items, sys_steps, j);
  return cudaGetLastError();
}

cudaError_t launch_residual_items(const SysDesc* descs, const RowItem* items, int nitems, const int* sel,
                                  int into_col2, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  residual_items_kernel<<<nitems, kRowItem, 0, s>>>(descs, items, sel, into_col2);
  return cudaGetLastError();
}

cudaError_t launch_seg_sumsq(const SysDesc* descs, const int* list, int nlist, int which, double* out,
                             cudaStream_t s) {
  if (nlist < 1) return cudaSuccess;
  seg_sumsq_kernel<<<nlist, 1024, 0, s>>>(descs, list, which, out);
  return cudaGetLastError();
}

cudaError_t launch_recover_items(int W, const SysDesc* descs, const RowItem* items, int nitems, const int* sys_w,
                                 const double* coords, int64_t c_stride, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  switch (W) {
#define ASCG_RB(WW)                                                                             \
  case WW:                                                                                      \
    recover_items_kernel<WW><<<nitems, kRowItem, 0, s>>>(descs, items, sys_w, coords, c_stride); \
    return cudaGetLastError();
    ASCG_RB(3) ASCG_RB(5) ASCG_RB(7) ASCG_RB(9) ASCG_RB(11) ASCG_RB(13) ASCG_RB(15) ASCG_RB(17) ASCG_RB(19)
    ASCG_RB(21) ASCG_RB(23) ASCG_RB(25) ASCG_RB(27) ASCG_RB(29) ASCG_RB(31) ASCG_RB(33)
#undef ASCG_RB
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ascg
