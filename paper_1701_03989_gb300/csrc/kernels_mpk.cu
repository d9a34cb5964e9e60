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
// row costs nnz_row + 1 FP64 instructions rather than nnz_row + 3 (nnz_row
// when sig_j = 1: the sigma term is the start value of the sum). That spends
// HBM capacity, of which a GB300 has plenty, to save FP64 work, which it lacks.
#include "ascg_common.cuh"

namespace ascg {

namespace {

__device__ __forceinline__ unsigned biased_exp(double v) { return ((unsigned)__double2hiint(v) >> 20) & 0x7ffu; }

// emax_part (optional, int[kMaxW][emax_ld]): lane 0 of each warp stores the
// warp's largest biased exponent of each column written (and, for j = 0, of
// the input columns 0 and 1) at emax_part[col * emax_ld + warp]; plain stores,
// no synchronisation. A warp past the last 32-row slice stores nothing: a row
// holds the ceil(n / 32) slices rounded up to 4, fewer than the grid's warps
// when n is not a multiple of 256, and such a store would land on the next
// column's first slices. emax_reduce_kernel folds them per column for the
// tensor-core Gram.
// emax_part (or nullptr): record exponents. R: also the R chain (every step of
// a block but the last). The entries of a row go in pairs: both index and value
// loads, then the four gathers, then the FMAs, so each warp keeps more loads
// in flight (the kernel waits mostly on its gathers). The chains and the sigma
// mode are compile-time parameters: with both as runtime flags the same step
// took 67.5 us instead of 57.1 us at 128^3. 6 CTAs per SM (up to 40 registers).
// The exponent work always runs (a few integer operations per row); a
// variant without it measured slower (63.5 us).
// SIG: 0 no sigma term (j = 0 or sig_j = 0); 1 sig_j = 1 exactly (the
// Chebyshev basis, where sigma_{j-1} = gamma_j); 2 any other sig_j. The sum
// starts from -sig_j rho_{j-1} and takes the diagonal term as its first FMA,
// so with SIG = 1 a row costs nnz_row FP64 instructions per chain.
template <int SIG, bool R>
__global__ void __launch_bounds__(kSpmvRows, 6)
    mpk_split_step_kernel(DevSell O, const double* __restrict__ oval, const double* __restrict__ dtil, double sig,
                          double* __restrict__ Y, int64_t ldY, int j, int* emax_part, int64_t emax_ld,
                          const int* __restrict__ gate) {
  pdl_wait();     // the previous step's columns (and the gate) are written by the kernel before
  pdl_release();  // the next step may be scheduled once every CTA of this one has started
  if (gate && !*gate) return;  // uniform: a block enqueued ahead that has nothing to do
  const int64_t row = (int64_t)blockIdx.x * kSpmvRows + threadIdx.x;
  unsigned e_op = 0, e_or = 0;
  if (row < O.n) {
    const double* pj = Y + (int64_t)(2 * j) * ldY;
    const double* rj = Y + (int64_t)(2 * j + 1) * ldY;
    const int64_t sl = row >> 5;
    const int l = (int)(row & 31);
    const int64_t b = O.ptr[sl];
    const int width = (int)((O.ptr[sl + 1] - b) >> 5);
    const double* v = oval + b + l;
    const int32_t* c = O.col + b + l;
    const double dt = dtil[row];
    // rho_{j+1} = (Dt_j + Ot_j) rho_j - sig_j rho_{j-1}
    double tp, tr = 0.0;
    if (SIG == 0) {
      tp = dt * pj[row];
      if (R) tr = dt * rj[row];
    } else {
      const double zp = Y[(int64_t)(2 * j - 2) * ldY + row];
      tp = fma(dt, pj[row], SIG == 1 ? -zp : -sig * zp);
      if (R) {
        const double zr = Y[(int64_t)(2 * j - 1) * ldY + row];
        tr = fma(dt, rj[row], SIG == 1 ? -zr : -sig * zr);
      }
    }
    int k = 0;
    for (; k + 2 <= width; k += 2) {
      const int c0 = __ldcs(c + kSlice * k), c1 = __ldcs(c + kSlice * (k + 1));
      const double a0 = __ldcs(v + kSlice * k), a1 = __ldcs(v + kSlice * (k + 1));
      const double p0 = __ldg(pj + c0), p1 = __ldg(pj + c1);
      if (R) {
        const double r0 = __ldg(rj + c0), r1 = __ldg(rj + c1);
        tp = fma(a0, p0, tp);
        tr = fma(a0, r0, tr);
        tp = fma(a1, p1, tp);
        tr = fma(a1, r1, tr);
      } else {
        tp = fma(a0, p0, tp);
        tp = fma(a1, p1, tp);
      }
    }
    if (k < width) {
      const double a = __ldcs(v + kSlice * k);
      const int cc = __ldcs(c + kSlice * k);
      tp = fma(a, __ldg(pj + cc), tp);
      if (R) tr = fma(a, __ldg(rj + cc), tr);
    }
    Y[(int64_t)(2 * j + 2) * ldY + row] = tp;
    if (R) Y[(int64_t)(2 * j + 3) * ldY + row] = tr;
    e_op = biased_exp(tp);
    if (R) e_or = biased_exp(tr);
  }
  const int64_t wg = ((int64_t)blockIdx.x * kSpmvRows + threadIdx.x) >> 5;
  if (!emax_part || wg * kSlice >= O.n) return;  // uniform over the warp
  // the warp's rows share one slice; lanes past n contribute 0
  e_op = __reduce_max_sync(0xffffffffu, e_op);
  e_or = __reduce_max_sync(0xffffffffu, e_or);
  if ((threadIdx.x & 31) == 0) {
    emax_part[(int64_t)(2 * j + 2) * emax_ld + wg] = (int)e_op;
    if (R) emax_part[(int64_t)(2 * j + 3) * emax_ld + wg] = (int)e_or;
  }
  if (j == 0) {
    // inputs p and r (columns 0, 1): reloaded here (cache hits) so that nothing
    // extra stays live across the loop above
    unsigned e_ip = 0, e_ir = 0;
    if (row < O.n) {
      e_ip = biased_exp(__ldcg(Y + row));
      e_ir = biased_exp(__ldcg(Y + ldY + row));
    }
    e_ip = __reduce_max_sync(0xffffffffu, e_ip);
    e_ir = __reduce_max_sync(0xffffffffu, e_ir);
    if ((threadIdx.x & 31) == 0) {
      emax_part[wg] = (int)e_ip;
      emax_part[emax_ld + wg] = (int)e_ir;
    }
  }
}

// col_emax[c] = max over the warp entries of column c: one CTA of 1024 threads
// per column, 16-byte loads, four in flight per thread. emax_ld is a multiple
// of 4 and entries past the warp count are zero.
__global__ void __launch_bounds__(1024) emax_reduce_kernel(const int* __restrict__ emax_part, int64_t emax_ld,
                                                           int* __restrict__ col_emax, const int* __restrict__ gate) {
  pdl_wait();
  pdl_release();
  if (gate && !*gate) return;
  const int c = blockIdx.x;
  const int4* src = reinterpret_cast<const int4*>(emax_part + (int64_t)c * emax_ld);
  const int64_t n4 = emax_ld / 4;
  int m0 = 0, m1 = 0, m2 = 0, m3 = 0;
  int64_t k = threadIdx.x;
  for (; k + 3072 < n4; k += 4096) {
    const int4 a = __ldcs(src + k), b = __ldcs(src + k + 1024), d = __ldcs(src + k + 2048), e = __ldcs(src + k + 3072);
    m0 = max(m0, max(max(a.x, a.y), max(a.z, a.w)));
    m1 = max(m1, max(max(b.x, b.y), max(b.z, b.w)));
    m2 = max(m2, max(max(d.x, d.y), max(d.z, d.w)));
    m3 = max(m3, max(max(e.x, e.y), max(e.z, e.w)));
  }
  for (; k < n4; k += 1024) {
    const int4 a = __ldcs(src + k);
    m0 = max(m0, max(max(a.x, a.y), max(a.z, a.w)));
  }
  int m = __reduce_max_sync(0xffffffffu, max(max(m0, m1), max(m2, m3)));
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = __reduce_max_sync(0xffffffffu, red[threadIdx.x]);
    if (threadIdx.x == 0) col_emax[c] = m;
  }
}

__global__ void shift_scale_kernel(const double* __restrict__ src, int64_t n, double theta, double scale,
                                   double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (src[i] - theta) * scale;
}

// x += Y x', r = Y r', p = Y p' over the first w columns (eq. coords).
// Each thread reads its whole row of Y before writing, so r and p may alias
// columns 1 and 0 of Y.
//
// All recovery kernels load a row's entries in groups of kRecGroup columns
// (streaming loads, which also keep the compiler from hoisting every load of
// the row) and add them in column order: the same sums (and bits) in every
// kernel, with about 40 registers, so 6 CTAs fit on an SM. Holding the whole
// row in registers (166 for W = 33) left one CTA per SM and took 279 us
// instead of 238 us for r and p at 128^3.
constexpr int kRecGroup = 8;

template <int W>
__global__ void __launch_bounds__(256, 6) recover_kernel(int64_t n, const double* Y, int64_t ldY,
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
    double sx = 0.0, sr = 0.0, sp = 0.0;
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += kRecGroup) {
      double y[kRecGroup];
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) y[q] = __ldcs(Y + (int64_t)(c0 + q) * ldY + i);
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) {
          sx = fma(y[q], cx[c0 + q], sx);
          sr = fma(y[q], cr[c0 + q], sr);
          sp = fma(y[q], cp[c0 + q], sp);
        }
    }
    x[i] = x[i] + sx;
    r[i] = sr;
    p[i] = sp;
  }
}

// CTAs for a grid-stride recovery over n rows: one row per thread up to 64
// CTAs per SM.
inline int rec_grid(int64_t n) { return grid_for(n, 256, 152 * 64); }

template <int W>
cudaError_t recover_w(int64_t n, const double* Y, int64_t ldY, const double* coords, double* x, double* r,
                      double* p, cudaStream_t s) {
  recover_kernel<W><<<rec_grid(n), 256, 0, s>>>(n, Y, ldY, coords, x, r, p);
  return cudaGetLastError();
}

// The recovery split in two, with the same sums as recover_kernel (so the
// same bits): r = Y r', p = Y p' (written to another buffer: Y stays intact),
// and x += Y x', which the next block does not need and which the solver
// runs later, beside the next block's condition estimates and controller.
template <int W>
__global__ void __launch_bounds__(256, 6) recover_rp_kernel(int64_t n, const double* __restrict__ Y, int64_t ldY,
                                                            const double* __restrict__ coords,
                                                            double* __restrict__ r, double* __restrict__ p,
                                                            const int* __restrict__ gate) {
  if (gate && !*gate) return;
  __shared__ double cr[W], cp[W];
  if (threadIdx.x < W) {
    cr[threadIdx.x] = coords[W + threadIdx.x];
    cp[threadIdx.x] = coords[2 * W + threadIdx.x];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sr = 0.0, sp = 0.0;
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += kRecGroup) {
      double y[kRecGroup];
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) y[q] = __ldcs(Y + (int64_t)(c0 + q) * ldY + i);
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) {
          sr = fma(y[q], cr[c0 + q], sr);
          sp = fma(y[q], cp[c0 + q], sp);
        }
    }
    r[i] = sr;
    p[i] = sp;
  }
}

// x += Y x'. One CTA per SM at most, each reserving most of the SM's shared
// memory (kXReserve of the 228 KB): the CTAs then never share an SM with the
// condition estimate and controller CTAs (about 11 KB each), whose FP64 issue
// they would otherwise slow.
constexpr int kXThreads = 512;
constexpr int kXReserve = 220 * 1024;
template <int W>
__global__ void __launch_bounds__(kXThreads, 1) recover_x_kernel(int64_t n, const double* __restrict__ Y,
                                                                 int64_t ldY, const double* __restrict__ coords,
                                                                 double* __restrict__ x, const int* __restrict__ gate) {
  if (gate && !*gate) return;
  __shared__ double cx[W];
  if (threadIdx.x < W) cx[threadIdx.x] = coords[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sx = 0.0;
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += kRecGroup) {
      double y[kRecGroup];
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) y[q] = __ldcs(Y + (int64_t)(c0 + q) * ldY + i);
#pragma unroll
      for (int q = 0; q < kRecGroup; ++q)
        if (c0 + q < W) sx = fma(y[q], cx[c0 + q], sx);
    }
    x[i] = x[i] + sx;
  }
}

template <int W>
cudaError_t recover_split_w(int64_t n, const double* Y, int64_t ldY, const double* coords, double* x, double* r,
                            double* p, int x_ctas, cudaStream_t s, const int* gate) {
  if (x) {
    static std::atomic<uint64_t> smem_set{0};  // one flag set per instance
    const cudaError_t e = smem_limit_once(smem_set, recover_x_kernel<W>, kXReserve);
    if (e != cudaSuccess) return e;
    recover_x_kernel<W><<<x_ctas, kXThreads, kXReserve, s>>>(n, Y, ldY, coords, x, gate);
  } else {
    recover_rp_kernel<W><<<rec_grid(n), 256, 0, s>>>(n, Y, ldY, coords, r, p, gate);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mpk_split_step(const DevSplit& O, const StepOp& op, double* Y, int64_t ldY, int j, int do_p,
                                  int do_r, int* emax_part, int64_t emax_ld, cudaStream_t s, const int* gate) {
  if (!do_p) return cudaErrorInvalidValue;  // every step forms the P column
  const int g = (int)((O.O.n + kSpmvRows - 1) / kSpmvRows);
  const int sig_mode = (op.sig == 0.0 || j < 1) ? 0 : (op.sig == 1.0 ? 1 : 2);
#define ASCG_MPK(S, R)                                                                                        \
  return launch_pdl(mpk_split_step_kernel<S, R>, g, kSpmvRows, s, O.O, op.oval, op.dtil, op.sig, Y, ldY, j, emax_part, \
                    emax_ld, gate)
  if (do_r) {
    if (sig_mode == 0) ASCG_MPK(0, true);
    else if (sig_mode == 1) ASCG_MPK(1, true);
    else ASCG_MPK(2, true);
  } else {
    if (sig_mode == 0) ASCG_MPK(0, false);
    else if (sig_mode == 1) ASCG_MPK(1, false);
    else ASCG_MPK(2, false);
  }
#undef ASCG_MPK
  return cudaGetLastError();
}

cudaError_t launch_emax_reduce(const int* emax_part, int64_t emax_ld, int64_t n, int w, int* col_emax,
                               cudaStream_t s, const int* gate) {
  (void)n;
  return launch_pdl(emax_reduce_kernel, w, 1024, s, emax_part, emax_ld, col_emax, gate);
}

cudaError_t launch_shift_scale(const double* src, int64_t n, double theta, double scale, double* dst,
                               cudaStream_t s) {
  shift_scale_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(src, n, theta, scale, dst);
  return cudaGetLastError();
}

cudaError_t launch_recover_rp(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* r,
                              double* p, cudaStream_t s, const int* gate) {
  switch (w) {
#define ASCG_RS(W) \
  case W:          \
    return recover_split_w<W>(n, Y, ldY, coords, nullptr, r, p, 0, s, gate);
    ASCG_RS(1) ASCG_RS(3) ASCG_RS(5) ASCG_RS(7) ASCG_RS(9) ASCG_RS(11) ASCG_RS(13) ASCG_RS(15) ASCG_RS(17)
    ASCG_RS(19) ASCG_RS(21) ASCG_RS(23) ASCG_RS(25) ASCG_RS(27) ASCG_RS(29) ASCG_RS(31) ASCG_RS(33)
#undef ASCG_RS
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_recover_x(int64_t n, int w, const double* Y, int64_t ldY, const double* coords, double* x,
                             int ctas, cudaStream_t s, const int* gate) {
  if (ctas < 1) ctas = 1;
  switch (w) {
#define ASCG_RX(W) \
  case W:          \
    return recover_split_w<W>(n, Y, ldY, coords, x, nullptr, nullptr, ctas, s, gate);
    ASCG_RX(1) ASCG_RX(3) ASCG_RX(5) ASCG_RX(7) ASCG_RX(9) ASCG_RX(11) ASCG_RX(13) ASCG_RX(15) ASCG_RX(17)
    ASCG_RX(19) ASCG_RX(21) ASCG_RX(23) ASCG_RX(25) ASCG_RX(27) ASCG_RX(29) ASCG_RX(31) ASCG_RX(33)
#undef ASCG_RX
    default:
      return cudaErrorInvalidValue;
  }
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
