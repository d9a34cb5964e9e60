// Gram matrix G = Y^T Y of the s-step basis (Sec. 2.1; Alg. 4 "Compute G").
//
// This is the largest FP64 cost of a block: w(w+1)/2 fused multiply-adds per
// row (561 at w = 33), against about 2 * (2s-1) * nnz/n for the matrix powers
// kernel. GB300 runs FP64 at one warp instruction per ~20 SM cycles, and DMMA
// (mma.sync m8n8k4 f64) shares that pipe at the same rate. So the Gram stays
// on CUDA cores, and the design goal is to keep every FP64 lane busy on a
// distinct product.
//
// Mapping: a CTA owns a contiguous range of 32-row chunks. Each chunk of Y
// (w columns x 32 rows) goes to shared memory. Lane l of every warp works on
// row l of the chunk. Warp g owns the upper-triangle pairs p = g, g + 16,
// g + 32, ..., and accumulates y_a * y_b for its pairs in registers. After the
// range, each warp reduces its accumulators across lanes (fixed shuffle tree)
// and writes one partial per pair. A second kernel adds the partials of all
// CTAs in index order. Results are bitwise reproducible for a given n, w and
// grid.
#include "ascg_common.cuh"

namespace ascg {

namespace {

constexpr int kGramWarps = 16;
constexpr int kGramThreads = kGramWarps * 32;
constexpr int kChunk = 32;  // rows per chunk = lanes

// SM count of each device (0: not looked up yet), for devices 0..63.
std::atomic<int> g_gram_grid[64];

// Partial Gram of 32-row chunks [c0, c1) of rows [0, n) of Y into out[NP]
// (row-major upper triangle). Called by every thread of a CTA of kGramThreads.
// Moment p of the monomial basis' Gram (interleaved columns: P_j = 2j,
// R_j = 2j + 1; S = (W - 1)/2), the pair of columns whose dot product gives
// it, and its output slot:
//   p = 0 .. 2S        mu_pp[k] = <P_floor(k/2), P_ceil(k/2)>, k = p
//   p = 2S+1 .. 4S     mu_pr[k] = <P_ceil(k/2), R_floor(k/2)>, k = p - 2S - 1
//   p = 4S+1 .. 6S-1   mu_rr[k] = <R_floor(k/2), R_ceil(k/2)>, k = p - 4S - 1
// slot = family * kMomFam + k.
__device__ __forceinline__ void moment_pair(int p, int S, int* a, int* b, int* slot) {
  if (p <= 2 * S) {
    const int k = p;
    *a = 2 * (k / 2);
    *b = 2 * ((k + 1) / 2);
    *slot = k;
  } else if (p <= 4 * S) {
    const int k = p - 2 * S - 1;
    *a = 2 * ((k + 1) / 2);
    *b = 2 * (k / 2) + 1;
    *slot = kMomFam + k;
  } else {
    const int k = p - 4 * S - 1;
    *a = 2 * (k / 2) + 1;
    *b = 2 * ((k + 1) / 2) + 1;
    *slot = 2 * kMomFam + k;
  }
}

// With G pair groups, this CTA takes the pairs p = g, g + G, g + 2G, ... only
// (group g of G) and writes just those; a pair's arithmetic is the same for
// any G. MOM: the 6S moment pairs of moment_pair instead of all W(W+1)/2,
// written at their slots (out holds kMomSlots).
template <int W, bool MOM = false>
__device__ __forceinline__ void gram_chunks(int64_t n, const double* __restrict__ Y, int64_t ldY, int64_t c0,
                                            int64_t c1, double* __restrict__ out, int g = 0, int G = 1) {
  constexpr int NP = MOM ? 3 * (W - 1) : W * (W + 1) / 2;
  constexpr int PPW = (NP + kGramWarps - 1) / kGramWarps;
  constexpr int ELEMS = W * kChunk;
  constexpr int LPT = (ELEMS + kGramThreads - 1) / kGramThreads;  // loads per thread per chunk
  __shared__ double tile[2][W][kChunk];
  __shared__ unsigned short pab[kGramWarps][PPW];  // a | b << 8 for each of the warp's pairs
  __shared__ unsigned char pslot[MOM ? kGramWarps : 1][MOM ? PPW : 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // pair p in row-major upper-triangle order: (0,0), (0,1), ..., (0,W-1), (1,1), ...
  for (int k = lane; k < PPW; k += 32) {
    const int p = g + G * (warp + kGramWarps * k);
    int a = 0, b = 0;
    if (p < NP) {
      if (MOM) {
        int sl = 0;
        moment_pair(p, (W - 1) / 2, &a, &b, &sl);
        pslot[MOM ? warp : 0][MOM ? k : 0] = (unsigned char)sl;
      } else {
        int rem = p;
        while (rem >= W - a) {
          rem -= W - a;
          ++a;
        }
        b = a + rem;
      }
    }
    pab[warp][k] = (unsigned short)(a | (b << 8));
  }


  double acc[PPW];
#pragma unroll
  for (int k = 0; k < PPW; ++k) acc[k] = 0.0;

  double pre[LPT];
  auto load = [&](int64_t c) {
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
      const int e = threadIdx.x + i * kGramThreads;
      double v = 0.0;
      if (e < ELEMS) {
        const int col = e / kChunk, r = e % kChunk;
        const int64_t row = c * kChunk + r;
        if (row < n) v = __ldcs(Y + (int64_t)col * ldY + row);
      }
      pre[i] = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
      const int e = threadIdx.x + i * kGramThreads;
      if (e < ELEMS) (&tile[buf][0][0])[e] = pre[i];
    }
  };

  if (c0 < c1) {
    load(c0);
    store(0);
  }
  __syncthreads();
  for (int64_t c = c0; c < c1; ++c) {
    const int buf = (int)((c - c0) & 1);
    const bool more = c + 1 < c1;
    if (more) load(c + 1);
    const double* t = &tile[buf][0][0];
#pragma unroll
    for (int k = 0; k < PPW; ++k) {
      if (g + G * (warp + kGramWarps * k) < NP) {
        const unsigned ab = pab[warp][k];
        const double ya = t[(ab & 0xff) * kChunk + lane];
        const double yb = t[(ab >> 8) * kChunk + lane];
        acc[k] = fma(ya, yb, acc[k]);
      }
    }
    if (more) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PPW; ++k) {
    const int p = g + G * (warp + kGramWarps * k);
    if (p >= NP) break;  // uniform over the warp
    const double v = warp_sum(acc[k]);
    if (lane == 0) out[MOM ? (int)pslot[MOM ? warp : 0][MOM ? k : 0] : p] = v;
  }
}

template <int W, bool MOM = false>
__global__ void __launch_bounds__(kGramThreads, 1) gram_partial_kernel(int64_t n, const double* __restrict__ Y,
                                                                        int64_t ldY, double* __restrict__ partials,
                                                                        const int* __restrict__ gate) {
  if (gate && !*gate) return;  // uniform: a block enqueued ahead that has nothing to do
  constexpr int NP = MOM ? kMomSlots : W * (W + 1) / 2;
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  gram_chunks<W, MOM>(n, Y, ldY, nchunks * blockIdx.x / gridDim.x, nchunks * (blockIdx.x + 1) / gridDim.x,
                      partials + (int64_t)blockIdx.x * NP);
}

// Batched solves: CTA (q, g) takes pair group g of item q (rows [row0, row0 +
// nrows) of one system). Items depend only on the system's own size, and a
// pair's sum does not depend on the number of groups, so a system's Gram is
// the same alone and in any batch. Items of inactive systems (sys_w 0) skip.
template <int W, bool MOM = false>
__global__ void __launch_bounds__(kGramThreads, 1) gram_items_kernel(const SysDesc* __restrict__ descs,
                                                                      const GramItem* __restrict__ items,
                                                                      const int* __restrict__ sys_w,
                                                                      double* __restrict__ partials) {
  constexpr int NP = MOM ? kMomSlots : W * (W + 1) / 2;
  const GramItem it = items[blockIdx.x];
  if (sys_w[it.sys] == 0) return;  // uniform over the CTA
  const SysDesc& d = descs[it.sys];
  gram_chunks<W, MOM>(it.nrows, d.Y + it.row0, d.ldY, 0, (it.nrows + kChunk - 1) / kChunk,
                      partials + (int64_t)blockIdx.x * NP, (int)blockIdx.y, (int)gridDim.y);
}

// G (w x w, interleaved order) from the moments mu[family * kMomFam + k]:
// entry (2i + alpha, 2j + beta) is mu_pp, mu_pr or mu_rr at k = i + j.
__device__ __forceinline__ void moments_to_gram(const double* mu, int w, double* G) {
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int a = e / w, b = e % w;
    const int fam = (a & 1) + (b & 1);  // 0: P P, 1: P R or R P, 2: R R
    G[e] = mu[fam * kMomFam + (a >> 1) + (b >> 1)];
  }
}

// The moments of one system from nparts partials (kMomSlots each), each
// summed over the partials in index order, then G.
__global__ void __launch_bounds__(128) gram_moment_finalize_kernel(int w, const double* __restrict__ partials,
                                                                   int nparts, double* __restrict__ G,
                                                                   const int* __restrict__ gate) {
  if (gate && !*gate) return;
  __shared__ double mu[kMomSlots];
  const int S = (w - 1) / 2;
  for (int sl = threadIdx.x; sl < kMomSlots; sl += blockDim.x) {
    const int fam = sl / kMomFam, k = sl % kMomFam;
    const int kmax = fam == 0 ? 2 * S : (fam == 1 ? 2 * S - 1 : 2 * S - 2);
    double acc = 0.0;
    if (k <= kmax)
      for (int c = 0; c < nparts; ++c) acc += partials[(int64_t)c * kMomSlots + sl];
    mu[sl] = acc;
  }
  __syncthreads();
  moments_to_gram(mu, w, G);
}

// Batched: one CTA per system, its items' partials in item order.
__global__ void __launch_bounds__(128) gram_items_moment_finalize_kernel(const double* __restrict__ partials,
                                                                         const int* __restrict__ sys_item0,
                                                                         const int* __restrict__ sys_nitems,
                                                                         const int* __restrict__ sys_w,
                                                                         double* __restrict__ G, int64_t g_stride) {
  const int q = blockIdx.x;
  const int w = sys_w[q];
  if (w == 0) return;
  __shared__ double mu[kMomSlots];
  const int S = (w - 1) / 2;
  const int i0 = sys_item0[q], ni = sys_nitems[q];
  for (int sl = threadIdx.x; sl < kMomSlots; sl += blockDim.x) {
    const int fam = sl / kMomFam, k = sl % kMomFam;
    const int kmax = fam == 0 ? 2 * S : (fam == 1 ? 2 * S - 1 : 2 * S - 2);
    double acc = 0.0;
    if (k <= kmax)
      for (int it = 0; it < ni; ++it) acc += partials[(int64_t)(i0 + it) * kMomSlots + sl];
    mu[sl] = acc;
  }
  __syncthreads();
  moments_to_gram(mu, w, G + (int64_t)q * g_stride);
}

// Four threads per pair (lanes 4q .. 4q+3 of a warp): thread t adds the
// partials of CTAs c = t, t + 4, t + 8, ... with loads unrolled eight deep,
// then the four sums combine as (s0 + s1) + (s2 + s3). Fixed order: the result
// is bitwise reproducible.
__global__ void __launch_bounds__(128) gram_finalize_kernel(int w, const double* __restrict__ partials, int nparts,
                                                            double* __restrict__ G, const int* __restrict__ gate) {
  pdl_wait();
  pdl_release();
  if (gate && !*gate) return;
  const int np = w * (w + 1) / 2;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = gt >> 2, t = gt & 3;
  double acc = 0.0;
  if (p < np) {
    int c = t;
    for (; c + 28 < nparts; c += 32) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = partials[(int64_t)(c + 4 * u) * np + p];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; c < nparts; c += 4) acc += partials[(int64_t)c * np + p];
  }
  const double a1 = __shfl_down_sync(0xffffffffu, acc, 1);
  const double a2 = __shfl_down_sync(0xffffffffu, acc, 2);
  const double a3 = __shfl_down_sync(0xffffffffu, acc, 3);
  if (t != 0 || p >= np) return;
  const double s = (acc + a1) + (a2 + a3);
  int a = 0, rem = p;
  while (rem >= w - a) {
    rem -= w - a;
    ++a;
  }
  const int b = a + rem;
  G[a * w + b] = s;
  G[b * w + a] = s;
}

// Batched solves: G of system q (w_q x w_q, stride w_q, both halves) at
// G + q * g_stride from its items' partials (computed with W >= w_q columns),
// added in item order. One CTA per system.
__global__ void __launch_bounds__(256) gram_items_finalize_kernel(int W, const double* __restrict__ partials,
                                                                  const int* __restrict__ sys_item0,
                                                                  const int* __restrict__ sys_nitems,
                                                                  const int* __restrict__ sys_w, double* __restrict__ G,
                                                                  int64_t g_stride) {
  const int q = blockIdx.x;
  const int w = sys_w[q];
  if (w == 0) return;
  const int NP = W * (W + 1) / 2;
  const int i0 = sys_item0[q], ni = sys_nitems[q];
  double* Gq = G + (int64_t)q * g_stride;
  for (int e = threadIdx.x; e < w * (w + 1) / 2; e += blockDim.x) {
    int a = 0, rem = e;
    while (rem >= w - a) {
      rem -= w - a;
      ++a;
    }
    const int b = a + rem;
    const int p = a * W - a * (a - 1) / 2 + (b - a);  // pair (a, b) in W-space
    double s = 0.0;
    for (int it = 0; it < ni; ++it) s += partials[(int64_t)(i0 + it) * NP + p];
    Gq[a * w + b] = s;
    Gq[b * w + a] = s;
  }
}

template <int W>
cudaError_t gram_w(int64_t n, const double* Y, int64_t ldY, double* partials, int grid, cudaStream_t s,
                   const int* gate) {
  gram_partial_kernel<W><<<grid, kGramThreads, 0, s>>>(n, Y, ldY, partials, gate);
  return cudaGetLastError();
}

}  // namespace

int gram_grid() {
  // the current device's SM count, looked up once per device (each thread may
  // look it up the first time; the value is the same)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int v = g_gram_grid[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  const bool ok = dev >= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                  sms > 0;
  if (!ok) return 1;
  if (cached) g_gram_grid[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

int gram_parts(int64_t n) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  return (int)(chunks < gram_grid() ? chunks : gram_grid());
}

cudaError_t launch_gram_partial(int64_t n, int w, const double* Y, int64_t ldY, double* partials, cudaStream_t s,
                                const int* gate) {
  const int grid = gram_parts(n);
  switch (w) {
#define ASCG_GW(W) \
  case W:          \
    return gram_w<W>(n, Y, ldY, partials, grid, s, gate);
    ASCG_GW(1) ASCG_GW(2) ASCG_GW(3) ASCG_GW(4) ASCG_GW(5) ASCG_GW(6) ASCG_GW(7) ASCG_GW(8) ASCG_GW(9)
    ASCG_GW(10) ASCG_GW(11) ASCG_GW(12) ASCG_GW(13) ASCG_GW(14) ASCG_GW(15) ASCG_GW(16) ASCG_GW(17)
    ASCG_GW(18) ASCG_GW(19) ASCG_GW(20) ASCG_GW(21) ASCG_GW(22) ASCG_GW(23) ASCG_GW(24) ASCG_GW(25)
    ASCG_GW(26) ASCG_GW(27) ASCG_GW(28) ASCG_GW(29) ASCG_GW(30) ASCG_GW(31) ASCG_GW(32) ASCG_GW(33)
#undef ASCG_GW
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gram_items(int W, const SysDesc* descs, const GramItem* items, int nitems, const int* sys_w,
                              double* partials, int pair_groups, bool moments, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  if (pair_groups < 1 || pair_groups > 65535) return cudaErrorInvalidValue;
  const dim3 grid(nitems, pair_groups);
  switch (W) {
#define ASCG_GI(WW)                                                                              \
  case WW:                                                                                       \
    if (moments)                                                                                 \
      gram_items_kernel<WW, true><<<grid, kGramThreads, 0, s>>>(descs, items, sys_w, partials);  \
    else                                                                                         \
      gram_items_kernel<WW><<<grid, kGramThreads, 0, s>>>(descs, items, sys_w, partials);        \
    return cudaGetLastError();
    ASCG_GI(3) ASCG_GI(5) ASCG_GI(7) ASCG_GI(9) ASCG_GI(11) ASCG_GI(13) ASCG_GI(15) ASCG_GI(17) ASCG_GI(19)
    ASCG_GI(21) ASCG_GI(23) ASCG_GI(25) ASCG_GI(27) ASCG_GI(29) ASCG_GI(31) ASCG_GI(33)
#undef ASCG_GI
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gram_items_finalize(int W, const double* partials, const int* sys_item0, const int* sys_nitems,
                                       const int* sys_w, int count, double* G, int64_t g_stride, bool moments,
                                       cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  if (moments)
    gram_items_moment_finalize_kernel<<<count, 128, 0, s>>>(partials, sys_item0, sys_nitems, sys_w, G, g_stride);
  else
    gram_items_finalize_kernel<<<count, 256, 0, s>>>(W, partials, sys_item0, sys_nitems, sys_w, G, g_stride);
  return cudaGetLastError();
}

cudaError_t launch_gram_moments(int64_t n, int w, const double* Y, int64_t ldY, double* partials, int* nparts,
                                cudaStream_t s, const int* gate) {
  const int grid = gram_parts(n);
  *nparts = grid;
  switch (w) {
#define ASCG_GM(W)                                                                       \
  case W:                                                                                \
    gram_partial_kernel<W, true><<<grid, kGramThreads, 0, s>>>(n, Y, ldY, partials, gate); \
    return cudaGetLastError();
    ASCG_GM(3) ASCG_GM(5) ASCG_GM(7) ASCG_GM(9) ASCG_GM(11) ASCG_GM(13) ASCG_GM(15) ASCG_GM(17) ASCG_GM(19)
    ASCG_GM(21) ASCG_GM(23) ASCG_GM(25) ASCG_GM(27) ASCG_GM(29) ASCG_GM(31) ASCG_GM(33)
#undef ASCG_GM
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gram_moment_finalize(int w, const double* partials, int nparts, double* G, cudaStream_t s,
                                        const int* gate) {
  gram_moment_finalize_kernel<<<1, 128, 0, s>>>(w, partials, nparts, G, gate);
  return cudaGetLastError();
}

cudaError_t launch_gram_finalize(int w, const double* partials, int nparts, double* G, cudaStream_t s,
                                 const int* gate) {
  const int np = w * (w + 1) / 2;
  return launch_pdl(gram_finalize_kernel, (4 * np + 127) / 128, 128, s, w, partials, nparts, G, gate);
}

}  // namespace ascg
