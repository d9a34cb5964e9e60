// Block controller of adaptive s-step CG (Alg. 4): condition estimates of the
// Gram submatrices (eq. condy), the choice of s~_k, the in-loop check
// (eq. check), the coordinate CG steps (Sec. 2.1), and the Newton-basis
// shifts.
//
// All of this is tiny dense work on matrices of order <= 33. On GB300 an FP64
// warp instruction costs ~20 SM cycles whether 1 or 32 lanes are active, and
// a dependent DFMA takes 64 cycles. So this code keeps the lanes busy on
// independent work: one lane per row for the Householder steps, and 64
// evaluation points per Sturm multisection round.
#include <math_constants.h>

#include "ascg_common.cuh"

namespace ascg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = e^2) that are
// smaller than x (Sturm count from the LDL^T pivots).
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int m, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int r = 1; r < m; ++r) {
    q = (d[r] - x) - e2[r - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Gershgorin interval of the tridiagonal, widened by a few ulps.
__device__ void gershgorin(const double* d, const double* e, int m, double* lo, double* hi, double* pivmin) {
  double gl = CUDART_INF, gh = -CUDART_INF, e2max = 0.0;
  for (int r = 0; r < m; ++r) {
    const double off = (r > 0 ? fabs(e[r - 1]) : 0.0) + (r + 1 < m ? fabs(e[r]) : 0.0);
    gl = fmin(gl, d[r] - off);
    gh = fmax(gh, d[r] + off);
    if (r + 1 < m) e2max = fmax(e2max, e[r] * e[r]);
  }
  const double widen = 4.0 * kEps * fmax(fabs(gl), fabs(gh)) * m + 1e-300;
  *lo = gl - widen;
  *hi = gh + widen;
  *pivmin = 2.2250738585072014e-308 * fmax(1.0, e2max);
}

// Number of eigenvalues smaller than x of the symmetric tridiagonal (d, e2 =
// e^2) of order M, scaled to norm <= 1, from the signs of the leading
// principal minors of T - xI. The minors follow p_k = (d_k - x) p_{k-1} -
// e2_{k-1} p_{k-2}, with no division: rounding gives the exact signs of a
// matrix whose d_k - x and e2 are perturbed by a few ulps (positive
// rescalings do not change signs), the backward error of the pivot form.
// The loop is unrolled with d and e2 in registers. Each step costs three FP64
// instructions (d_k - x, the product with e2 and the FMA); on GB300 an SM
// sub-partition issues about one FP64 warp instruction per 64 cycles, and
// that rate, not latency, sets the time of a multisection round. The leading
// minors grow at most like (1 + sqrt 2)^k <= 2^43 for M <= 33, so they cannot
// overflow. One integer test of the exponent per step catches, on a rarely
// taken branch, both a minor below 2^-256 (rescaled exactly by 2^256, with
// its predecessor) and a zero minor (replaced by a tiny value of the sign
// opposite to its predecessor).
template <int M>
__device__ __forceinline__ int sturm_unrolled(const double (&d)[M], const double (&e2)[M], double x) {
  const double kUp = 1.157920892373162e77;     // 2^256
  const double kTiny = 8.636168555094445e-78;  // 2^-256
  double pm2 = 1.0;
  double pm1 = d[0] - x;
  if (pm1 == 0.0) pm1 = -kTiny * kTiny;
  int hprev = __double2hiint(pm1);
  int cnt = (int)((unsigned)hprev >> 31);
#pragma unroll
  for (int k = 1; k < M; ++k) {
    const double t = e2[k - 1] * pm2;
    double p = fma(d[k] - x, pm1, -t);
    int hp = __double2hiint(p);
    if (((hp >> 20) & 0x7ff) < 767) {  // |p| < 2^-256 or p == 0 (rare)
      if (((hp & 0x7fffffff) | __double2loint(p)) == 0) {
        p = -copysign(fabs(pm1) * kTiny, pm1);
      } else {  // exact rescaling of p_k and p_{k-1}
        p *= kUp;
        pm1 *= kUp;
      }
      hp = __double2hiint(p);
    }
    cnt += (int)((unsigned)(hp ^ hprev) >> 31);
    pm2 = pm1;
    pm1 = p;
    hprev = hp;
  }
  return cnt;
}

// 65-way multisection by a pair of warps (64 evaluation points per round, 32
// per warp, the pair synchronised by the named barrier bar_id of 64 threads),
// for the smallest x with count(x) >= target on [lo, hi]. half: the warp's
// place in the pair. geo0: the first round uses the points hi * 2^(k - 64),
// k = 0..63. stop_below: if the first geometric bracket lies at or below this
// value, sets *below and stops. Both warps compute the same brackets.
template <int M>
__device__ void multisect_pair(const double* ds, const double* e2s, int target, int rounds, bool geo0,
                               double stop_below, double* lo_io, double* hi_io, int* below, int half, int bar_id,
                               unsigned* s_mask) {
  const int lane = threadIdx.x & 31;
  const int k = lane + 32 * half;
  double d[M], e2[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    d[q] = ds[q];
    e2[q] = q + 1 < M ? e2s[q] : 0.0;
  }
  const double kStep = 1.0 / 65.0;
  double lo = *lo_io, hi = *hi_io;
  for (int round = 0; round < rounds; ++round) {
    const bool geo = geo0 && round == 0;
    const double x = geo ? ldexp(hi, k - 64) : lo + (hi - lo) * ((double)(k + 1) * kStep);
    const unsigned mk = __ballot_sync(kFull, sturm_unrolled<M>(d, e2, x) >= target);
    if (lane == 0) s_mask[half] = mk;
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
    const unsigned long long both = (unsigned long long)s_mask[0] | ((unsigned long long)s_mask[1] << 32);
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");  // both masks read before the next round
    // the point k' of either warp, recomputed from the shared bracket
    auto point = [&](int kk) {
      return geo ? ldexp(hi, kk - 64) : lo + (hi - lo) * ((double)(kk + 1) * kStep);
    };
    double nlo = lo, nhi = hi;
    if (both == 0ull) {
      nlo = point(63);
    } else {
      const int f = __ffsll((long long)both) - 1;
      nhi = point(f);
      nlo = f > 0 ? point(f - 1) : (geo ? 0.0 : lo);
    }
    if (geo && nhi <= stop_below) {
      *below = 1;
      break;
    }
    lo = nlo;
    hi = nhi;
  }
  *lo_io = lo;
  *hi_io = hi;
}

__device__ void multisect_pair_dispatch(int m, const double* ds, const double* e2s, int target, int rounds,
                                        bool geo0, double stop_below, double* lo, double* hi, int* below, int half,
                                        int bar_id, unsigned* s_mask) {
  switch (m) {
#define ASCG_MP(M)                                                                                          \
  case M:                                                                                                   \
    multisect_pair<M>(ds, e2s, target, rounds, geo0, stop_below, lo, hi, below, half, bar_id, s_mask); \
    break;
    ASCG_MP(3) ASCG_MP(5) ASCG_MP(7) ASCG_MP(9) ASCG_MP(11) ASCG_MP(13) ASCG_MP(15) ASCG_MP(17)
    ASCG_MP(19) ASCG_MP(21) ASCG_MP(23) ASCG_MP(25) ASCG_MP(27) ASCG_MP(29) ASCG_MP(31) ASCG_MP(33)
#undef ASCG_MP
    default:
      break;
  }
}

// Warp-wide min and max (identical in all lanes).
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// kappa(G_{k,i}). G_{k,i} is the leading (2i+1) block of G
// (interleaved column order). The FP64 pipe is shared by the whole SM, so the
// kernel avoids redundant FP64 work: warp 0 alone forms each Householder
// reflection's scalars (norm, square root, one division) and publishes them
// in shared memory. Only the O(len^2) product and rank-2 update are split by
// columns over the four warps. The tridiagonal is then scaled to unit norm.
// Warps 0 and 1 bracket lambda_min and warps 2 and 3 lambda_max, each pair
// with 64 Sturm counts per round (the four warps sit on the SM's four
// sub-partitions, so the pairs' FP64 work runs side by side) for a fixed 6
// rounds. For lambda_min, the first round is on the powers of two
// 2^-64..2^-1 times min d, which finds its magnitude within a factor 2 and
// decides certification (is it below the floor (2i+1) sqrt(n) eps
// lambda_max?); five more rounds of 65 subintervals leave a bracket of
// relative width < 1e-9. lambda_max starts from [max d, Gershgorin bound], at
// most 2 lambda_max wide, and six rounds leave < 2e-10 of it. kappa is thus
// known to about 1e-9, far inside the 1e-6 to which rounding in G already
// makes decisions near a threshold uncertain.
constexpr int kKappaRounds = 6;

// Run by a whole CTA of 128 threads: sqrt(kappa(G_{k,i})) into st->sqrt_kappa[i-1]
// (G: the system's w x w Gram matrix, w = 2 sbar + 1).
__device__ void kappa_body(const double* __restrict__ G, BlockState* st, int i, int sbar) {
  const int m = 2 * i + 1;
  const int w = 2 * sbar + 1;
  __shared__ double A[kMaxW][kMaxW];  // odd row stride: conflict-free column access
  __shared__ double vb[2][32];         // Householder vectors of steps k (slot k & 1) and k + 1
  __shared__ double part[4][32];
  __shared__ double d[kMaxW], e[kMaxW], e2[kMaxW];
  __shared__ double lo_s[2], hi_s[2];
  __shared__ double den_s[2], floor_s;
  __shared__ int go_s[2], uncert_s;
  __shared__ unsigned s_mask[2][2];
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) A[idx / m][idx % m] = G[(idx / m) * w + (idx % m)];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The reflection that zeroes column kk below its subdiagonal (run by warp 0):
  // v = x - alpha e_1 over rows kk+1 .. m-1, alpha = -sign(x_0) ||x||, and
  // beta = 2 / v^T v = 1 / (s2 + |x_0| ||x||) (v^T v = 2 (s2 + |x_0| ||x||));
  // warp 0 publishes the denominator and every warp divides for itself.
  auto reflector = [&](int kk, int slot) {
    const int len_ = m - kk - 1;
    const bool on_ = lane < len_;
    const double xi = on_ ? A[kk + 1 + lane][kk] : 0.0;
    const double s2 = warp_sum(xi * xi);
    const double x0 = __shfl_sync(kFull, xi, 0);
    const int go = s2 > 0.0;
    double alpha = 0.0, vv = 0.0;
    if (go) {
      const double r = sqrt(s2);
      alpha = -copysign(r, x0);
      vv = on_ ? (lane == 0 ? x0 - alpha : xi) : 0.0;
      if (lane == 0) den_s[slot] = s2 + fabs(x0) * r;  // beta = 1 / den, formed by each warp when needed
    }
    vb[slot][lane] = vv;
    if (lane == 0) {
      go_s[slot] = go;
      e[kk] = alpha;  // s2 == 0: the column is already zero
    }
  };
  // Householder tridiagonalisation with look-ahead: in step k every warp
  // forms the product p = A22 v (columns split evenly), then, redundantly in
  // each warp, w = beta p - (beta^2 v^T p / 2) v, and applies the rank-2
  // update to its columns. Warp 0 owns only the first trailing column (column
  // k+1), so it can form the next step's reflection while warps 1..3 update
  // the rest. Two barriers per step; the arithmetic, and so every bit, is the
  // same as updating in turn.
  if (warp == 0 && m >= 3) reflector(0, 0);
  __syncthreads();
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;  // rows k+1 .. m-1, at most 32
    const int row = k + 1 + lane;
    const bool on = lane < len;
    const int sl = k & 1;
    if (go_s[sl]) {  // uniform
      const double vi = on ? vb[sl][lane] : 0.0;
      const double beta = 1.0 / den_s[sl];  // off warp 0's path: it overlaps this warp's product below
      const int c0 = (len * warp) >> 2, c1 = (len * (warp + 1)) >> 2;
      double p0 = 0.0, p1 = 0.0;
      if (on) {
        int c = c0;
        for (; c + 1 < c1; c += 2) {
          p0 = fma(A[row][k + 1 + c], vb[sl][c], p0);
          p1 = fma(A[row][k + 2 + c], vb[sl][c + 1], p1);
        }
        if (c < c1) p0 = fma(A[row][k + 1 + c], vb[sl][c], p0);
      }
      part[warp][lane] = p0 + p1;
      __syncthreads();
      const double pi = beta * ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane]));
      const double K = 0.5 * beta * warp_sum(vi * pi);
      const double wi = pi - K * vi;
      // rank-2 update of this warp's columns: warp 0 column 0, warps 1..3 the rest
      const int g0 = warp == 0 ? 0 : 1 + (((len - 1) * (warp - 1)) / 3);
      const int g1 = warp == 0 ? 1 : 1 + (((len - 1) * warp) / 3);
      for (int c = g0; c < g1; ++c) {
        const double vc = __shfl_sync(kFull, vi, c), wc = __shfl_sync(kFull, wi, c);
        if (on) A[row][k + 1 + c] = fma(-vi, wc, fma(-wi, vc, A[row][k + 1 + c]));
      }
    }
    if (warp == 0 && k + 3 < m) {
      __syncwarp();
      reflector(k + 1, sl ^ 1);
    }
    __syncthreads();
  }
  if (warp == 0) {
    // tridiagonal (d, e), Gershgorin bounds and scaling by warp reductions; lane r
    // holds row r (and row r + 32 for m = 33)
    for (int r = lane; r < m; r += 32) d[r] = A[r][r];
    if (lane == 0) e[m - 2] = A[m - 1][m - 2];
    __syncwarp();
    double gl = CUDART_INF, gh = -CUDART_INF, dmin = CUDART_INF, dmax = -CUDART_INF;
    for (int r = lane; r < m; r += 32) {
      const double off = (r > 0 ? fabs(e[r - 1]) : 0.0) + (r + 1 < m ? fabs(e[r]) : 0.0);
      gl = fmin(gl, d[r] - off);
      gh = fmax(gh, d[r] + off);
      dmin = fmin(dmin, d[r]);
      dmax = fmax(dmax, d[r]);
    }
    gl = warp_min(gl);
    gh = warp_max(gh);
    dmin = warp_min(dmin);
    dmax = warp_max(dmax);
    const double S = fmax(fabs(gl), fabs(gh));
    const double inv = S > 0.0 ? 1.0 / S : 1.0;
    for (int r = lane; r < m; r += 32) {
      d[r] *= inv;
      if (r + 1 < m) {
        const double er = e[r] * inv;
        e[r] = er;
        e2[r] = er * er;
      }
    }
    if (lane == 0) {
      dmin *= inv;
      dmax *= inv;
      // Gershgorin upper bound of the scaled matrix, widened by a few ulps
      const double ghs = gh * inv + 4.0 * kEps * (double)m + 1e-300;
      // certification floor, below the true one since lambda_max >= max d
      floor_s = (double)m * st->sqrt_n * kEps * dmax;
      lo_s[0] = 0.0;                              // lambda_min in [0, min d] unless uncertified
      hi_s[0] = dmin + 4.0 * kEps * fabs(dmin) + 1e-300;
      lo_s[1] = dmax - 4.0 * kEps * fabs(dmax);   // lambda_max in [max d, Gershgorin]
      hi_s[1] = ghs;
      // min d bounds lambda_min from above: at or below the floor, uncertified outright
      uncert_s = !(dmin > 0.0) || !(dmax > 0.0) || !(hi_s[0] > floor_s);
    }
  }
  __syncthreads();
  {
    const int pair = warp >> 1, half = warp & 1;  // pair 0: lambda_min (geometric first round), 1: lambda_max
    double lo = lo_s[pair], hi = hi_s[pair];
    int below = 0;
    if (!(pair == 0 && uncert_s))  // uniform over the pair
      multisect_pair_dispatch(m, d, e2, pair == 0 ? 1 : m, kKappaRounds, pair == 0, pair == 0 ? floor_s : -1.0, &lo,
                              &hi, &below, half, 1 + pair, s_mask[pair]);
    __syncthreads();  // every warp has read lo_s, hi_s and uncert_s
    if (lane == 0 && half == 0) {
      lo_s[pair] = lo;
      hi_s[pair] = hi;
      if (below) uncert_s = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double lmin = 0.5 * (lo_s[0] + hi_s[0]);
    const double lmax = 0.5 * (lo_s[1] + hi_s[1]);
    double sk;
    // reading: uncertified when lambda_min <= (2i+1) sqrt(n) eps lambda_max
    if (uncert_s || !(lmax > 0.0) || lmin <= (double)m * st->sqrt_n * kEps * lmax)
      sk = CUDART_INF;
    else
      sk = sqrt(lmax / lmin);
    st->sqrt_kappa[i - 1] = sk;
  }
}

// (B v)[t] for the interleaved coordinates of an s-step basis of size ss
// (eq. AVVB): chain ch = t & 1 (0: P, 1: R), position j = t >> 1, last
// position L = ss (P) or ss - 1 (R), whose column of B is zero.
__device__ __forceinline__ double bapply(const double* v, int t, int ss, const double* th, const double* sg,
                                         const double* gm) {
  const int ch = t & 1, j = t >> 1;
  const int L = ch ? ss - 1 : ss;
  double acc = 0.0;
  if (j >= 1) acc = gm[j - 1] * v[t - 2];
  if (j < L) acc = fma(th[j], v[t], acc);
  if (j + 1 < L) acc = fma(sg[j], v[t + 2], acc);
  return acc;
}

// g = Gs v over the first w rows and columns, by the CTA's four warps. Lane r
// holds row r (r < 32); warp q sums the columns c = q mod 4 in increasing
// order, and the row is (s0 + s1) + (s2 + s3). Each column keeps its slot for
// any w, so appending zero entries to v changes no bit of g. Row 32 (w = 33)
// is a lane-parallel product and a fixed tree in warp 1. Ends with a barrier.
__device__ __forceinline__ void gmatvec4(const double (*Gs)[kMaxW], const double* v, int w, double* g,
                                         double (*part)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < w) {
    double acc = 0.0;
    for (int c = warp; c < w; c += 4) acc = fma(Gs[lane][c], v[c], acc);
    part[warp][lane] = acc;
  }
  if (w > 32 && warp == 1) {
    double t = Gs[32][lane] * v[lane];
    if (lane == 0) t = fma(Gs[32][32], v[32], t);
    t = warp_sum(t);
    if (lane == 0) g[32] = t;
  }
  __syncthreads();
  if (warp == 0 && lane < w) g[lane] = (part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane]);
  __syncthreads();
}

// sum_r a[r] b[r] over the first w rows, by warp 0 (valid in all its lanes).
__device__ __forceinline__ double dot_rows(const double* a, const double* b, int w) {
  const int lane = threadIdx.x & 31;
  double t = warp_sum(lane < w ? a[lane] * b[lane] : 0.0);
  if (w > 32) t += a[32] * b[32];
  return t;
}

// Records of the speculative coordinate steps, per system: for step j =
// 1..kMaxS, x', r', p' after the step (3 kMaxW) and alpha_j, beta_j,
// sqrt(max(r'^T G r', 0)); then the number of steps taken.
constexpr int kSpecRow = 3 * kMaxW + 3;
constexpr int kSpecDone = kMaxS * kSpecRow;
static_assert(kSpecDone + 1 == kSpecDoubles, "spec record layout");

// The coordinate CG steps (Alg. 4 inner loop, Sec. 2.1) on the whole basis of
// size sbar, before s~_k is known. Because p' and r' after j steps have no
// component beyond P_j and R_{j-1}, steps 1..s~ on the whole basis give the
// same numbers as on the basis of size s~ (the extra entries of every
// product are exact zeros). The loop stops at min(sbar, max_steps) steps, at
// a step whose denominators are not positive and finite (breakdown), or at a
// step that reaches eps* (which ends the block whatever s~ is); the break
// test of eq. (check) needs s~ and is applied afterwards.
__device__ void spec_steps(const double* __restrict__ G, const double* __restrict__ th_g,
                           const double* __restrict__ sg_g, const double* __restrict__ gm_g, const BlockState* st,
                           double* __restrict__ rec) {
  __shared__ double Gs[kMaxW][kMaxW];  // odd row stride: conflict-free
  __shared__ double pc[kMaxW + 2], rc[kMaxW + 2], xc[kMaxW + 2], u[kMaxW + 2], rn[kMaxW + 2], g[kMaxW + 2];
  __shared__ double part[4][32];
  __shared__ double th[kMaxS], sg[kMaxS], gm[kMaxS];
  __shared__ int s_flag;
  __shared__ double s_alpha, s_beta;
  const int t = threadIdx.x;
  const int sbar = st->sbar;
  const int w = 2 * sbar + 1;
  const double eps_star = st->eps_star;
  for (int idx = t; idx < w * w; idx += blockDim.x) Gs[idx / w][idx % w] = G[idx];
  if (t < kMaxS) {
    th[t] = th_g[t];
    sg[t] = sg_g[t];
    gm[t] = gm_g[t];
  }
  if (t < kMaxW + 2) {
    pc[t] = (t == 0) ? 1.0 : 0.0;  // p' = e_1 (column p_0)
    rc[t] = (t == 1) ? 1.0 : 0.0;  // r' = e_{s+2} (column r_0)
    xc[t] = 0.0;
    u[t] = 0.0;
    rn[t] = 0.0;
    g[t] = 0.0;
  }
  __syncthreads();
  // thread owning coordinate row r: t = r for r < 32, t = 32 (warp 1, lane 0) for r = 32
  const int myrow = t < 32 ? t : (t == 32 ? 32 : -1);
  const bool own = myrow >= 0 && myrow < w;
  double rGr = Gs[1][1];
  const int nsteps = min(sbar, st->max_steps);
  int done = 0;
  for (int j = 1; j <= nsteps; ++j) {
    // alpha = (r'^T G r') / (p'^T G B p')
    if (own) u[myrow] = bapply(pc, myrow, sbar, th, sg, gm);
    __syncthreads();
    gmatvec4(Gs, u, w, g, part);
    if (t < 32) {
      const double pGBp = dot_rows(pc, g, w);
      if (t == 0) {
        const int ok = (pGBp > 0.0) && isfinite(pGBp) && (rGr > 0.0) && isfinite(rGr);
        s_flag = ok;
        s_alpha = ok ? rGr / pGBp : 0.0;
      }
    }
    __syncthreads();
    if (!s_flag) break;  // breakdown at step j: steps 1..j-1 stand
    const double alpha = s_alpha;
    // q' = alpha p'; x' += q'; r' -= B q'
    if (own) {
      const double q = alpha * pc[myrow];
      u[myrow] = q;
      xc[myrow] += q;
    }
    __syncthreads();
    if (own) rn[myrow] = rc[myrow] - bapply(u, myrow, sbar, th, sg, gm);
    __syncthreads();
    gmatvec4(Gs, rn, w, g, part);
    double* r = rec + (int64_t)(j - 1) * kSpecRow;
    if (t < 32) {
      const double rGr_new = dot_rows(rn, g, w);
      if (t == 0) {
        const double beta = rGr_new / rGr;
        const double rnn = sqrt(fmax(rGr_new, 0.0));
        r[3 * kMaxW] = alpha;
        r[3 * kMaxW + 1] = beta;
        r[3 * kMaxW + 2] = rnn;
        s_beta = beta;
        s_flag = rnn <= eps_star;  // converged: no later step can be taken
        s_alpha = rGr_new;
      }
    }
    __syncthreads();
    const double beta = s_beta;
    if (own) {
      pc[myrow] = fma(beta, pc[myrow], rn[myrow]);  // p' = r'_new + beta p'
      rc[myrow] = rn[myrow];
      r[myrow] = xc[myrow];
      r[kMaxW + myrow] = rn[myrow];
      r[2 * kMaxW + myrow] = pc[myrow];
    }
    rGr = s_alpha;
    done = j;
    const int conv = s_flag;
    __syncthreads();
    if (conv) break;
  }
  if (t == 0) rec[kSpecDone] = (double)done;
}

// Applies eq. (condy) and eq. (check) to the kappa values and the step
// records (one CTA; the other CTAs' writes are read with L1-bypassing loads),
// writes the block's outcome, the histories of the steps taken and their
// coordinates. All loads are issued at once by the CTA's threads into shared
// memory; thread 0 then decides on shared values only, so the decision does
// not wait on a chain of dependent global loads.
__device__ void select_steps(const double* __restrict__ G, BlockState* st, const double* __restrict__ rec,
                             double* __restrict__ coords, double* __restrict__ hist, double* __restrict__ res_hist,
                             int res_cap, double* __restrict__ ab_hist, int ab_cap) {
  __shared__ int s_steps;
  __shared__ double s_sk[kMaxS], s_step[kMaxS][3], s_g11, s_done;
  const int t = threadIdx.x;
  const int sbar = st->sbar;
  const int w = 2 * sbar + 1;
  if (t < 3 * sbar) s_step[t / 3][t % 3] = __ldcg(rec + (int64_t)(t / 3) * kSpecRow + 3 * kMaxW + t % 3);
  if (t >= 64 && t < 64 + sbar) s_sk[t - 64] = __ldcg(&st->sqrt_kappa[t - 64]);
  if (t == 96) s_g11 = __ldcg(G + 1 * w + 1);
  if (t == 97) s_done = __ldcg(rec + kSpecDone);
  __syncthreads();
  if (t < 32) {
    // warp 0, lane j - 1 for step j and submatrix i = j: the same scalar
    // formulas as a serial scan, evaluated for all j at once (an FP64
    // instruction costs the same for 1 or 32 lanes), then ballots
    const int lane = t;
    const int adaptive = st->method == ASCG_ADAPTIVE;
    const double eps_star = st->eps_star, cc = st->c, bnorm = st->bnorm;
    // ||r_{m+1}|| from G: column 1 is rho_0(A) r = r
    const double rnorm = sqrt(fmax(s_g11, 0.0));
    // eq. (condy) takes c_{k,s_max}
    const double c_condy = st->c_step > 0.0 ? st->c_step * st->c_smax : cc;
    const double T = rnorm > 0.0 ? eps_star / (c_condy * kEps * rnorm) : CUDART_INF;
    int stilde;
    double gamma;
    if (adaptive) {
      // eq. (condy): largest prefix i with sqrt(kappa(G_{k,i})) <= T; none -> 1
      const unsigned ok = __ballot_sync(kFull, lane < sbar && s_sk[lane < sbar ? lane : 0] <= T);
      stilde = __ffs(~ok) - 1;
      if (stilde < 1) stilde = 1;
      gamma = s_sk[stilde - 1];
    } else {
      stilde = sbar;
      gamma = 0.0;
    }
    const int done = (int)s_done;
    const int nmax = min(stilde, st->max_steps);
    // step j ends the loop: breakdown (j > done), convergence, or eq. (check),
    // a break when gamma >= eps* / (c_{k,j} eps (r'^T G r')^(1/2))
    const int j = lane + 1;
    const double rnn = s_step[lane < kMaxS ? lane : 0][2];
    const bool bd = j > done;
    const bool conv = !bd && rnn <= eps_star;
    bool brk = false;
    if (!bd && !conv && adaptive && st->check_in_loop) {
      const double cj = st->c_step > 0.0 ? st->c_step * j : cc;
      const double Tj = rnn > 0.0 ? eps_star / (cj * kEps * rnn) : CUDART_INF;
      brk = gamma >= Tj;
    }
    const unsigned ev = __ballot_sync(kFull, j <= nmax && (bd || conv || brk));
    const unsigned cv = __ballot_sync(kFull, conv);
    const unsigned bdm = __ballot_sync(kFull, bd);
    int steps, stop;
    if (ev == 0u) {
      steps = nmax;
      stop = steps < stilde ? ASCG_STOP_MAXITER : ASCG_STOP_DONE;
    } else {
      const int f = __ffs(ev) - 1;  // step f + 1 ends the loop
      if ((bdm >> f) & 1u) {
        steps = f;
        stop = ASCG_STOP_BREAKDOWN;
      } else {
        steps = f + 1;
        stop = ((cv >> f) & 1u) ? ASCG_STOP_CONVERGED : ASCG_STOP_BREAK;
      }
    }
    if (lane == 0) {
      st->rnorm = rnorm;
      st->threshold = T;
      st->stilde = stilde;
      st->gamma = gamma;
      st->s_k = steps;
      st->stop = stop;
      st->converged = stop == ASCG_STOP_CONVERGED;
      st->rel_res = steps > 0 ? s_step[steps - 1][2] / bnorm : rnorm / bnorm;
      s_steps = steps;
    }
  }
  __syncthreads();
  const int steps = s_steps;
  // histories of the steps taken: step j (1-based) is iteration m + j
  if (t < steps) {
    const int j = t + 1;
    const double alpha = s_step[t][0], beta = s_step[t][1], relres = s_step[t][2] / st->bnorm;
    const int it = st->m + j;
    if (res_hist && it < res_cap) res_hist[it] = relres;
    if (ab_hist && it - 1 < ab_cap) {
      ab_hist[it - 1] = alpha;
      ab_hist[ab_cap + it - 1] = beta;
    }
    if (hist) {
      hist[3 * t] = alpha;
      hist[3 * t + 1] = beta;
      hist[3 * t + 2] = relres;
    }
  }
  const double* r = rec + (int64_t)(steps - 1) * kSpecRow;
  for (int c = t; c < w; c += blockDim.x) {
    if (steps > 0) {
      coords[c] = __ldcg(r + c);
      coords[w + c] = __ldcg(r + kMaxW + c);
      coords[2 * w + c] = __ldcg(r + 2 * kMaxW + c);
    } else {  // no step: x' = 0, r' and p' select r and p
      coords[c] = 0.0;
      coords[w + c] = c == 1 ? 1.0 : 0.0;
      coords[2 * w + c] = c == 0 ? 1.0 : 0.0;
    }
  }
}

// The block after its Gram matrix, for system q = blockIdx.y (a single solve:
// one system): CTA 0 runs the coordinate steps speculatively (spec_steps)
// while CTAs i = 1..sbar compute kappa(G_{k,i}) (adaptive method only). The
// last CTA to finish (a ticket counter per system, reset afterwards; nothing
// waits) selects s~_k and s_k and writes the outputs. The condition
// estimates and the steps thus overlap instead of following each other.
__global__ void __launch_bounds__(128) block_ctrl_kernel(const double* __restrict__ G,
                                                         const double* __restrict__ th_g,
                                                         const double* __restrict__ sg_g,
                                                         const double* __restrict__ gm_g, BlockState* st,
                                                         double* __restrict__ coords, double* __restrict__ hist,
                                                         double* __restrict__ res_hist, int res_cap,
                                                         double* __restrict__ ab_hist, int ab_cap, int64_t g_stride,
                                                         int64_t c_stride, double* __restrict__ spec,
                                                         unsigned* counters) {
  pdl_wait();
  pdl_release();
  const int q = blockIdx.y;
  G += (int64_t)q * g_stride;
  st += q;
  coords += (int64_t)q * c_stride;
  spec += (int64_t)q * (kSpecDone + 1);
  counters += q;
  if (res_hist) res_hist += (int64_t)q * res_cap;
  if (ab_hist) ab_hist += (int64_t)q * 2 * ab_cap;
  if (!st->active) return;  // uniform over the system's CTAs
  const int sbar = st->sbar;
  const int parts = st->method == ASCG_ADAPTIVE ? sbar + 1 : 1;
  if ((int)blockIdx.x >= parts) return;
  if (blockIdx.x == 0)
    spec_steps(G, th_g, sg_g, gm_g, st, spec);
  else
    kappa_body(G, st, (int)blockIdx.x, sbar);
  __shared__ unsigned s_ticket;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's records before its ticket
    s_ticket = atomicAdd(counters, 1u);
  }
  __syncthreads();
  if (s_ticket != (unsigned)(parts - 1)) return;
  __threadfence();
  select_steps(G, st, spec, coords, hist, res_hist, res_cap, ab_hist, ab_cap);
  if (threadIdx.x == 0) *counters = 0u;
}

// Carries a single solve from block j to block j+1 on the device: m, k and the
// iteration budget of block j+1 from block j's outcome, and block j+1's flag,
// cleared when block j ended the solve (converged, no step, a wait that ran
// out, or the iteration cap reached), so that a block enqueued ahead does
// nothing.
__global__ void block_advance_kernel(const BlockState* __restrict__ prev, BlockState* __restrict__ cur,
                                     int max_iters) {
  pdl_wait();
  pdl_release();
  if (threadIdx.x != 0) return;
  const int m = prev->m + prev->s_k;
  cur->m = m;
  cur->k = prev->k + 1;
  cur->max_steps = max_iters - m;
  cur->active = prev->active && prev->s_k > 0 && !prev->converged && prev->status == ASCG_OK && m < max_iters;
}

// Ritz values of the CG tridiagonal (k <= 32), one lane per eigenvalue index by
// bisection, then Leja order computed by the whole warp.
__global__ void __launch_bounds__(32) newton_shifts_kernel(const double* __restrict__ al,
                                                           const double* __restrict__ be, int k,
                                                           double* __restrict__ shifts) {
  __shared__ double d[32], e[32], e2[32], ritz[32];
  __shared__ double gl, gh, pm;
  const int lane = threadIdx.x;
  if (lane < k) {
    d[lane] = 1.0 / al[lane] + (lane > 0 ? be[lane - 1] / al[lane - 1] : 0.0);
    if (lane + 1 < k) {
      e[lane] = sqrt(be[lane]) / al[lane];
      e2[lane] = e[lane] * e[lane];
    }
  }
  __syncwarp();
  if (lane == 0) {
    double lo, hi, piv;
    gershgorin(d, e, k, &lo, &hi, &piv);
    gl = lo;
    gh = hi;
    pm = piv;
  }
  __syncwarp();
  if (lane < k) {
    // the (lane+1)-th smallest eigenvalue: smallest x with count(x) >= lane + 1
    double lo = gl, hi = gh;
    for (int it = 0; it < 200; ++it) {
      const double scale = fmax(fabs(lo), fabs(hi));
      if (hi - lo <= 2.0 * kEps * scale || !(hi > lo)) break;
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(d, e2, k, mid, pm) >= lane + 1)
        hi = mid;
      else
        lo = mid;
    }
    ritz[lane] = 0.5 * (lo + hi);
  }
  __syncwarp();
  // Leja order: first the largest |value|; then the largest product of distances
  // to the values chosen so far. Ties: larger value, then lower index.
  const double val = lane < k ? ritz[lane] : 0.0;
  double score = fabs(val);
  bool avail = lane < k;
  for (int step = 0; step < k; ++step) {
    double bs = avail ? score : -1.0, bv = val;
    int bi = avail ? lane : 64;
    for (int o = 16; o > 0; o >>= 1) {
      const double os = __shfl_xor_sync(kFull, bs, o);
      const double ov = __shfl_xor_sync(kFull, bv, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      const bool better = (os > bs) || (os == bs && (ov > bv || (ov == bv && oi < bi)));
      if (better) {
        bs = os;
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) shifts[step] = bv;
    if (lane == bi) avail = false;
    const double dist = fabs(val - bv);
    score = (step == 0) ? dist : score * dist;
  }
}

}  // namespace

cudaError_t launch_block_ctrl(const double* G, const double* theta, const double* sigma, const double* gamma,
                              BlockState* st, int sbar, int adaptive, double* coords, double* hist, double* res_hist,
                              int res_cap, double* ab_hist, int ab_cap, double* spec, unsigned* counter,
                              cudaStream_t s) {
  return launch_pdl_ex(block_ctrl_kernel, dim3(adaptive ? sbar + 1 : 1, 1), dim3(128), 0, s, G, theta, sigma, gamma,
                       st, coords, hist, res_hist, res_cap, ab_hist, ab_cap, (int64_t)0, (int64_t)0, spec, counter);
}

cudaError_t launch_block_ctrl_batch(const double* G, int64_t g_stride, const double* theta, const double* sigma,
                                    const double* gamma, BlockState* st, int count, int max_sbar, int adaptive,
                                    double* coords, int64_t c_stride, double* res_hist, int res_cap, double* ab_hist,
                                    int ab_cap, double* spec, unsigned* counters, cudaStream_t s) {
  if (count < 1 || max_sbar < 1) return cudaSuccess;
  block_ctrl_kernel<<<dim3(adaptive ? max_sbar + 1 : 1, count), 128, 0, s>>>(
      G, theta, sigma, gamma, st, coords, nullptr, res_hist, res_cap, ab_hist, ab_cap, g_stride, c_stride, spec,
      counters);
  return cudaGetLastError();
}

cudaError_t launch_block_advance(const BlockState* prev, BlockState* cur, int max_iters, cudaStream_t s) {
  return launch_pdl(block_advance_kernel, 1, 32, s, prev, cur, max_iters);
}

cudaError_t launch_newton_shifts(const double* alphas, const double* betas, int k, double* shifts,
                                 cudaStream_t s) {
  newton_shifts_kernel<<<1, 32, 0, s>>>(alphas, betas, k, shifts);
  return cudaGetLastError();
}

}  // namespace ascg
