// Gram matrix G = Y^T Y (eq. gram) on the tensor cores.
//
// On GB300 the FP64 pipe, not HBM, bounds a direct FP64 Gram: w(w+1)/2 FMAs
// per row of Y at about 2 DFMA per clock per SM. This kernel moves the
// products to the fp16 tensor cores with an error-free splitting of the
// operands (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication",
// Numer. Algorithms 59, 2012), in the fixed-point form with one exponent per
// column:
//
//  1. E_a is the exponent of the largest entry of column a (|y| < 2^E_a).
//     Each entry becomes the integer Y = trunc(y 2^(55 - E_a)), |Y| < 2^55,
//     written in seven balanced base-256 digits d_0 (most significant) ..
//     d_6, every |d_i| <= 128. A digit is exact in fp16.
//  2. The tensor cores form the digit products D[(i,a),(j,b)] =
//     sum_k d_i,a,k d_j,b,k over chunks of 1024 rows of Y with FP32
//     accumulation. Every product is an integer of magnitude <= 2^14 and a
//     chunk sum stays <= 2^24, so the FP32 accumulator holds it exactly.
//  3. Only pairs with i + j <= 7 are kept (the rest weigh below 2^-61
//     relative to 2^(E_a + E_b) per row). G is symmetric, so each ordered
//     pair ((i,a),(j,b)) is needed once, for the entry G_ab with a <= b. The
//     128 digits with i <= 3, a <= 31 (set T0) multiply all 231 digits in
//     tile 0 (M = 128, N = 240); a pair whose first digit is outside T0 is
//     read there transposed, except pairs with a top digit (j <= 3) of
//     column 32 as the partner, which tile 1 (M = 128, N = 16) supplies.
//     That is 32.8K multiply-adds per row of Y instead of 53K for all pairs.
//  4. Each needed product, scaled to its level L = i + j, is added to exact
//     integer sums hi_ab (L <= 3, times 2^(8(3-L))) and lo_ab (L >= 4, times
//     2^(8(7-L))): per chunk in int64 registers, then into the CTA's sums in
//     shared memory, kept as three 32-bit words of 17-bit slices each so that
//     plain 32-bit shared-memory reductions add them exactly. Integer sums do
//     not depend on the order: the result is deterministic.
//     G_ab = 2^(E_a + E_b - 14) (hi 2^-24 + lo 2^-56), formed in FP64 once per
//     CTA; the finalize kernel of the FP64 path adds the per-CTA partials in a
//     fixed order.
//
// Error: truncating y to the grid 2^(E - 55) gives |G^_ab - G_ab| <= about
// 2^-51 (max|y_a| ||y_b||_1 + max|y_b| ||y_a||_1) + gamma_(parts+1) |y_a|^T |y_b|,
// a normwise bound of the size of the FP64 rounding error of a dot product.
//
// Operand layout: 256 rows of fp16 digits per stage of 64 rows of Y, in
// 8-row x 16-byte core matrices, K-major with no swizzle (LBO = 128 B along
// K, SBO = 1024 B between 8-row groups). Row order: T0 i-major (rows 0..127),
// (i <= 3, 32) (128..131), (i >= 4, 32) (132..134), zeros (135..143),
// (i >= 4, a <= 31) i-major (144..239), zeros (240..255). Each TMEM load of
// the drain is then one aligned 16-column block of a single digit level.
//
// Pipeline (PTX ISA, tcgen05 and cp.async.bulk.tensor), linked by mbarriers,
// 29 warps with fixed roles:
//  - a loader thread issues one 2D tensor-map copy per stage (66 rows x 33
//    columns of Y; rows past n and columns past w arrive as zeros);
//  - two groups of 9 converter warps take alternate stages: 8 warps for
//    columns 0..31, where a thread turns 8 rows of one column from FP64 into
//    digits with one 16-byte store per digit, and one for column 32, 2 rows
//    per thread;
//  - two threads issue tcgen05.mma kind::f16 (f16 x f16 -> f32) into one of
//    two TMEM buffers, one tile 0 (at 256 p + 0..239), the other tile 1 (at
//    256 p + 240..255): a small MMA costs about as much as a large one, and
//    issuing the two tiles from two threads overlaps them better;
//  - 8 drain warps, two per TMEM lane quarter, fold a chunk's accumulators
//    into the integer sums while the next chunk is multiplied.
// All waits are bounded; a wait that runs out writes NaN partials and reports
// ASCG_ERR_TIMEOUT through the launch's error word, when one is given.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <math_constants.h>

#include <mutex>

#include "ascg_common.cuh"

namespace ascg {
namespace {

constexpr int kTW = 33;              // columns (w padded to 33)
constexpr int kDig = 7;              // digits per entry
constexpr int kSub = 64;             // rows of Y per stage (MMA K)
constexpr int kSubPerChunk = 16;
constexpr int kTChunk = kSub * kSubPerChunk;  // 1024 rows per TMEM accumulation
constexpr int kDStages = 3;          // digit operand stages
constexpr int kFStages = 6;          // FP64 staging stages (tensor copies in flight); even: a slot keeps its group
constexpr int kBoxRows = 66;         // rows per tensor copy: column stride 528 B (bank offset)
constexpr uint32_t kColStride = kBoxRows * 8;
constexpr uint32_t kFStageBytes = ((kTW * kColStride + 127) / 128) * 128;
constexpr uint32_t kFBoxBytes = kTW * kColStride;   // bytes one tensor copy delivers
constexpr uint32_t kLBO = 128;       // bytes between core matrices along K
constexpr uint32_t kSBO = (kSub / 8) * 128;   // bytes between 8-row groups (1024)
constexpr uint32_t kDStageBytes = 256 * kSub * 2;  // 32 KB: 256 digit rows x 64 fp16
constexpr int kN0 = 240, kN1 = 16;   // MMA N of tiles 0 and 1
constexpr int kTile1Col = 240;       // TMEM column of tile 1 within a buffer
constexpr int kGroupWarps = 9;       // converters per group: 8 for columns 0..31, 1 for column 32
constexpr int kConvWarps = 2 * kGroupWarps;
constexpr int kDrainWarp0 = kConvWarps, kDrainWarps = 8;  // drain warp d: lane quarter d & 3, half d >> 2
constexpr int kLoadWarp = kDrainWarp0 + kDrainWarps;
constexpr int kMmaWarp = kLoadWarp + 1, kMma1Warp = kMmaWarp + 1;  // tile 0 and tile 1 issuers
constexpr int kTcThreads = (kMma1Warp + 1) * 32;                   // 928
constexpr long long kWaitLimit = 1ll << 20;  // polls; with the suspend hint a wait ends within ~2 s
constexpr long long kTestWaitLimit = 1ll << 12;  // the stall test's limit: a few milliseconds
static_assert(kFStages % 2 == 0, "a staging slot must belong to one converter group");

// dynamic shared memory layout
constexpr size_t kDOff = 0;
constexpr size_t kFOff = kDOff + (size_t)kDStages * kDStageBytes;
constexpr int kSlices = 3;           // 17-bit slices of an int64 sum, one 32-bit word each
constexpr size_t kAccOff = kFOff + (size_t)kFStages * kFStageBytes;  // u32 [2 (hi, lo)][3][33][33]
constexpr size_t kBarOff = kAccOff + 2 * kSlices * 4 * kTW * kTW;
constexpr int kNumBars = 2 * kFStages + 2 * kDStages + 6;
constexpr size_t kSlotOff = kBarOff + 8 * kNumBars;
constexpr size_t kEmaxOff = kSlotOff + 16;
constexpr size_t kErrOff = kEmaxOff + 4 * kTW;
constexpr size_t kTcSmem = kErrOff + 16;
static_assert(kFOff % 1024 == 0 && kFStageBytes % 128 == 0 && kAccOff % 16 == 0 && kBarOff % 8 == 0,
              "alignment");
static_assert(kTcSmem <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start, LBO, SBO (all >> 4),
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D f32 (bit 4), A and B f16 (format 0),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 2D tensor-map copy of the box at (row0, 0) into shared memory; completion
// counted on the mbarrier's transaction count.
__device__ __forceinline__ void tensor_g2s(void* dst, const CUtensorMap* map, int row0, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(row0), "r"(0), "r"(smem_u32(bar))
      : "memory");
}

// One test of the phase; a thread whose phase is not complete is suspended
// for up to kSuspendNs (woken early when the phase completes), so waiting
// warps leave the issue slots to the working ones.
constexpr uint32_t kSuspendNs = 2000;
__device__ __forceinline__ int bar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return (int)ok;
}

// Waits until the phase of the given parity has completed. Gives up after
// `limit` polls or once another role has given up; returns 0 then.
__device__ __forceinline__ int bar_wait(uint64_t* bar, uint32_t parity, volatile int* err, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  if (bar_try(a, parity)) return 1;
  for (uint32_t it = 1; it < limit; ++it) {
    if (bar_try(a, parity)) return 1;
    if ((it & 15) == 0 && *err) return 0;
  }
  *err = 1;
  return 0;
}

// Bounded wait that ignores the error flag: lets copies and MMAs already
// issued finish before the CTA exits after an error.
__device__ __forceinline__ void bar_drain(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < limit; ++it)
    if (bar_try(a, parity)) return;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
}

// Balanced digits, step 1. With E = emax - 1022 for the column's largest
// biased exponent emax, Y = trunc(y 2^(55 - E)) (|Y| < 2^55), and
// Z = Y + sum_{k<7} 128 * 256^k + 0x6400 * 2^48. Byte k of Z (k < 6) is
// c_k + 128, and the top 16 bits of Z are 0x6400 + c_6 + 128 (no carry out:
// c_6 + 128 <= 256), the fp16 bit pattern of 1024 + c_6 + 128, where
// Y = sum_k c_k 256^k with c_k in [-128, 127] (k < 6) and c_6 in
// [-128, 128]. Integer operations only; any emax, zeros and subnormals
// included.
constexpr unsigned long long kZBias = 0x6480808080808080ull;
__device__ __forceinline__ void split_z(double y, int emax, uint32_t& zlo, uint32_t& zhi) {
  const int hi = __double2hiint(y);
  const uint32_t lo = (uint32_t)__double2loint(y);
  const int e = (hi >> 20) & 0x7ff;
  const uint32_t mhi = ((uint32_t)hi & 0xFFFFFu) | (e != 0 ? 0x100000u : 0u);
  // M = m * 8 (56 bits), Y = M >> s with s = emax + 1 - max(e, 1) >= 1
  const uint32_t Mhi = __funnelshift_l(lo, mhi, 3);
  const uint32_t Mlo = lo << 3;
  int s = emax + 1 - (e > 1 ? e : 1);
  s = s < 63 ? s : 63;
  unsigned long long Y = (((unsigned long long)Mhi << 32) | Mlo) >> s;
  if (hi < 0) Y = 0ull - Y;
  const unsigned long long Z = Y + kZBias;
  zlo = (uint32_t)Z;
  zhi = (uint32_t)(Z >> 32);
}

// The same Z for a column with emax >= 55, in fewer operations:
// Y = (m 4) >> (emax - e) with the implicit bit always set, which is
// (m 8) >> (emax + 1 - e) for e >= 1; a zero or subnormal entry (e = 0) then
// shifts by >= 55 and gives 0, as it must (its true Y is 0 below 2^-968).
// The sign is applied as (Y ^ s) - s with s = 0 or all ones.
constexpr int kFastSplitMinEmax = 55;
__device__ __forceinline__ void split_z_fast(double y, int emax, uint32_t& zlo, uint32_t& zhi) {
  const int hi = __double2hiint(y);
  const uint32_t lo = (uint32_t)__double2loint(y);
  const uint32_t t = (uint32_t)(emax - ((hi >> 20) & 0x7ff));
  const uint32_t Mhi = (__funnelshift_l(lo, (uint32_t)hi, 2) & 0x3FFFFFu) | 0x400000u;
  const unsigned long long M = ((unsigned long long)Mhi << 32) | (lo << 2);
  unsigned long long Y;
  asm("shr.b64 %0, %1, %2;" : "=l"(Y) : "l"(M), "r"(t));  // a shift of 64 or more gives 0
  const unsigned long long sm = (unsigned long long)(long long)(hi >> 31);
  const unsigned long long Z = (Y ^ sm) + kZBias - sm;
  zlo = (uint32_t)Z;
  zhi = (uint32_t)(Z >> 32);
}

// The seven digits of two entries as fp16 pairs (exact), w[i] holding digit
// i = 0 (c_6, most significant) .. 6 (c_0) of entry 0 in the low half and of
// entry 1 in the high half. Bytes k, k + 1 of both Z are first gathered into
// one word; each fp16 pair is then 0x64 | byte (1024 + c + 128), minus 1152;
// the top digit comes with its 0x64 already in place (kZBias).
__device__ __forceinline__ void digit_words(uint32_t zl0, uint32_t zh0, uint32_t zl1, uint32_t zh1,
                                            uint32_t (&w)[kDig]) {
  const uint32_t x01 = __byte_perm(zl0, zl1, 0x5140);  // z0.b0 z1.b0 z0.b1 z1.b1
  const uint32_t x23 = __byte_perm(zl0, zl1, 0x7362);  // z0.b2 z1.b2 z0.b3 z1.b3
  const uint32_t x45 = __byte_perm(zh0, zh1, 0x5140);  // bytes 4, 5
  uint32_t t[kDig];
  t[0] = __byte_perm(x01, 0x64646464u, 0x4140);
  t[1] = __byte_perm(x01, 0x64646464u, 0x4342);
  t[2] = __byte_perm(x23, 0x64646464u, 0x4140);
  t[3] = __byte_perm(x23, 0x64646464u, 0x4342);
  t[4] = __byte_perm(x45, 0x64646464u, 0x4140);
  t[5] = __byte_perm(x45, 0x64646464u, 0x4342);
  t[6] = __byte_perm(zh0, zh1, 0x7632);  // the top 16 bits of each Z
  const __half2 c = __floats2half2_rn(1152.0f, 1152.0f);
#pragma unroll
  for (int k = 0; k < kDig; ++k) {
    const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&t[k]), c);
    w[kDig - 1 - k] = *reinterpret_cast<const uint32_t*>(&h);
  }
}

// A converter thread's task in every stage of its group. In converter warp
// k < 8 of a group, lane l takes rows 8 g .. 8 g + 7 of column
// a = 8 (k & 3) + (l & 7), g = 4 (k >> 2) + (l >> 3): the 8 lanes of a
// quarter warp share g and cover 8 consecutive columns, so each 16-byte load
// from the staging box (column stride 528 B) and each 16-byte digit store
// (8 consecutive operand rows of one core matrix) is free of bank conflicts.
// Warp 8 takes column 32, rows 2 l and 2 l + 1 in lane l.
//
// Digit i of column a <= 31 goes to operand row 32 i + a (i <= 3) or
// 32 i + 16 + a (i >= 4), at byte (row >> 3) 1024 + g 128 + (row & 7) 16
// of the stage, and of column 32 to row 128 + i; see the layout above.
struct ConvTask {
  uint32_t src;   // byte offset of the task's values in an FP64 stage; ~0u: no task
  uint32_t base;  // byte offset of digit 0 in a digit stage
  int emax;       // the column's largest biased exponent
};

__device__ __forceinline__ ConvTask conv_task(int k, int lane, int w, const int* s_emax) {
  ConvTask c;
  int a;
  if (k < 8) {
    a = 8 * (k & 3) + (lane & 7);
    const int g = 4 * (k >> 2) + (lane >> 3);
    c.base = (uint32_t)((a >> 3) * kSBO + g * kLBO + (a & 7) * 16);
    c.src = (uint32_t)(a * kColStride + g * 64);
  } else {
    a = 32;
    c.base = (uint32_t)(16 * kSBO + (lane >> 2) * kLBO + (lane & 3) * 4);
    c.src = (uint32_t)(a * kColStride + lane * 16);
  }
  const bool on = a < w;
  if (!on) c.src = ~0u;
  c.emax = s_emax[on ? a : 0];
  return c;
}

template <int N>
__device__ __forceinline__ void split_n(const double (&y)[N], int emax, uint32_t (&zl)[N], uint32_t (&zh)[N]) {
  if (emax >= kFastSplitMinEmax) {
#pragma unroll
    for (int q = 0; q < N; ++q) split_z_fast(y[q], emax, zl[q], zh[q]);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) split_z(y[q], emax, zl[q], zh[q]);
  }
}

// Converts the thread's task of one stage (zeros past n arrive as zeros):
// columns 0..31, 8 rows into 7 digit rows of 8 fp16, one 16-byte store per
// digit; column 32, 2 rows into 7 fp16 pairs.
__device__ __forceinline__ void convert_main(unsigned char* dst, const unsigned char* fst, const ConvTask& c) {
  const double2* src = reinterpret_cast<const double2*>(fst + c.src);
  double y[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 v = src[q];
    y[2 * q] = v.x;
    y[2 * q + 1] = v.y;
  }
  uint32_t zl[8], zh[8];
  split_n<8>(y, c.emax, zl, zh);
  uint32_t wd[4][kDig];
#pragma unroll
  for (int p = 0; p < 4; ++p) digit_words(zl[2 * p], zh[2 * p], zl[2 * p + 1], zh[2 * p + 1], wd[p]);
#pragma unroll
  for (int i = 0; i < kDig; ++i) {
    const uint32_t off = c.base + (uint32_t)i * 4u * kSBO + (i >= 4 ? 2u * kSBO : 0u);
    *reinterpret_cast<uint4*>(dst + off) = make_uint4(wd[0][i], wd[1][i], wd[2][i], wd[3][i]);
  }
}

__device__ __forceinline__ void convert_col32(unsigned char* dst, const unsigned char* fst, const ConvTask& c) {
  const double2 v = *reinterpret_cast<const double2*>(fst + c.src);
  const double y[2] = {v.x, v.y};
  uint32_t zl[2], zh[2], wd[kDig];
  split_n<2>(y, c.emax, zl, zh);
  digit_words(zl[0], zh[0], zl[1], zh[1], wd);
#pragma unroll
  for (int i = 0; i < kDig; ++i) *reinterpret_cast<uint32_t*>(dst + c.base + 16u * i) = wd[i];
}

// Adds an int64 v (|v| < 2^50) to the CTA's sum at word index idx of the slice
// arrays: v = s2 2^34 + s1 2^17 + s0 with s0, s1 in [0, 2^17) and |s2| < 2^16,
// each added by a 32-bit shared-memory reduction. Up to 2^15 additions per
// sum stay exact.
__device__ __forceinline__ void slice_add(uint32_t* acc, int idx, long long v) {
  constexpr int kPlane = kTW * kTW;
  atomicAdd(acc + idx, (uint32_t)(v & 0x1FFFF));
  atomicAdd(acc + kPlane + idx, (uint32_t)((v >> 17) & 0x1FFFF));
  atomicAdd(reinterpret_cast<int*>(acc) + 2 * kPlane + idx, (int)(v >> 34));
}

// The exact int64 value of a sliced sum.
__device__ __forceinline__ long long slice_value(const uint32_t* acc, int idx) {
  constexpr int kPlane = kTW * kTW;
  return ((long long)reinterpret_cast<const int*>(acc)[2 * kPlane + idx] << 34) +
         ((long long)acc[kPlane + idx] << 17) + (long long)acc[idx];
}

// acc += d 2^k for an exact integer product sum d held as an fp32 (|d| <= 2^24):
// one conversion and one wide multiply-add.
template <int K>
__device__ __forceinline__ void add_scaled(long long& acc, uint32_t fbits) {
  const int d = __float2int_rn(__uint_as_float(fbits));
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(d), "r"(1 << K));
}

// Product sum of level L = I + J into hi (L <= 3) or lo (4 <= L <= 7).
template <int L>
__device__ __forceinline__ void level_sum(long long& hi, long long& lo, uint32_t fbits) {
  if constexpr (L <= 3)
    add_scaled<8 * (3 - L)>(hi, fbits);
  else if constexpr (L <= 7)
    add_scaled<8 * (7 - L)>(lo, fbits);
}

// The four columns of tile 0 for each of the seven digit levels J of entries
// b = B0 .. B0 + 3 (TMEM columns t0 + {0, 32, 64, 96, 144, 176, 208}): seven
// loads, then one wait.
__device__ __forceinline__ void tmem_ld4x7(uint32_t t0, uint32_t (&r)[7][4]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%28];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%29];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%30];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%31];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16,%17,%18,%19}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%20,%21,%22,%23}, [%33];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%24,%25,%26,%27}, [%34];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]),
        "=r"(r[1][3]), "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[3][0]), "=r"(r[3][1]),
        "=r"(r[3][2]), "=r"(r[3][3]), "=r"(r[4][0]), "=r"(r[4][1]), "=r"(r[4][2]), "=r"(r[4][3]), "=r"(r[5][0]),
        "=r"(r[5][1]), "=r"(r[5][2]), "=r"(r[5][3]), "=r"(r[6][0]), "=r"(r[6][1]), "=r"(r[6][2]), "=r"(r[6][3])
      : "r"(t0), "r"(t0 + 32), "r"(t0 + 64), "r"(t0 + 96), "r"(t0 + 144), "r"(t0 + 176), "r"(t0 + 208)
      : "memory");
}

// Level J of the four columns held in r, for the T0 digit (I, a) of the
// lane: the product with (J, b) stands for ((I,a),(J,b)), counted when
// a <= b, and, when (J, b) is not in T0 (J >= 4), also for ((J,b),(I,a)),
// counted when b <= a. The sums keep the two kinds apart (near: J <= 3,
// far: J >= 4) and weigh them per entry afterwards.
template <int I, int J>
__device__ __forceinline__ void drain_level(const uint32_t (&r)[4], long long (&hn)[4], long long (&ln)[4],
                                           long long (&lf)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if constexpr (J <= 3)
      level_sum<I + J>(hn[t], ln[t], r[t]);
    else if constexpr (I + J <= 7)
      add_scaled<8 * (7 - (I + J))>(lf[t], r[t]);
  }
}

// Drains the chunk in TMEM columns tq + 0..255 for a warp of lane quarter I:
// half 0 takes tile 0's entries b = 0..15, half 1 entries b = 16..32 and
// tile 1. Sums per entry in registers, then one sliced addition per entry
// into the CTA's sums (acc_hi, acc_lo). Lanes of a warp have distinct a, so
// their entries differ.
template <int I>
__device__ __forceinline__ void drain_quarter(uint32_t tq, int a, int w, uint32_t* acc_hi, uint32_t* acc_lo,
                                              int half) {
#pragma unroll 1
  for (int B0 = 16 * half; B0 < 16 * half + 16; B0 += 4) {
    uint32_t r[7][4];
    tmem_ld4x7(tq + (uint32_t)B0, r);
    long long hn[4], ln[4], lf[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) hn[t] = ln[t] = lf[t] = 0;
    drain_level<I, 0>(r[0], hn, ln, lf);
    drain_level<I, 1>(r[1], hn, ln, lf);
    drain_level<I, 2>(r[2], hn, ln, lf);
    drain_level<I, 3>(r[3], hn, ln, lf);
    drain_level<I, 4>(r[4], hn, ln, lf);
    drain_level<I, 5>(r[5], hn, ln, lf);
    drain_level<I, 6>(r[6], hn, ln, lf);
    if (a < w) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int b = B0 + t;
        if (b >= w) break;
        const bool le = a <= b;
        const long long hi = le ? hn[t] : 0;
        const long long lo = (le ? ln[t] : 0) + (a == b ? 2 * lf[t] : lf[t]);
        const int idx = le ? a * kTW + b : b * kTW + a;
        if (hi != 0) slice_add(acc_hi, idx, hi);
        if (lo != 0) slice_add(acc_lo, idx, lo);
      }
    }
  }
  if (half == 0) return;
  // entry b = 32 (> a): TMEM columns 128..134 hold the digits (J, 32), J = 0..6
  {
    uint32_t r[8];
    tmem_ld8(tq + 128, r);
    long long hi = 0, lo = 0;
    level_sum<I + 0>(hi, lo, r[0]);
    level_sum<I + 1>(hi, lo, r[1]);
    level_sum<I + 2>(hi, lo, r[2]);
    level_sum<I + 3>(hi, lo, r[3]);
    level_sum<I + 4>(hi, lo, r[4]);
    level_sum<I + 5>(hi, lo, r[5]);
    level_sum<I + 6>(hi, lo, r[6]);
    if (a < w && w == kTW) {
      if (hi != 0) slice_add(acc_hi, a * kTW + 32, hi);
      if (lo != 0) slice_add(acc_lo, a * kTW + 32, lo);
    }
  }
  // Tile 1, operand row R = 128 + 32 I + a: columns 0..3 hold D[R, (j, 32)],
  // j = 0..3. Row (i <= 3, 32): ((i,32),(j,32)) -> G_32,32. Row (i >= 4, 32):
  // also ((j,32),(i,32)), so twice. Row (i >= 4, a' <= 31): ((i,a'),(j,32))
  // -> G_a',32.
  if (w == kTW) {
    uint32_t r[16];
    tmem_ld16(tq + kTile1Col, r);
    const int R = 128 + 32 * I + a;
    int i = 0, times = 1, ent = -1;
    if (R < 132) {
      i = R - 128;
      ent = 32 * kTW + 32;
    } else if (R < 135) {
      i = 4 + (R - 132);
      times = 2;
      ent = 32 * kTW + 32;
    } else if (R >= 144 && R < 240) {
      i = 4 + (R - 144) / 32;
      ent = ((R - 144) % 32) * kTW + 32;
    }
    if (ent >= 0) {
      long long hi = 0, lo = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int L = i + j;
        const long long d = (long long)__float2int_rn(__uint_as_float(r[j])) * times;
        if (L <= 3)
          hi += d << (8 * (3 - L));
        else if (L <= 7)
          lo += d << (8 * (7 - L));
      }
      if (hi != 0) slice_add(acc_hi, ent, hi);
      if (lo != 0) slice_add(acc_lo, ent, lo);
    }
  }
}

// The Gram partial of the chunks ch = c_lo, c_lo + c_step, ... < c_hi of the
// rows [row_base, row_base + n_local) of the tensor map's matrix (chunk ch
// starts at row row_base + ch * kTChunk), with the column exponents col_emax,
// written to out[w (w + 1) / 2]. Run by a whole CTA of kTcThreads. guard: the
// wait limit, where a wait that ran out is reported, and the stall test's
// stage (see TcGuard).
__device__ __forceinline__ void gram_tc_body(const CUtensorMap* ymap_p, int w, int64_t row_base, int64_t c_lo,
                                             int64_t c_hi, int64_t c_step, int64_t n_local,
                                             const int* __restrict__ col_emax, double* __restrict__ out,
                                             const TcGuard guard) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* dstage = smem + kDOff;
  unsigned char* fstage = smem + kFOff;
  uint32_t* acc_hi = reinterpret_cast<uint32_t*>(smem + kAccOff);  // [3][33][33] slices
  uint32_t* acc_lo = acc_hi + kSlices * kTW * kTW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBarOff);
  uint64_t* f_full = bars;                  // tensor copy landed (tx count)
  uint64_t* f_empty = bars + kFStages;      // converters done reading
  uint64_t* d_full = bars + 2 * kFStages;   // converters done writing digits
  uint64_t* d_empty = d_full + kDStages;    // MMAs done reading digits
  uint64_t* acc_full = d_empty + kDStages;  // [2] a chunk's MMAs are complete
  uint64_t* acc_empty = acc_full + 2;       // [2] its accumulators are drained
  uint64_t* mma_done = acc_empty + 2;       // [2] per issuer: its MMAs are complete (error path)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kSlotOff);
  int* s_emax = reinterpret_cast<int*>(smem + kEmaxOff);
  volatile int* s_err = reinterpret_cast<volatile int*>(smem + kErrOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // digit rows never written stay zero; the sums start at zero
  for (uint32_t o = tid * 16; o < kDStages * kDStageBytes; o += kTcThreads * 16)
    *reinterpret_cast<uint4*>(dstage + o) = make_uint4(0, 0, 0, 0);
  for (int k = tid; k < 2 * kSlices * kTW * kTW; k += kTcThreads) acc_hi[k] = 0u;
  if (tid < kTW) s_emax[tid] = tid < w ? col_emax[tid] : 0;
  if (tid == 0) {
    *s_err = 0;
    for (int k = 0; k < kFStages; ++k) {
      bar_init(f_full + k, 1);
      bar_init(f_empty + k, kGroupWarps);
    }
    for (int k = 0; k < kDStages; ++k) {
      bar_init(d_full + k, kGroupWarps);
      bar_init(d_empty + k, 2);  // both issuers commit
    }
    for (int k = 0; k < 2; ++k) {
      bar_init(acc_full + k, 2);
      bar_init(acc_empty + k, kDrainWarps);
      bar_init(mma_done + k, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const int64_t n = n_local;
  const uint32_t lim = (uint32_t)(guard.wait_limit < 0xFFFFFFFFll ? guard.wait_limit : 0xFFFFFFFFll);
  const bool stall_here = guard.stall_stage >= 0 && blockIdx.x == 0;
  uint32_t armed = 0;   // loader: stages whose copies were issued
  uint32_t issued = 0;  // MMA issuers: stages whose MMAs this thread issued

  if (warp < kConvWarps) {
    // ---- converters: group G takes the stages t with t % 2 == G ----
    const uint32_t G = warp >= kGroupWarps ? 1u : 0u;
    const int k = warp - (int)G * kGroupWarps;
    const ConvTask task = conv_task(k, lane, w, s_emax);
    uint32_t T = 0;  // stages of this CTA
    for (int64_t ch = c_lo; ch < c_hi; ch += c_step) {
      const int64_t left = (n - ch * kTChunk + kSub - 1) / kSub;
      T += (uint32_t)(left < kSubPerChunk ? left : kSubPerChunk);
    }
    // stage t: staging slot fs = t % kFStages of parity fpar = (t / kFStages) & 1,
    // digit slot ds = t % kDStages with dq = t / kDStages
    uint32_t fs = G, fpar = 0, ds = G, dq = 0;
    for (uint32_t t = G; t < T; t += 2) {
      if (!bar_wait(f_full + fs, fpar, s_err, lim)) goto done;
      if (t >= kDStages && !bar_wait(d_empty + ds, (dq - 1) & 1, s_err, lim)) goto done;
      if (task.src != ~0u) {
        if (k < 8)
          convert_main(dstage + ds * kDStageBytes, fstage + fs * kFStageBytes, task);
        else
          convert_col32(dstage + ds * kDStageBytes, fstage + fs * kFStageBytes, task);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        bar_arrive(f_empty + fs);
        bar_arrive(d_full + ds);
      }
      fs += 2;
      if (fs >= (uint32_t)kFStages) {
        fs -= kFStages;
        fpar ^= 1;
      }
      ds += 2;
      if (ds >= (uint32_t)kDStages) {
        ds -= kDStages;
        ++dq;
      }
    }
  } else if (warp < kDrainWarp0 + kDrainWarps) {
    // ---- drain: warp of lane quarter I folds each chunk into the sums ----
    const int I = warp & 3;
    const uint32_t tl = tbase + ((uint32_t)(I * 32) << 16);
    uint32_t cu = 0;
    for (int64_t ch = c_lo; ch < c_hi; ch += c_step, ++cu) {
      const uint32_t p = cu & 1;
      if (!bar_wait(acc_full + p, (cu >> 1) & 1, s_err, lim)) goto done;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tq = tl + 256u * p;
      switch (I) {
        case 0: drain_quarter<0>(tq, lane, w, acc_hi, acc_lo, (warp - kDrainWarp0) >> 2); break;
        case 1: drain_quarter<1>(tq, lane, w, acc_hi, acc_lo, (warp - kDrainWarp0) >> 2); break;
        case 2: drain_quarter<2>(tq, lane, w, acc_hi, acc_lo, (warp - kDrainWarp0) >> 2); break;
        default: drain_quarter<3>(tq, lane, w, acc_hi, acc_lo, (warp - kDrainWarp0) >> 2); break;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(acc_empty + p);
    }
  } else if (warp == kLoadWarp) {
    // ---- loader: one tensor copy per stage ----
    if (lane == 0) {
      uint32_t t = 0;
      for (int64_t ch = c_lo; ch < c_hi; ch += c_step) {
        const int64_t left = (n - ch * kTChunk + kSub - 1) / kSub;
        const int nsub = left < kSubPerChunk ? (int)left : kSubPerChunk;
        for (int sub = 0; sub < nsub; ++sub, ++t) {
          const int fs = (int)(t % kFStages);
          if (t >= kFStages && !bar_wait(f_empty + fs, (t / kFStages - 1) & 1, s_err, lim)) goto done;
          armed = t + 1;
          if (stall_here && t == (uint32_t)guard.stall_stage) continue;  // the stall test: never armed
          bar_expect_tx(f_full + fs, kFBoxBytes);
          tensor_g2s(fstage + fs * kFStageBytes, ymap_p, (int)(row_base + ch * kTChunk + (int64_t)sub * kSub),
                     f_full + fs);
        }
      }
    }
  } else if (warp == kMmaWarp || warp == kMma1Warp) {
    // ---- MMA issue: tile 0 (rows 0..127 x 0..239) or tile 1 (rows 128..255 x 128..143) ----
    if (lane == 0) {
      const bool t0 = warp == kMmaWarp;
      const uint32_t aoff = t0 ? 0u : 16u * kSBO;  // operand row 0 or 128
      const uint32_t idesc = t0 ? instr_desc(128, kN0) : instr_desc(128, kN1);
      uint32_t t = 0, cu = 0;
      for (int64_t ch = c_lo; ch < c_hi; ch += c_step, ++cu) {
        const int64_t left = (n - ch * kTChunk + kSub - 1) / kSub;
        const int nsub = left < kSubPerChunk ? (int)left : kSubPerChunk;
        const uint32_t p = cu & 1;
        if (cu >= 2 && !bar_wait(acc_empty + p, ((cu >> 1) - 1) & 1, s_err, lim)) goto done;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d0 = tbase + 256u * p + (t0 ? 0u : (uint32_t)kTile1Col);
        for (int sub = 0; sub < nsub; ++sub, ++t) {
          const int ds = (int)(t % kDStages);
          if (!bar_wait(d_full + ds, (t / kDStages) & 1, s_err, lim)) goto done;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sb = smem_u32(dstage + ds * kDStageBytes) + aoff;
#pragma unroll
          for (int ks = 0; ks < kSub / 16; ++ks) {
            const uint64_t desc = smem_desc(sb + ks * 2 * kLBO);
            mma_f16(d0, desc, desc, idesc, (sub > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(d_empty + ds);
          issued = t + 1;
        }
        mma_commit(acc_full + p);
      }
    }
  }
done:
  if (*s_err) {
    // error path: let the copies and MMAs already in flight land first
    if (warp == kLoadWarp && lane == 0)
      for (uint32_t k = armed > (uint32_t)kFStages ? armed - kFStages : 0; k < armed; ++k)
        bar_drain(f_full + k % kFStages, (k / kFStages) & 1, lim);
    if ((warp == kMmaWarp || warp == kMma1Warp) && lane == 0 && issued > 0) {
      mma_commit(mma_done + (warp - kMmaWarp));  // tracks this thread's MMAs only
      bar_drain(mma_done + (warp - kMmaWarp), 0, lim);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  const int ok = !*s_err;
  if (!ok && tid == 0 && guard.err) atomicExch(guard.err, (int)ASCG_ERR_TIMEOUT);
  const int np = w * (w + 1) / 2;
  for (int p = tid; p < np; p += kTcThreads) {
    int a = 0, rem = p;
    while (rem >= w - a) {
      rem -= w - a;
      ++a;
    }
    const int b = a + rem;
    double v;
    if (!ok || s_emax[a] == 0x7ff || s_emax[b] == 0x7ff) {
      v = CUDART_NAN;
    } else {
      const long long hi = slice_value(acc_hi, a * kTW + b), lo = slice_value(acc_lo, a * kTW + b);
      // G_ab = 2^(E_a + E_b - 14) (hi 2^-24 + lo 2^-56), E = emax - 1022
      const double s = ldexp((double)hi, -24) + ldexp((double)lo, -56);
      v = ldexp(s, s_emax[a] + s_emax[b] - 2058);
    }
    out[p] = v;
  }
  if (warp == kMmaWarp) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
  }
}

// One matrix: CTA b takes the chunks b, b + gridDim.x, ... of the n rows.
__global__ void __launch_bounds__(kTcThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap ymap, int64_t n, int w, const int* __restrict__ col_emax,
                   double* __restrict__ partials, const TcGuard guard) {
  pdl_wait();
  pdl_release();
  if (guard.gate && !*guard.gate) return;  // uniform, before any barrier or tensor memory
  gram_tc_body(&ymap, w, 0, blockIdx.x, (n + kTChunk - 1) / kTChunk, gridDim.x, n, col_emax,
               partials + (int64_t)blockIdx.x * (w * (w + 1) / 2), guard);
}

// Many systems whose bases are row ranges of one matrix (the tensor map's):
// CTA q takes item q, whole chunks of one system (rows [row0, row0 + nrows),
// nrows a multiple of kTChunk), with that system's column exponents
// (emax_all + sys * kTW). Items of systems with sys_w 0 skip.
__global__ void __launch_bounds__(kTcThreads, 1)
    gram_tc_items_kernel(const __grid_constant__ CUtensorMap ymap, int w, const GramItem* __restrict__ items,
                         const int* __restrict__ sys_w, const int* __restrict__ emax_all,
                         double* __restrict__ partials) {
  const GramItem it = items[blockIdx.x];
  if (sys_w[it.sys] == 0) return;  // uniform over the CTA, before any barrier
  const int64_t nch = it.nrows / kTChunk;
  gram_tc_body(&ymap, w, it.row0, 0, nch, 1, nch * kTChunk, emax_all + (int64_t)it.sys * kTW,
               partials + (int64_t)blockIdx.x * (w * (w + 1) / 2), TcGuard{kWaitLimit, -1, nullptr, nullptr});
}

// Largest biased exponent of each column, reduced into col_emax (zeroed
// before the launch) with one atomicMax per column and CTA. Rows are split
// into even-sized ranges; 16-byte loads, four in flight per thread.
constexpr int kExpBlocks = 1216;
__global__ void __launch_bounds__(256) col_exponent_kernel(int64_t n, int w, const double* __restrict__ Y,
                                                           int64_t ldY, int* __restrict__ col_emax) {
  __shared__ unsigned red[8][kTW];
  const int64_t per = (((n + gridDim.x - 1) / gridDim.x) + 1) & ~1ll;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = n < r0 + per ? n : r0 + per;
  const int64_t full = r1 > r0 ? (r1 - r0) >> 1 : 0;  // whole double2 slots
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto ex = [](double v) { return ((unsigned)__double2hiint(v) >> 20) & 0x7ffu; };
  for (int a = 0; a < w; ++a) {
    const double2* col = reinterpret_cast<const double2*>(Y + (int64_t)a * ldY + r0);
    unsigned m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int64_t q = threadIdx.x;
    for (; q + 768 < full; q += 1024) {
      const double2 v0 = __ldcs(col + q), v1 = __ldcs(col + q + 256), v2 = __ldcs(col + q + 512),
                    v3 = __ldcs(col + q + 768);
      m0 = max(m0, max(ex(v0.x), ex(v0.y)));
      m1 = max(m1, max(ex(v1.x), ex(v1.y)));
      m2 = max(m2, max(ex(v2.x), ex(v2.y)));
      m3 = max(m3, max(ex(v3.x), ex(v3.y)));
    }
    for (; q < full; q += 256) {
      const double2 v = __ldcs(col + q);
      m0 = max(m0, max(ex(v.x), ex(v.y)));
    }
    if (threadIdx.x == 0 && r0 + 2 * full < r1) m0 = max(m0, ex(Y[(int64_t)a * ldY + r0 + 2 * full]));
    const unsigned m = __reduce_max_sync(0xffffffffu, max(max(m0, m1), max(m2, m3)));
    if (lane == 0) red[warp][a] = m;
  }
  __syncthreads();
  if (threadIdx.x < w) {
    unsigned m = 0;
    for (int g = 0; g < 8; ++g) m = max(m, red[g][threadIdx.x]);
    if (m > 0) atomicMax(col_emax + threadIdx.x, (int)m);
  }
}

// Column exponents of many systems: CTA q takes item q (the rows of one
// system) and folds the largest biased exponent of each of its w columns into
// emax_all[sys * kTW + c] (zeroed before the launch).
__global__ void __launch_bounds__(256) tc_items_exponent_kernel(int w, const double* __restrict__ Y, int64_t ldY,
                                                                const GramItem* __restrict__ items,
                                                                const int* __restrict__ sys_w,
                                                                int* __restrict__ emax_all) {
  __shared__ unsigned red[8][kTW];
  const GramItem it = items[blockIdx.x];
  if (sys_w[it.sys] == 0) return;  // uniform over the CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto ex = [](double v) { return ((unsigned)__double2hiint(v) >> 20) & 0x7ffu; };
  for (int a = 0; a < w; ++a) {
    const double2* col = reinterpret_cast<const double2*>(Y + (int64_t)a * ldY + it.row0);
    unsigned m0 = 0, m1 = 0;
    int64_t q = threadIdx.x;
    for (; q + 256 < it.nrows / 2; q += 512) {
      const double2 v0 = __ldcs(col + q), v1 = __ldcs(col + q + 256);
      m0 = max(m0, max(ex(v0.x), ex(v0.y)));
      m1 = max(m1, max(ex(v1.x), ex(v1.y)));
    }
    for (; q < it.nrows / 2; q += 256) {
      const double2 v = __ldcs(col + q);
      m0 = max(m0, max(ex(v.x), ex(v.y)));
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, max(m0, m1));
    if (lane == 0) red[warp][a] = m;
  }
  __syncthreads();
  if (threadIdx.x < w) {
    unsigned m = 0;
    for (int g = 0; g < 8; ++g) m = max(m, red[g][threadIdx.x]);
    if (m > 0) atomicMax(emax_all + (int64_t)it.sys * kTW + threadIdx.x, (int)m);
  }
}

// ---------------------------------------------------------------------------
// Recovery (eq. coords) on the tensor cores: x += Y x', r = Y r', p = Y p' in
// one pass over Y, with the digit split of the Gram.
//
// Per column j, Y_ij = Yt_ij 2^(E_j - 55), Yt the truncated 55-bit integer of
// the Gram in seven balanced base-256 digits. The coefficients take the column
// scale in, u_vj = c_vj 2^(E_j - 55) (exact), and get one exponent per vector
// v (x', r', p'): u_vj = ut_vj 2^(F_v - 55), ut again a truncated 55-bit
// integer in seven digits. Then sum_j Y_ij c_vj = 2^(F_v - 55) sum_j Yt_ij
// ut_vj, and digit d of Yt times digit e of ut weighs 256^(12 - d - e).
// One MMA chain per 128 rows of Y (M = 128, K = 231 = 33 columns x 7 digits
// padded to 240, N = 24 = 3 vectors x 8 levels padded to 32) forms
// D[i, (v, L)] = sum_{j, d} yt_ijd ut_vj(L-d): each sum holds the products of
// one level L = d + e, exact in FP32 (|D| < 2^22). Levels L >= 8 are dropped
// (below 2^-56 of the largest product). Per row and vector,
// T = sum_{L <= 7} D_L 256^(7 - L) = T_hi 2^32 + T_lo (two int64), and the
// result T 2^(F_v - 15) is rounded once to FP64 (one fma).
// Error against the exact sum_j Y_ij c_vj: at most 2^-53 |result| +
// 2^-54 sum_j ||y_j||_inf |c_vj| + (w + 2) 2^-52 max_j ||y_j||_inf |c_vj|, a
// normwise bound like the Gram's (the FP64 recovery's is componentwise,
// gamma_w sum_j |Y_ij c_vj|).
//
// Pipeline, 26 warps: a loader thread (one tensor-map copy of 128 rows x 33
// columns per tile, two staging slots); 20 converter warps (16 take 8 columns
// of one row each, 4 take column 32), two digit slots; one MMA thread, the
// 15 K-steps of a tile alternating between two accumulators so that
// consecutive MMAs do not wait on each other; 4 drain warps, one per TMEM
// lane quarter, each lane one row. All waits are bounded, as in the Gram.
constexpr int kRTile = 128;                         // rows of Y per tile (MMA M)
constexpr int kRK = 240;                            // MMA K: 224 (digits x columns 0..31) + 7 (column 32) + 9 zeros
constexpr uint32_t kRSBO = (kRK / 8) * 128;         // bytes between 8-row groups (3840)
constexpr uint32_t kRABytes = (kRTile / 8) * kRSBO; // one digit tile (61440)
constexpr uint32_t kRFBytes = kTW * kRTile * 8;     // one staging tile (33792)
constexpr uint32_t kRBBytes = 4 * kRSBO;            // coefficient digits, 32 rows (15360)
constexpr int kRN = 32;                             // MMA N: (v, L) = 8 v + L
constexpr int kRConvWarps = 20, kRDrainWarp0 = 20, kRLoadWarp = 24, kRMmaWarp = 25;
constexpr int kRThreads = 26 * 32;
constexpr size_t kRAOff = 0;
constexpr size_t kRFOff = kRAOff + 2 * (size_t)kRABytes;
constexpr size_t kRBOff = kRFOff + 2 * (size_t)kRFBytes;
constexpr size_t kRBarOff = kRBOff + kRBBytes;
constexpr int kRNumBars = 13;
constexpr size_t kRSlotOff = kRBarOff + 8 * kRNumBars;
constexpr size_t kREmaxOff = kRSlotOff + 16;
constexpr size_t kRFvOff = (kREmaxOff + 4 * kTW + 15) / 16 * 16;  // int[4]: per-vector exponents, a NaN flag
constexpr size_t kRScaleOff = kRFvOff + 16;        // double[3]
constexpr size_t kRErrOff = kRScaleOff + 24;
constexpr size_t kRSmem = kRErrOff + 16;
static_assert(kRFOff % 1024 == 0 && kRBOff % 1024 == 0 && kRBarOff % 8 == 0 && kRScaleOff % 8 == 0, "alignment");
static_assert(kRSmem <= 227 * 1024, "shared memory per CTA");

// Byte offset of operand row R, K index k (a multiple of 8), in a digit tile.
__host__ __device__ constexpr uint32_t rec_off(int R, int k) {
  return (uint32_t)((R >> 3) * kRSBO + (k >> 3) * 128 + (R & 7) * 16);
}

__device__ __forceinline__ uint64_t rec_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kRSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tmem_ld8x2(uint32_t a0, uint32_t a1, uint32_t (&r)[2][8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
        "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
        "=r"(r[1][6]), "=r"(r[1][7])
      : "r"(a0), "r"(a1)
      : "memory");
}

// One row and vector: the levels L = 0..7 in two accumulators (e, o) to the
// FP64 value T 2^(F_v - 15), scale = 2^(F_v - 15).
__device__ __forceinline__ double rec_value(const uint32_t (&e)[8], const uint32_t (&o)[8], double scale) {
  long long hi = 0, lo = 0;
#pragma unroll
  for (int L = 0; L < 8; ++L) {
    const int d = __float2int_rn(__uint_as_float(e[L]) + __uint_as_float(o[L]));  // exact: |e|, |o| < 2^21
    if (L <= 3)
      asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(hi) : "r"(d), "r"(1 << (8 * (3 - L))));
    else
      asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(lo) : "r"(d), "r"(1 << (8 * (7 - L))));
  }
  // |hi|, |lo| < 2^47: both exact in FP64; one rounding in the fma
  return fma((double)hi, 4294967296.0, (double)lo) * scale;
}

__global__ void __launch_bounds__(kRThreads, 1)
    recover_tc_kernel(const __grid_constant__ CUtensorMap ymap, int64_t n, int w, const int* __restrict__ col_emax,
                      const double* __restrict__ coords, double* __restrict__ x, double* __restrict__ r,
                      double* __restrict__ p, const TcGuard guard) {
  pdl_wait();
  pdl_release();
  // uniform, before any barrier or tensor memory: a block enqueued ahead with
  // nothing to do, or one whose Gram already failed (its error word is set),
  // leaves x, r and p alone
  if ((guard.gate && !*guard.gate) || (guard.err && *guard.err != 0)) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* astage = smem + kRAOff;
  unsigned char* fstage = smem + kRFOff;
  unsigned char* bop = smem + kRBOff;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kRBarOff);
  uint64_t* f_full = bars;          // [2] tensor copy landed
  uint64_t* f_empty = bars + 2;     // [2] converters done reading
  uint64_t* a_full = bars + 4;      // [2] digits written
  uint64_t* a_empty = bars + 6;     // [2] MMAs done reading them
  uint64_t* acc_full = bars + 8;    // [2] a tile's MMAs complete
  uint64_t* acc_empty = bars + 10;  // [2] its accumulators drained
  uint64_t* mma_done = bars + 12;   // the MMA thread's MMAs complete (error path)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kRSlotOff);
  int* s_emax = reinterpret_cast<int*>(smem + kREmaxOff);
  int* s_fv = reinterpret_cast<int*>(smem + kRFvOff);
  double* s_scale = reinterpret_cast<double*>(smem + kRScaleOff);
  volatile int* s_err = reinterpret_cast<volatile int*>(smem + kRErrOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // digit tiles and coefficient digits start at zero (padding stays zero)
  for (uint32_t o = tid * 16; o < 2 * kRABytes; o += kRThreads * 16)
    *reinterpret_cast<uint4*>(astage + o) = make_uint4(0, 0, 0, 0);
  for (uint32_t o = tid * 16; o < kRBBytes; o += kRThreads * 16)
    *reinterpret_cast<uint4*>(bop + o) = make_uint4(0, 0, 0, 0);
  if (tid < kTW) s_emax[tid] = tid < w ? col_emax[tid] : 0;
  if (tid < 4) s_fv[tid] = 0;
  if (tid == 0) {
    *s_err = 0;
    for (int k = 0; k < 2; ++k) {
      bar_init(f_full + k, 1);
      bar_init(f_empty + k, kRConvWarps);
      bar_init(a_full + k, kRConvWarps);
      bar_init(a_empty + k, 1);
      bar_init(acc_full + k, 1);
      bar_init(acc_empty + k, 4);
    }
    bar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kRMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  // coefficients: u_vj = c_vj 2^(E_j - 55), E_j = emax_j - 1022; per vector the
  // largest biased exponent f_v; a NaN or infinite column or coefficient
  // makes every result NaN
  const int cv = tid / kTW, cj = tid % kTW;
  const bool cthr = tid < 3 * kTW && cj < w;
  double u = 0.0;
  if (cthr) {
    // a zero column (emax 0) takes no part: its digits are all zero
    u = s_emax[cj] == 0 ? 0.0 : ldexp(coords[cv * w + cj], s_emax[cj] - 1077);
    const int eu = (__double2hiint(u) >> 20) & 0x7ff;
    atomicMax(s_fv + cv, eu);
    if (eu == 0x7ff || s_emax[cj] == 0x7ff) atomicMax(s_fv + 3, 1);
  }
  __syncthreads();
  if (cthr) {
    // B[(v, L), (j, d)] = digit L - d of ut_vj: column j <= 31 at K = 32 d + j,
    // column 32 at K = 224 + d
    uint32_t zl, zh, dw[kDig];
    split_z(u, s_fv[cv], zl, zh);
    digit_words(zl, zh, zl, zh, dw);
    unsigned short* b16 = reinterpret_cast<unsigned short*>(bop);
#pragma unroll
    for (int d = 0; d < kDig; ++d)
#pragma unroll
      for (int e = 0; e < kDig; ++e) {
        if (d + e > 7) continue;
        const int R = 8 * cv + d + e, k = cj <= 31 ? 32 * d + cj : 224 + d;
        b16[(rec_off(R, k & ~7) + (k & 7) * 2) / 2] = (unsigned short)(dw[e] & 0xFFFFu);
      }
  }
  if (tid < 3) s_scale[tid] = ldexp(1.0, s_fv[tid] - 1037);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const int64_t ntiles = (n + kRTile - 1) / kRTile;
  const uint32_t T = ntiles > blockIdx.x ? (uint32_t)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0u;
  const uint32_t lim = (uint32_t)(guard.wait_limit < 0xFFFFFFFFll ? guard.wait_limit : 0xFFFFFFFFll);
  uint32_t armed = 0, issued = 0;

  if (warp < kRConvWarps) {
    // ---- converters: warp k < 16 takes columns 8 (k & 3) .. + 7 of row
    // 32 (k >> 2) + lane; warps 16..19 column 32 of row 32 (k - 16) + lane ----
    const bool col32 = warp >= 16;
    const int jb = warp & 3;
    const int row = col32 ? 32 * (warp - 16) + lane : 32 * (warp >> 2) + lane;
    const bool on = col32 ? w == kTW : 8 * jb < w;
    // the columns' exponents, the same in every lane of the warp
    int em[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) em[c] = s_emax[col32 ? 32 : 8 * jb + c];
    bool all_fast = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) all_fast = all_fast && em[c] >= kFastSplitMinEmax;
    for (uint32_t t = 0; t < T; ++t) {
      const uint32_t s = t & 1, par = (t >> 1) & 1;
      if (!bar_wait(f_full + s, par, s_err, lim)) goto rdone;
      if (t >= 2 && !bar_wait(a_empty + s, par ^ 1, s_err, lim)) goto rdone;
      if (on) {
        const double* f = reinterpret_cast<const double*>(fstage + s * kRFBytes);
        unsigned char* dst = astage + s * kRABytes;
        if (!col32) {
          double y[8];
          uint32_t zl[8], zh[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) y[c] = f[(8 * jb + c) * kRTile + row];
          if (all_fast) {
#pragma unroll
            for (int c = 0; c < 8; ++c) split_z_fast(y[c], em[c], zl[c], zh[c]);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) split_z(y[c], em[c], zl[c], zh[c]);
          }
          uint32_t wd[4][kDig];
#pragma unroll
          for (int q = 0; q < 4; ++q) digit_words(zl[2 * q], zh[2 * q], zl[2 * q + 1], zh[2 * q + 1], wd[q]);
#pragma unroll
          for (int d = 0; d < kDig; ++d)
            *reinterpret_cast<uint4*>(dst + rec_off(row, 32 * d + 8 * jb)) =
                make_uint4(wd[0][d], wd[1][d], wd[2][d], wd[3][d]);
        } else {
          const double y = f[32 * kRTile + row];
          uint32_t zl, zh, dw[kDig];
          if (all_fast)
            split_z_fast(y, em[0], zl, zh);
          else
            split_z(y, em[0], zl, zh);
          digit_words(zl, zh, zl, zh, dw);
          // digits 0..6 at K = 224..230, K = 231 zero
          *reinterpret_cast<uint4*>(dst + rec_off(row, 224)) =
              make_uint4(__byte_perm(dw[0], dw[1], 0x5410), __byte_perm(dw[2], dw[3], 0x5410),
                         __byte_perm(dw[4], dw[5], 0x5410), dw[6] & 0xFFFFu);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        bar_arrive(f_empty + s);
        bar_arrive(a_full + s);
      }
    }
  } else if (warp < kRDrainWarp0 + 4) {
    // ---- drain: lane quarter q, one row per lane ----
    const int q = warp & 3;
    const bool bad = s_fv[3] != 0;
    const double sc0 = s_scale[0], sc1 = s_scale[1], sc2 = s_scale[2];
    for (uint32_t t = 0; t < T; ++t) {
      const uint32_t b = t & 1;
      if (!bar_wait(acc_full + b, (t >> 1) & 1, s_err, lim)) goto rdone;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 64u * b;
      uint32_t v0[2][8], v1[2][8], v2[2][8];
      tmem_ld8x2(ta + 0, ta + 32, v0);
      tmem_ld8x2(ta + 8, ta + 40, v1);
      tmem_ld8x2(ta + 16, ta + 48, v2);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(acc_empty + b);
      const int64_t i = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * kRTile + 32 * q + lane;
      if (i < n) {
        double dx = rec_value(v0[0], v0[1], sc0), dr = rec_value(v1[0], v1[1], sc1),
               dp = rec_value(v2[0], v2[1], sc2);
        if (bad) dx = dr = dp = CUDART_NAN;
        x[i] = x[i] + dx;
        r[i] = dr;
        p[i] = dp;
      }
    }
  } else if (warp == kRLoadWarp) {
    if (lane == 0) {
      for (uint32_t t = 0; t < T; ++t) {
        const uint32_t s = t & 1;
        if (t >= 2 && !bar_wait(f_empty + s, ((t >> 1) & 1) ^ 1, s_err, lim)) goto rdone;
        armed = t + 1;
        bar_expect_tx(f_full + s, kRFBytes);
        tensor_g2s(fstage + s * kRFBytes, &ymap, (int)(((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * kRTile),
                   f_full + s);
      }
    }
  } else if (warp == kRMmaWarp) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(128, kRN);
      const uint32_t bbase = smem_u32(bop);
      for (uint32_t t = 0; t < T; ++t) {
        const uint32_t s = t & 1, b = t & 1;
        if (!bar_wait(a_full + s, (t >> 1) & 1, s_err, lim)) goto rdone;
        if (t >= 2 && !bar_wait(acc_empty + b, ((t >> 1) & 1) ^ 1, s_err, lim)) goto rdone;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t abase = smem_u32(astage + s * kRABytes);
        const uint32_t d0 = tbase + 64u * b;
#pragma unroll
        for (int ks = 0; ks < kRK / 16; ++ks)
          mma_f16(d0 + 32u * (ks & 1), rec_desc(abase + 256u * ks), rec_desc(bbase + 256u * ks), idesc,
                  ks >= 2 ? 1u : 0u);
        mma_commit(a_empty + s);
        mma_commit(acc_full + b);
        issued = t + 1;
      }
    }
  }
rdone:
  if (*s_err) {
    if (warp == kRLoadWarp && lane == 0)
      for (uint32_t k = armed > 2u ? armed - 2u : 0u; k < armed; ++k) bar_drain(f_full + (k & 1), (k >> 1) & 1, lim);
    if (warp == kRMmaWarp && lane == 0 && issued > 0) {
      mma_commit(mma_done);
      bar_drain(mma_done, 0, lim);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*s_err && tid == 0 && guard.err) atomicExch(guard.err, (int)ASCG_ERR_TIMEOUT);
  if (warp == kRMmaWarp) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tbase));
  }
}

// cuTensorMapEncodeTiled, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

cudaError_t encode_map(CUtensorMap* map, const double* Y, int64_t n, int w, int64_t ldY, int box_rows = kBoxRows) {
  {
    std::lock_guard<std::mutex> lock(g_encode_mu);
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)w};
  const cuuint64_t strides[1] = {(cuuint64_t)ldY * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)kTW};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(Y), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

std::atomic<uint64_t> g_tc_smem_set{0}, g_tc_items_smem_set{0}, g_rec_smem_set{0};

}  // namespace

int gram_tc_parts(int64_t n) {
  const int64_t chunks = (n + kTChunk - 1) / kTChunk;
  const int g = gram_grid();
  return (int)(chunks < g ? chunks : g);
}

bool gram_tc_applies(int w) { return w >= kGramTcMinW && w <= kTW; }

bool gram_tc_aligned(const double* Y, int64_t ldY) {
  return (reinterpret_cast<uintptr_t>(Y) & 15) == 0 && (ldY & 1) == 0;
}

bool gram_tc_fits(int64_t n) {
  // a sliced sum takes <= 10 additions per chunk: at most 2^11 chunks per CTA
  return n >= 1 && n <= 0x7fffffffll && (n + kTChunk - 1) / kTChunk <= (int64_t)gram_tc_parts(n) * 2048;
}

cudaError_t launch_gram_tc(int64_t n, int w, const double* Y, int64_t ldY, int* exp_parts, bool emax_ready,
                           double* partials, cudaStream_t s, int* err, bool stall_test, const int* gate) {
  if (w < 1 || w > kTW || !gram_tc_fits(n) || !gram_tc_aligned(Y, ldY)) return cudaErrorInvalidValue;
  const int parts = gram_tc_parts(n);
  cudaError_t e = smem_limit_once(g_tc_smem_set, gram_tc_kernel, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  e = encode_map(&map, Y, n, w, ldY);
  if (e != cudaSuccess) return e;
  if (!emax_ready) {
    e = cudaMemsetAsync(exp_parts, 0, sizeof(int) * kTW, s);
    if (e != cudaSuccess) return e;
    const int64_t eb = (n + 255) / 256;
    col_exponent_kernel<<<(int)(eb < kExpBlocks ? eb : kExpBlocks), 256, 0, s>>>(n, w, Y, ldY, exp_parts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const TcGuard guard{stall_test ? kTestWaitLimit : kWaitLimit, stall_test ? 0 : -1, err, gate};
  return launch_pdl_ex(gram_tc_kernel, dim3(parts), dim3(kTcThreads), kTcSmem, s, map, n, w, exp_parts, partials,
                       guard);
}

cudaError_t launch_gram_tc_items(int w, const double* Y, int64_t ldY, int64_t rows, const GramItem* items,
                                 int nitems, const int* sys_w, int nsys, int* emax_all, double* partials,
                                 cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  if (!gram_tc_applies(w) || !gram_tc_aligned(Y, ldY) || rows < 1 || rows > 0x7fffffffll || rows > ldY ||
      (rows % kTChunk) != 0)
    return cudaErrorInvalidValue;
  cudaError_t e = smem_limit_once(g_tc_items_smem_set, gram_tc_items_kernel, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  e = encode_map(&map, Y, rows, w, ldY);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(emax_all, 0, sizeof(int) * kTW * nsys, s);
  if (e != cudaSuccess) return e;
  tc_items_exponent_kernel<<<nitems, 256, 0, s>>>(w, Y, ldY, items, sys_w, emax_all);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_tc_items_kernel<<<nitems, kTcThreads, kTcSmem, s>>>(map, w, items, sys_w, emax_all, partials);
  return cudaGetLastError();
}

cudaError_t launch_recover_tc(int64_t n, int w, const double* Y, int64_t ldY, const int* col_emax,
                              const double* coords, double* x, double* r, double* p, cudaStream_t s, int* err,
                              const int* gate) {
  if (!gram_tc_applies(w) || !gram_tc_aligned(Y, ldY) || n < 1 || n > 0x7fffffffll) return cudaErrorInvalidValue;
  cudaError_t e = smem_limit_once(g_rec_smem_set, recover_tc_kernel, (int)kRSmem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  e = encode_map(&map, Y, n, w, ldY, kRTile);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kRTile - 1) / kRTile;
  const int g = gram_grid();
  const TcGuard guard{kWaitLimit, -1, err, gate};
  return launch_pdl_ex(recover_tc_kernel, dim3((unsigned)(tiles < g ? tiles : g)), dim3(kRThreads), kRSmem, s, map, n,
                       w, col_emax, coords, x, r, p, guard);
}

cudaError_t launch_col_exponents(int64_t n, int w, const double* Y, int64_t ldY, int* col_emax, cudaStream_t s) {
  if (w < 1 || w > kTW || n < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(col_emax, 0, sizeof(int) * kTW, s);
  if (e != cudaSuccess) return e;
  const int64_t eb = (n + 255) / 256;
  col_exponent_kernel<<<(int)(eb < kExpBlocks ? eb : kExpBlocks), 256, 0, s>>>(n, w, Y, ldY, col_emax);
  return cudaGetLastError();
}

cudaError_t launch_gram_any(int64_t n, int w, const double* Y, int64_t ldY, bool force_fp64, int* exp_parts,
                            bool emax_ready, double* partials, int* nparts, cudaStream_t s, int* err,
                            bool stall_test, const int* gate) {
  if (!force_fp64 && gram_tc_applies(w) && gram_tc_aligned(Y, ldY) && gram_tc_fits(n)) {
    *nparts = gram_tc_parts(n);
    return launch_gram_tc(n, w, Y, ldY, exp_parts, emax_ready, partials, s, err, stall_test, gate);
  }
  *nparts = gram_parts(n);
  return launch_gram_partial(n, w, Y, ldY, partials, s, gate);
}

}  // namespace ascg
