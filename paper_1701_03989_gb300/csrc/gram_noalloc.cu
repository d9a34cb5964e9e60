// ascg_gram_noalloc: the Gram matrix G = Y^T Y without any device allocation.
//
// ascg_gram obtains its per-CTA partial sums from cudaMalloc and releases them
// with cudaFree on every call. Some callers cannot allow that. Examples are code
// that runs under a fixed device-memory budget owned by a host framework, and
// latency-sensitive loops where the implicit device synchronisation of
// cudaFree would stall other streams. This variant keeps its partial sums in
// one statically sized device array instead.
//
// The array holds kScratchParts x 561 doubles (701 KB), and a second one the
// kScratchParts x 33 column exponents of the tensor-core kernel (21 KB).
// Every GPU that loads the library holds them until the process exits. They
// fit any Gram of up to 33 columns computed with at most kScratchParts CTAs.
// The kernels use one CTA per SM, capped by the number of row chunks, so that
// covers every GPU with up to 160 SMs (GB300 has 152).
#include <mutex>
#include <string>

#include "ascg_common.cuh"

namespace {

using namespace ascg;

constexpr int kScratchParts = 160;
constexpr size_t kScratchDoubles = (size_t)kScratchParts * kMaxPairs;

// The scratch itself. In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];
static __device__ __align__(256) int g_gram_exp_scratch[kScratchParts * kMaxW];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};
int* g_exp_addr[kMaxDevices] = {};

ascg_status fail(ascg_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

extern "C" ascg_status ascg_gram_noalloc(int64_t n, int w, const double* Y, int64_t ldY, double* G,
                                         void* cuda_stream) {
  set_last_error("");
  if (!Y || !G || n < 1 || ldY < n)
    return fail(ASCG_ERR_INVALID, "ascg_gram_noalloc: Y and G must be non-NULL, n >= 1 and ldY >= n");
  if (w < 1 || w > kMaxW)
    return fail(ASCG_ERR_INVALID,
                "ascg_gram_noalloc: w must be in 1..33 (the static scratch holds 33-column Grams at most)");
  const int parts =
      gram_tc_applies(w) && gram_tc_aligned(Y, ldY) && gram_tc_fits(n) ? gram_tc_parts(n) : gram_parts(n);
  if (parts > kScratchParts)
    return fail(ASCG_ERR_INVALID, "ascg_gram_noalloc: this GPU would use " + std::to_string(parts) +
                                      " CTAs, more than the 160 the static scratch holds");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(ASCG_ERR_CUDA, std::string("ascg_gram_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(ASCG_ERR_INVALID, "ascg_gram_noalloc: device " + std::to_string(dev) +
                                      " is beyond the 64 devices whose scratch addresses this library keeps");
  double* scratch = nullptr;
  int* exp_scratch = nullptr;
  {
    // One-time set-up per device, with that device current: look up the
    // device address of the static array. The first call on a device does
    // this, so make that first call before any stream capture.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_gram_scratch);
      if (e != cudaSuccess || !p)
        return fail(ASCG_ERR_CUDA,
                    std::string("ascg_gram_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      void* q = nullptr;
      e = cudaGetSymbolAddress(&q, g_gram_exp_scratch);
      if (e != cudaSuccess || !q)
        return fail(ASCG_ERR_CUDA,
                    std::string("ascg_gram_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = static_cast<double*>(p);
      g_exp_addr[dev] = static_cast<int*>(q);
    }
    scratch = g_addr[dev];
    exp_scratch = g_exp_addr[dev];
  }
  // Every CTA writes all of its partials before the finalize kernel reads
  // them, so nothing left in the array by an earlier call is ever read.
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int used = 0;
  e = launch_gram_any(n, w, Y, ldY, false, exp_scratch, false, scratch, &used, s);
  if (e == cudaSuccess) e = launch_gram_finalize(w, scratch, used, G, s);
  if (e != cudaSuccess)
    return fail(ASCG_ERR_CUDA, std::string("ascg_gram_noalloc: launch: ") + cudaGetErrorString(e));
  return ASCG_OK;
}
