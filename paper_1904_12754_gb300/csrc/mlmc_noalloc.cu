// mlmc_trace_noalloc: the walk recorder of mlmc_trace without any device
// allocation.  mlmc_trace obtains the scratch that the walk kernel needs
// (per-row sums, launch totals, the work counter, an FP32 copy of v) from
// cudaMalloc and returns it with cudaFree, which synchronises the whole device.
// Callers that must not do that -- a process whose device memory is reserved
// up front by another allocator, or one that cannot afford a device-wide
// synchronisation while other streams are busy -- use this entry point: its
// scratch is a fixed array in static device memory, sized for at most
// kNoAllocMaxRows rows.
#include <cuda.h>

#include <mutex>
#include <string>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

// Largest matrix order the static scratch serves.
constexpr int64_t kNoAllocMaxRows = int64_t{1} << 18;

// Scratch layout (bytes): work counter | launch totals | per-row sums | FP32 v.
constexpr size_t kOffWork = 0;
constexpr size_t kOffTotals = 256;
constexpr size_t kOffSums = 512;
constexpr size_t kOffV32 = kOffSums + sizeof(double) * kNoAllocMaxRows;
constexpr size_t kScratchBytes = kOffV32 + sizeof(float) * kNoAllocMaxRows;

// About 3 MB, held by every GPU that loads the library until the process
// exits.  Shared by all calls on a device: it keeps the previous call's
// contents, and calls whose GPU work overlaps (for example on two streams)
// race on it.
static __device__ __align__(256) unsigned char g_trace_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// Per device: the array's device address and the CUDA context it belongs
// to.  Only a successful lookup is kept, so a failed one is retried by the
// next call; a new context on the device (after cudaDeviceReset the module
// is loaded again, possibly elsewhere) triggers a new lookup.
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context (0 when none is current
// or the driver cannot say).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag resolved;
  std::call_once(resolved, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

mlmc_status noalloc_fail(mlmc_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_trace_noalloc(mlmc_plan* p, int32_t level, int32_t coarse,
                                          int64_t rep_begin, int64_t reps, const double* v,
                                          uint64_t seed, mlmc_walk_record* rec) {
  if (!p || !v || !rec) return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: NULL argument");
  if (level < 0 || level > 24 || (coarse && level < 1))
    return noalloc_fail(MLMC_ERR_INVALID_ARG,
                        "mlmc_trace_noalloc: level must be in [0,24] (>= 1 when coarse)");
  if (p->source_active && (level < 1 || (coarse && level < 2)))
    return noalloc_fail(MLMC_ERR_INVALID_ARG,
                        "mlmc_trace_noalloc: with a source term the level must be >= 1 (>= 2 when coarse)");
  if (rep_begin < 0 || reps < 0 || rep_begin > (int64_t{1} << 56) ||
      reps > (int64_t{1} << 56) - rep_begin)
    return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: replica range out of [0, 2^56)");
  if (p->sched.mode == MLMC_FORWARD)
    return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: backward-mode plans only");
  if (!pieces_fit(p, level, coarse != 0))
    return noalloc_fail(MLMC_ERR_INVALID_ARG,
                        "mlmc_trace_noalloc: the proposal's time pieces need 2^level (coarse: "
                        "2^(level-1)) to be a multiple of the piece count");
  if (p->n > kNoAllocMaxRows)
    return noalloc_fail(MLMC_ERR_INVALID_ARG,
                        "mlmc_trace_noalloc: n = " + std::to_string(p->n) +
                            " exceeds the static scratch limit of " +
                            std::to_string(kNoAllocMaxRows) + " rows; use mlmc_trace");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess)
    return noalloc_fail(MLMC_ERR_CUDA, std::string("mlmc_trace_noalloc: cudaGetDevice: ") +
                                           cudaGetErrorString(err));
  if (dev != p->device)
    return noalloc_fail(MLMC_ERR_INVALID_ARG,
                        "mlmc_trace_noalloc: the plan's device must be the current device");
  if (dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: device index out of range");
  // Once per device and context, with that device current: the device
  // address of the static array (in host code its name is only a host-side
  // stand-in).  The lookup also makes the device's context current on this
  // thread, so the context is identified after it.
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = current_context_id();
    if (ctx == 0 || g_scratch_ctx[dev] != ctx || !g_scratch_addr[dev]) {
      void* addr = nullptr;
      err = cudaGetSymbolAddress(&addr, g_trace_scratch);
      if (err != cudaSuccess || !addr) {
        g_scratch_addr[dev] = nullptr;
        g_scratch_ctx[dev] = 0;
        return noalloc_fail(MLMC_ERR_CUDA, std::string("mlmc_trace_noalloc: cudaGetSymbolAddress: ") +
                                               cudaGetErrorString(err));
      }
      g_scratch_addr[dev] = static_cast<unsigned char*>(addr);
      g_scratch_ctx[dev] = current_context_id();
    }
    base = g_scratch_addr[dev];
  }
  // The counter, totals and row sums must start at zero; the FP32 copy of v
  // is rewritten by the call.
  err = cudaMemsetAsync(base, 0, kOffSums + sizeof(double) * p->n, p->stream);
  if (err != cudaSuccess)
    return noalloc_fail(MLMC_ERR_CUDA, std::string("mlmc_trace_noalloc: memset: ") +
                                           cudaGetErrorString(err));
  WalkLaunch w;
  w.level = level;
  w.coarse = coarse != 0;
  w.rep_begin = rep_begin;
  w.reps = reps;
  w.seed = seed;
  w.v = v;
  w.sum_y = reinterpret_cast<double*>(base + kOffSums);
  w.totals = reinterpret_cast<double*>(base + kOffTotals);
  w.trace = rec;
  err = launch_walk_scratch(p, w, reinterpret_cast<unsigned long long*>(base + kOffWork),
                            reinterpret_cast<float*>(base + kOffV32));
  if (err != cudaSuccess)
    return noalloc_fail(MLMC_ERR_CUDA, std::string("mlmc_trace_noalloc: launch: ") +
                                           cudaGetErrorString(err));
  return MLMC_OK;
}
