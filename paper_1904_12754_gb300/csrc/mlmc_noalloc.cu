// mlmc_trace_noalloc: the walk recorder of mlmc_trace without any device
// allocation.  mlmc_trace obtains the scratch that the walk kernel needs
// (per-row sums, launch totals, the work counter, an FP32 copy of v) from
// cudaMalloc and returns it with cudaFree, which synchronises the whole device.
// Callers that must not do that -- a process whose device memory is reserved
// up front by another allocator, or one that cannot afford a device-wide
// synchronisation while other streams are busy -- use this entry point: its
// scratch is a fixed array in static device memory, sized for at most
// kNoAllocMaxRows rows.
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
std::once_flag g_setup_once[kMaxDevices];
unsigned char* g_scratch_addr[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];

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
  if (rep_begin < 0 || reps < 0 || rep_begin + reps > (int64_t{1} << 56))
    return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: replica range out of [0, 2^56)");
  if (p->sched.mode == MLMC_FORWARD)
    return noalloc_fail(MLMC_ERR_INVALID_ARG, "mlmc_trace_noalloc: backward-mode plans only");
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
  // Once per device, with that device current: the device address of the
  // static array (in host code its name is only a host-side stand-in).
  std::call_once(g_setup_once[dev], [dev] {
    void* addr = nullptr;
    g_setup_err[dev] = cudaGetSymbolAddress(&addr, g_trace_scratch);
    g_scratch_addr[dev] = static_cast<unsigned char*>(addr);
  });
  if (g_setup_err[dev] != cudaSuccess || !g_scratch_addr[dev])
    return noalloc_fail(MLMC_ERR_CUDA, std::string("mlmc_trace_noalloc: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(g_setup_err[dev]));
  unsigned char* base = g_scratch_addr[dev];
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
