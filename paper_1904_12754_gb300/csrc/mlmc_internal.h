// Internal declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include <cuda_runtime.h>

#include "../../include/mlmc.h"
#include "mlmc_device.cuh"

namespace mlmc {

// Error flags raised by kernels (bitwise OR into Plan::d_flags[0]).
enum : uint32_t {
  kFlagBadRowPtr = 1u << 0,
  kFlagBadCol = 1u << 1,
  kFlagUnsorted = 1u << 2,
  kFlagNonFinite = 1u << 3,
  kFlagWalkLimit = 1u << 4,
  kFlagNonFiniteY = 1u << 5,
  kFlagBounds = 1u << 6,      // checked build: a table index out of range
};

// Device accumulators of one level: sums of Y per row, and totals.
struct LevelAcc {
  double* sum_y = nullptr;  // [n]
  int64_t reps = 0;         // walks per row taken so far
  double seconds = 0.0;
  int64_t launches = 0;     // walk kernel launches
  bool pending = false;     // events recorded since the last read-out
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Totals slots of the per-level device scalars (doubles).
enum { kTotY2 = 0, kTotJumps = 1, kTotWalks = 2, kTotLimit = 3, kTotStill = 4, kTotSumSq = 5,
       kTotSum = 6, kTotSlots = 8 };

struct WalkLaunch {
  int64_t row_begin = 0;   // rows row_begin .. row_begin + row_count - 1
  int64_t row_count = -1;  // -1: every row
  int level = 0;
  bool coarse = false;
  int64_t rep_begin = 0;
  int64_t reps = 0;
  uint64_t seed = 0;
  const double* v = nullptr;
  double* sum_y = nullptr;
  double* totals = nullptr;         // kTotSlots doubles
  mlmc_walk_record* trace = nullptr;  // non-null selects the recording kernel
  // Intermediate times (backward walks): n_times > 1 also samples x(t k /
  // n_times), k < n_times, into sum_times [(n_times-1) x n] (and, with trace,
  // each record's samples into trace_times [(n_times-1) per record]).
  int n_times = 0;
  double* sum_times = nullptr;
  double* trace_times = nullptr;
};

}  // namespace mlmc

struct mlmc_plan {
  int64_t n = 0;
  int64_t nnz = 0;
  double t = 0.0;
  double rel_tol = 0.0;
  int32_t l0 = 0;
  mlmc_schedule sched{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int64_t launches = 0;

  // Resident CSR copy.
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;

  // Tables (Eq. 1 split, Eq. 12 alias), carved from one allocation in the
  // order: records of the plan's precision | its fused entries | plain alias
  // | records of the other precision | FP32 still thresholds, so that the
  // walk reads one contiguous range (its L2 access-policy window).
  unsigned char* d_tables = nullptr;
  mlmc::Meta32* d_meta32 = nullptr;
  mlmc::Meta64* d_meta64 = nullptr;
  int32_t* d_still32 = nullptr;   // FP32: per-row still threshold index (in d_tables)
  // Fused entries of the plan's precision (FusedEntry32 or FusedEntry64),
  // at the same positions as the alias entries.
  void* d_fused = nullptr;
  double* d_lii = nullptr;
  mlmc::AliasEntry* d_alias = nullptr;
  double dmax_scaled = 0.0;  // max_i max(|t d_i|, t L_ii)
  // Importance-sampling proposal (mlmc_plan_set_tilt): when active the
  // walks use d_alias_is and carry log(k/q) in their exponent; with tilted
  // clocks (clock_tilt) they also read the row records and FP32 still
  // thresholds of the rates lambda (d_meta32_t / d_meta64_t / d_still32_t),
  // and every jump carries log(L/lambda).  One allocation (d_is_block):
  // [proposal entries | Meta32 | Meta64 | still thresholds | lambda], each
  // part 256-byte aligned, so the walk's tables form one L2 window.
  unsigned char* d_is_block = nullptr;
  mlmc::AliasEntryIS* d_alias_is = nullptr;
  mlmc::Meta32* d_meta32_t = nullptr;
  mlmc::Meta64* d_meta64_t = nullptr;
  int32_t* d_still32_t = nullptr;
  double* d_lam = nullptr;
  bool clock_tilt = false;
  // Time pieces of the installed proposal (reading R19; 1: one law): every
  // part of d_is_block but the still thresholds and d_h hold `pieces`
  // consecutive copies, piece k's k n (entries: k nnz) after piece 0's.
  // is_pieces_cap: the pieces d_is_block and d_h have room for.
  int32_t pieces = 1;
  int32_t is_pieces_cap = 0;
  // Rows the table builds give a block each (stored length 32..8192): the
  // list (d_heavy), its device count and, once classified, its host count
  // (-1 before).
  int32_t* d_heavy = nullptr;
  uint32_t* d_heavy_count = nullptr;
  int64_t heavy_count = -1;
  int heavy_cap = 0;  // the longest listed row's length, rounded up to 4
  // The last mlmc_learn_tilt: the per-walk variance each pilot measured
  // (pilot k walked with the law installed before round k; the last one
  // with the final tilt) and which law was installed (-1: none).
  std::vector<double> learn_var;
  int32_t learn_choice = -1;
  // The learning's training rows (row i repeated 1 + deg_i / mean degree
  // times), kept across calls: they depend on the matrix alone.
  int64_t* d_train_rows = nullptr;
  int64_t n_train_rows = 0;
  // Forward mode (the tables above are then built from A^T): start weights,
  // their prefix sums and total, scan scratch.
  int64_t* d_wstart = nullptr;
  int64_t* d_cdf = nullptr;
  int32_t* d_guide = nullptr;  // [n] guide table of the start draw (cutpoints)
  int64_t* d_scan_tmp = nullptr;
  unsigned long long start_total = 0;
  float* d_h = nullptr;
  double alpha = 0.0;
  bool proposal_active = false;
  // Source term (mlmc_plan_set_source): when active every walk also carries
  // the Simpson sums of F along its path (Algorithm 3).
  double* d_src = nullptr;   // [n] F
  float* d_src32 = nullptr;  // [n] FP32 copy for the FP32 walk
  bool source_active = false;

  // L2 access-policy windows of the walk kernels (l2_persist): FP32 walks
  // read meta32 + alias, FP64 walks alias + meta64, proposal walks the
  // proposal tables.  Zero bytes: no window.
  size_t l2_persist_bytes = 0;     // persisting set-aside this plan asked for
  size_t l2_max_window = 0;        // device limit on one window
  const void* l2_base32 = nullptr;
  size_t l2_bytes32 = 0;
  const void* l2_base64 = nullptr;
  size_t l2_bytes64 = 0;

  // Work buffers.
  uint32_t* d_flags = nullptr;                 // [4]
  unsigned long long* d_work = nullptr;        // [1] dynamic work counter
  double* d_totals = nullptr;                  // [max_levels * kTotSlots]
  double* d_v = nullptr;                       // [n]
  float* d_v32 = nullptr;                      // [n] FP32 copy for the FP32 walk
  double* d_x = nullptr;                       // [n]
  double* d_norm2 = nullptr;                   // [4]
  double* d_sumpair = nullptr;                 // [2] sum, sum of squares
  double* d_red_part = nullptr;                // [red_partials(num_sms)] per-block partials
  std::vector<mlmc::LevelAcc> levels;          // per level slot (index l - l0)
  std::vector<mlmc_level_stats> last_stats;
  // Rows walked by the controller (ENTRY mode: one row); -1 = every row.
  int64_t ctl_row_begin = 0;
  int64_t ctl_row_count = -1;
  // The last controller call (mlmc_plan_save_state, mlmc_expmv_resume):
  // levels in use, seed and target (-1: no solve yet).
  int32_t ctl_nl = 0;
  uint64_t ctl_seed = 0;
  int32_t ctl_target = -1;
  double last_est_rel_err = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // Sharded solve (mlmc_plan_set_shard): this rank walks its part of every
  // level's new walk indices; before each controller decision the caller's
  // exchange sums the per-level row sums and totals over the ranks (in the
  // caller's buffer exch_buf), and d_glob receives the sums of all ranks:
  // [max_levels x n row sums | max_levels x kTotSlots totals].
  int32_t shard_rank = 0;
  int32_t shard_world = 1;
  mlmc_exchange_fn exch_fn = nullptr;
  void* exch_ctx = nullptr;
  double* exch_buf = nullptr;
  int64_t exch_cap = 0;
  double* d_glob = nullptr;
  bool shard_stop = false;  // the last exchange's vote: a rank is past its deadline

  // Intermediate times (mlmc_expmv_times): per level the row sums of the
  // samples at t k / T, k < T ([max_levels][T_max - 1][n], allocated on first
  // use for T_max = 16), and the T of the current solve (0: none).
  double* d_times = nullptr;
  double* d_xtimes = nullptr;   // [T_max - 1][n] the final sums of the times
  int32_t ctl_times = 0;
};

namespace mlmc {

// NVTX range for the timeline of a profiler (header-only NVTX 3; a no-op
// unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Thread-local error message.
void set_error(const std::string& msg);

// The L2 access-policy window for a walk launch over `base`..+`bytes`
// (count 0 when off); fills attr and returns the attribute count.
int l2_window_attr(const mlmc_plan* p, const void* base, size_t bytes, cudaLaunchAttribute* attr);

// Table kernels (mlmc_tables.cu).
cudaError_t launch_validate(mlmc_plan* p);
// Raise `func`'s dynamic shared memory limit to `bytes` once per device
// (the attribute belongs to the current device's context); `done` holds one
// bit per device already set.
template <typename F>
cudaError_t ensure_dynamic_smem(F* func, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t{1} << dev) : 0;
  if (bit && (done.load() & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit);
  return e;
}

// Doubles of per-block partials the controller's reductions need.
int64_t red_partials(int num_sms);
cudaError_t launch_build_tables(mlmc_plan* p);
cudaError_t launch_build_is_tables(mlmc_plan* p);

// A level's row sums and totals as the controller reads them: this rank's
// own (unsharded) or the exchanged sums of every rank.
inline bool sharded(const mlmc_plan* p) { return p->shard_world > 1; }
inline double* level_sums(const mlmc_plan* p, int slot) {
  return sharded(p) ? p->d_glob + static_cast<int64_t>(slot) * p->n : p->levels[slot].sum_y;
}
inline double* level_totals(const mlmc_plan* p, int slot) {
  return sharded(p) ? p->d_glob + static_cast<int64_t>(p->sched.max_levels) * p->n + slot * kTotSlots
                    : p->d_totals + slot * kTotSlots;
}
// Rank `rank` of `world` takes new walk indices [lo, hi) of `extra` (an
// even split, the first extra % world ranks one more).
inline void shard_range(int64_t extra, int32_t rank, int32_t world, int64_t* lo, int64_t* hi) {
  const int64_t q = extra / world, r = extra % world;
  *lo = rank * q + std::min<int64_t>(rank, r);
  *hi = *lo + q + (rank < r ? 1 : 0);
}

// The row records and FP32 still thresholds the walks of the plan read: the
// tilted ones when a proposal with tilted clocks is active.
inline const void* walk_meta(const mlmc_plan* p, bool fp64) {
  if (p->proposal_active && p->clock_tilt)
    return fp64 ? static_cast<const void*>(p->d_meta64_t) : static_cast<const void*>(p->d_meta32_t);
  return fp64 ? static_cast<const void*>(p->d_meta64) : static_cast<const void*>(p->d_meta32);
}
// Whether the installed proposal's time pieces fit the grids of a walk at
// `level` (coarse: and of level - 1): every piece boundary a grid point.
inline bool pieces_fit(const mlmc_plan* p, int level, bool coarse) {
  if (!p->proposal_active || p->pieces <= 1) return true;
  const int lv = coarse ? level - 1 : level;
  return lv >= 0 && lv <= 30 && (1 << lv) % p->pieces == 0;
}
inline const int32_t* walk_still32(const mlmc_plan* p) {
  return (p->proposal_active && p->clock_tilt) ? p->d_still32_t : p->d_still32;
}
// The L2 window of proposal walks: their alias entries and row records.
inline size_t is_window_bytes(const mlmc_plan* p, bool fp64) {
  const size_t k = static_cast<size_t>(p->is_pieces_cap > 0 ? p->is_pieces_cap : 1);
  const size_t ent = static_cast<size_t>(p->nnz > 0 ? p->nnz : 1) * k;
  size_t b = (sizeof(AliasEntryIS) * ent + 255) & ~size_t{255};
  if (p->clock_tilt) {
    b += (sizeof(Meta32) * static_cast<size_t>(p->n) * k + 255) & ~size_t{255};
    if (fp64) b += sizeof(Meta64) * static_cast<size_t>(p->n) * k;
  }
  return b;
}

// Walk kernels (mlmc_walk.cu).  Splits the replica range into launches of at
// most about 2^31 walks; returns the number of launches in *launches.
cudaError_t launch_walk(mlmc_plan* p, const WalkLaunch& w, int64_t* launches = nullptr);
// Forward-mode walks (mlmc_walk.cu) and their set-up (mlmc_forward.cu).
cudaError_t launch_walk_forward(mlmc_plan* p, const WalkLaunch& w, int64_t* launches = nullptr);
cudaError_t launch_transpose(mlmc_plan* p, const int64_t* rp, const int32_t* col, const double* val,
                             int64_t* rp_t, int32_t* col_t, double* val_t, int64_t* work);
cudaError_t launch_start_table(mlmc_plan* p, const double* v, int64_t* w, int64_t* cdf,
                               int64_t* tmp, unsigned long long* vmax_bits);
cudaError_t scan_int64(mlmc_plan* p, int64_t n, const int64_t* in, int64_t* out, int64_t* tmp);
// guide[b] = the smallest s with cdf[s] > floor(b W / n), b < n (W = cdf[n-1]).
cudaError_t launch_start_guide(mlmc_plan* p, const int64_t* cdf, unsigned long long W, int32_t* guide);
// As launch_walk, with the work counter and the FP32 copy of v in the given
// device memory instead of the plan's buffers.
cudaError_t launch_walk_scratch(mlmc_plan* p, const WalkLaunch& w, unsigned long long* work,
                                float* v32, int64_t* launches = nullptr);


// Batched rounds (mlmc_batch.cu): one persistent walk launch over every
// (problem, level, replica range) segment of a round.  A segment's items are
// the global work items [item_begin, item_begin + n * chunks_per_row); the
// kernel reads the round's header and segments from device memory, so one
// captured graph serves every round.
struct BatchSeg {
  const void* meta;           // row records of the problem's plan (its walk precision)
  const void* alias;          // fused entries, or proposal entries when is != 0
  const void* v_walk;         // right-hand side in the walk precision
  const int32_t* still32;     // FP32: per-row still threshold index
  double* sum_y;              // per-row sums of the (problem, level)
  double* totals;             // kTotSlots totals of the (problem, level)
  int64_t n, nnz;
  int64_t rep_begin, reps;    // replica range of every row
  int64_t chunk;              // walks per item (32 x walks per lane)
  int64_t chunks_per_row;
  unsigned long long item_begin;
  int64_t max_jumps;
  int32_t level, coarse, is, pad;
  uint32_t ctr3, pad2;
  PhiloxRoundKeys rk;         // the problem's seed
};
struct BatchRound {
  unsigned long long total_items;
  int32_t nseg;
  int32_t pad;
};
// Launch the persistent walk kernel of a round on `stream` (grid: every SM
// at its occupancy for `block` threads); the header and segments are read
// from device memory.
cudaError_t launch_walk_batch(bool fp64, const BatchRound* round, const BatchSeg* segs,
                              unsigned long long* work, uint32_t* flags, int num_sms, int block,
                              cudaStream_t stream);

// Reductions (mlmc_reduce.cu).
// out[0] += sum_i a_i, out[1] += sum_i a_i^2 (out must be zeroed by the caller).
cudaError_t launch_sum_sumsq(mlmc_plan* p, const double* a, double* out);
cudaError_t launch_finalize(mlmc_plan* p, int num_levels, double* x, double* norm2);
// x_times[(k-1) n + i] = sum_l S_l,k[i] / M_l for k = 1..n_times-1.
cudaError_t launch_finalize_times(mlmc_plan* p, int num_levels, int n_times, double* x_times);
constexpr int kMaxTimesAll = 16;
// Time pieces of a proposal (reading R19): at most this many.
constexpr int kMaxPieces = 16;

}  // namespace mlmc
