// C ABI of libmlmc and the MLMC controller (Algorithm 1).
//
// The controller keeps, per level l (slot l - l0), the device vector S_l of
// per-row sums of Y and four totals (sum Y^2, jumps, walks, limit hits).
// After each round of launches it reduces sum_i S_l,i^2 on the device and
// reads back a handful of scalars per level:
//   V_l   = (sum Y^2 - sum_i S_l,i^2 / M_l) / (M_l - 1)    total variance of
//           one sample (one walk from every row), unbiased;
//   C_l   = n (1 + jumps / walks)                          events per sample;
//   m_l   = S_l / M_l,  ||m_l||^2 = sum_i S_l,i^2 / M_l^2.
// With eps = rel_tol ||x|| it sets M_l = ceil(2/eps^2 sqrt(V_l/C_l)
// sum_k sqrt(V_k C_k)) (Giles' optimum; the paper's Eq. 11 prints it without
// the root and the factor 2), tops levels up, and stops when
// sum_l V_l/M_l <= eps^2/2 and max(||m_L||, ||m_{L-1}||/4)/3 <= eps/sqrt(2)
// (weak order 2, Eq. 13); otherwise it appends level L+1 (Algorithm 1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "mlmc_internal.h"

namespace mlmc {

namespace {
thread_local std::string g_last_error;

mlmc_status fail(mlmc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

mlmc_status cuda_fail(cudaError_t err, const char* what) {
  return fail(err == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(err));
}

#define MLMC_CUDA(call, what)                   \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// The device FP64 neglog uses literal coefficients; they must be the
// correctly rounded 1/(2k+1), which is what IEEE division on the host
// produces.  (The FP32 polynomial's coefficients are themselves the
// definition.)
bool coefficients_ok() {
  for (int k = 0; k < kNeglogTerms64; ++k) {
    volatile double d = static_cast<double>(2 * k + 1);
    if (neglog_c64(k) != 1.0 / d) return false;
  }
  return true;
}

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

void free_plan(mlmc_plan* p) {
  if (!p) return;
  cudaFree(p->d_row_ptr);
  cudaFree(p->d_col);
  cudaFree(p->d_val);
  cudaFree(p->d_tables);
  cudaFree(p->d_lii);
  cudaFree(p->d_heavy);
  cudaFree(p->d_train_rows);
  cudaFree(p->d_is_block);
  cudaFree(p->d_glob);
  cudaFree(p->d_times);
  cudaFree(p->d_xtimes);
  cudaFree(p->d_h);
  cudaFree(p->d_src);
  cudaFree(p->d_src32);
  cudaFree(p->d_flags);
  cudaFree(p->d_work);
  cudaFree(p->d_totals);
  cudaFree(p->d_v);
  cudaFree(p->d_v32);
  cudaFree(p->d_x);
  cudaFree(p->d_norm2);
  cudaFree(p->d_sumpair);
  cudaFree(p->d_red_part);
  cudaFree(p->d_wstart);
  cudaFree(p->d_cdf);
  cudaFree(p->d_guide);
  cudaFree(p->d_scan_tmp);
  if (!p->levels.empty()) cudaFree(p->levels[0].sum_y);
  for (auto& L : p->levels) {
    if (L.ev0) cudaEventDestroy(L.ev0);
    if (L.ev1) cudaEventDestroy(L.ev1);
  }
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

mlmc_status read_flags(mlmc_plan* p, uint32_t* out) {
  MLMC_CUDA(cudaMemcpyAsync(out, p->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, p->stream),
            "read flags");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  return MLMC_OK;
}

std::string flag_text(uint32_t f) {
  std::string s;
  if (f & kFlagBadRowPtr) s += " row_ptr not monotone / not ending at nnz;";
  if (f & kFlagBadCol) s += " column index out of range;";
  if (f & kFlagUnsorted) s += " columns not strictly increasing within a row;";
  if (f & kFlagNonFinite) s += " non-finite matrix value;";
  if (f & kFlagWalkLimit) s += " a walk exceeded max_jumps_per_walk;";
  if (f & kFlagNonFiniteY) s += " non-finite walk weight;";
  if (f & kFlagBounds) s += " table index out of range (checked build);";
  return s;
}

struct HostLevel {
  double y2, jumps, walks, limit, still, sumsq, sum;
};

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

static bool forward_mode(const mlmc_plan* p) { return p->sched.mode == MLMC_FORWARD; }

// Forward mode: start weights and prefix sums for v (device), W read back.
static mlmc_status prepare_starts(mlmc_plan* p, const double* v) {
  MLMC_CUDA(launch_start_table(p, v, p->d_wstart, p->d_cdf, p->d_scan_tmp,
                               reinterpret_cast<unsigned long long*>(p->d_norm2 + 2)),
            "start table");
  int64_t W = 0;
  MLMC_CUDA(cudaMemcpyAsync(&W, p->d_cdf + (p->n - 1), sizeof(int64_t), cudaMemcpyDeviceToHost,
                            p->stream), "read W");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  p->start_total = static_cast<unsigned long long>(W);
  if (W <= 0) return MLMC_OK;  // v = 0: no walks (launch_walk_forward makes none), x = 0
  MLMC_CUDA(launch_start_guide(p, p->d_cdf, p->start_total, p->d_guide), "start guide");
  return MLMC_OK;
}

static cudaError_t launch_any(mlmc_plan* p, const WalkLaunch& w, int64_t* nl) {
  return forward_mode(p) ? launch_walk_forward(p, w, nl) : launch_walk(p, w, nl);
}

// Per-level device scalars live at d_totals[slot * kTotSlots].
static double* totals_of(mlmc_plan* p, int slot) { return p->d_totals + slot * kTotSlots; }

// Launch `extra` more walks per row at level slot `slot`.  The walks are
// issued in batches of at most kBatchWalks, with a synchronisation after
// each, so that a large top-up stops at the wall-clock deadline; *stopped is
// set when it did.
// A sharded plan walks only its shard_range of the `extra` new indices (and
// is never cut short here: the ranks stop together at an exchange).
static mlmc_status run_level(mlmc_plan* p, int slot, int64_t extra, uint64_t seed,
                             std::vector<char>& timed,
                             std::chrono::steady_clock::time_point deadline, bool* stopped) {
  constexpr int64_t kBatchWalks = int64_t{1} << 36;  // ~0.5-1 s of FP32 walks
  LevelAcc& L = p->levels[slot];
  const int64_t rows = forward_mode(p) ? 1 : (p->ctl_row_count < 0 ? p->n : p->ctl_row_count);
  const int64_t batch_reps = std::max<int64_t>(32, kBatchWalks / rows);
  if (stopped) *stopped = false;
  int64_t my_lo = 0, my_hi = extra;
  if (sharded(p)) shard_range(extra, p->shard_rank, p->shard_world, &my_lo, &my_hi);
  const int64_t base = L.reps;
  if (sharded(p)) L.reps = base + extra;  // the level's global count
  for (int64_t done = my_lo; done < my_hi;) {
    const int64_t reps = std::min(batch_reps, my_hi - done);
    WalkLaunch w;
    w.row_begin = p->ctl_row_begin;
    w.row_count = p->ctl_row_count;
    w.level = p->l0 + slot;
    w.coarse = slot > 0;
    w.rep_begin = base + done;
    w.reps = reps;
    w.seed = seed;
    w.v = p->d_v;
    w.sum_y = L.sum_y;
    w.totals = totals_of(p, slot);
    if (p->ctl_times > 1) {
      w.n_times = p->ctl_times;
      w.sum_times = p->d_times + static_cast<int64_t>(slot) * (kMaxTimesAll - 1) * p->n;
    }
    int64_t nl = 0;
    NvtxRange range("mlmc level walks");
    MLMC_CUDA(cudaEventRecord(L.ev0, p->stream), "event record");
    MLMC_CUDA(launch_any(p, w, &nl), "walk kernel launch");
    MLMC_CUDA(cudaEventRecord(L.ev1, p->stream), "event record");
    L.launches += nl;
    if (!sharded(p)) L.reps += reps;
    done += reps;
    timed[slot] = 1;
    if (done < my_hi && !sharded(p)) {
      // Mid top-up: read this batch's time now and check the deadline.
      MLMC_CUDA(cudaEventSynchronize(L.ev1), "event synchronize");
      float ms = 0.f;
      MLMC_CUDA(cudaEventElapsedTime(&ms, L.ev0, L.ev1), "event elapsed");
      L.seconds += 1e-3 * ms;
      if (std::chrono::steady_clock::now() > deadline) {
        if (stopped) *stopped = true;
        return MLMC_OK;
      }
    } else {
      L.pending = true;  // read by collect() after its synchronisation
    }
  }
  return MLMC_OK;
}

// Sharded plans: sum this rank's row sums and totals of levels 0..nl-1 over
// the ranks through the caller's exchange (in its buffer: nl x n sums |
// nl x kTotSlots totals | the deadline vote) into d_glob, and take the
// vote: some rank is past its deadline.
static mlmc_status exchange(mlmc_plan* p, int nl, bool past_deadline) {
  const int64_t n = p->n;
  const int64_t ns = static_cast<int64_t>(nl) * n;
  const int64_t nt = static_cast<int64_t>(nl) * kTotSlots;
  const int64_t count = ns + nt + 1;
  const double vote = past_deadline ? 1.0 : 0.0;
  double got_vote = 0.0;
  MLMC_CUDA(cudaMemcpyAsync(p->exch_buf, p->levels[0].sum_y, sizeof(double) * ns,
                            cudaMemcpyDefault, p->stream), "exchange: copy sums");
  MLMC_CUDA(cudaMemcpyAsync(p->exch_buf + ns, p->d_totals, sizeof(double) * nt, cudaMemcpyDefault,
                            p->stream), "exchange: copy totals");
  MLMC_CUDA(cudaMemcpyAsync(p->exch_buf + ns + nt, &vote, sizeof(double), cudaMemcpyDefault,
                            p->stream), "exchange: copy vote");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "exchange: synchronize");
  {
    NvtxRange range("mlmc exchange");
    if (p->exch_fn(count, p->exch_ctx) != 0)
      return fail(MLMC_ERR_EXCHANGE, "the exchange callback of a sharded solve failed");
  }
  MLMC_CUDA(cudaMemcpyAsync(p->d_glob, p->exch_buf, sizeof(double) * ns, cudaMemcpyDefault,
                            p->stream), "exchange: read sums");
  MLMC_CUDA(cudaMemcpyAsync(p->d_glob + static_cast<int64_t>(p->sched.max_levels) * n,
                            p->exch_buf + ns, sizeof(double) * nt, cudaMemcpyDefault, p->stream),
            "exchange: read totals");
  MLMC_CUDA(cudaMemcpyAsync(&got_vote, p->exch_buf + ns + nt, sizeof(double), cudaMemcpyDefault,
                            p->stream), "exchange: read vote");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "exchange: synchronize");
  p->shard_stop = got_vote > 0.0;
  return MLMC_OK;
}

// Reduce sum_i S_i^2 per level and ||x||^2, and read the scalars back.
static mlmc_status collect(mlmc_plan* p, int nl, std::vector<HostLevel>& out, double* norm2,
                           bool past_deadline = false) {
  if (sharded(p)) {
    mlmc_status st = exchange(p, nl, past_deadline);
    if (st != MLMC_OK) return st;
  }
  for (int k = 0; k < nl; ++k) {
    MLMC_CUDA(cudaMemsetAsync(level_totals(p, k) + kTotSumSq, 0, 2 * sizeof(double), p->stream), "memset");
    MLMC_CUDA(launch_sum_sumsq(p, level_sums(p, k), p->d_sumpair), "sum");
    MLMC_CUDA(cudaMemcpyAsync(level_totals(p, k) + kTotSumSq, p->d_sumpair + 1, sizeof(double),
                              cudaMemcpyDeviceToDevice, p->stream), "copy");
    MLMC_CUDA(cudaMemcpyAsync(level_totals(p, k) + kTotSum, p->d_sumpair, sizeof(double),
                              cudaMemcpyDeviceToDevice, p->stream), "copy");
    MLMC_CUDA(cudaMemsetAsync(p->d_sumpair, 0, 2 * sizeof(double), p->stream), "memset");
  }
  MLMC_CUDA(launch_finalize(p, nl, nullptr, p->d_norm2), "finalize");
  std::vector<double> h(static_cast<size_t>(nl) * kTotSlots + 1);
  MLMC_CUDA(cudaMemcpyAsync(h.data(), level_totals(p, 0), sizeof(double) * nl * kTotSlots,
                            cudaMemcpyDeviceToHost, p->stream), "read totals");
  MLMC_CUDA(cudaMemcpyAsync(h.data() + nl * kTotSlots, p->d_norm2, sizeof(double),
                            cudaMemcpyDeviceToHost, p->stream), "read norm");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (int k = 0; k < nl; ++k) {
    LevelAcc& L = p->levels[k];
    if (!L.pending) continue;
    float ms = 0.f;
    MLMC_CUDA(cudaEventElapsedTime(&ms, L.ev0, L.ev1), "event elapsed");
    L.seconds += 1e-3 * ms;
    L.pending = false;
  }
  out.resize(nl);
  for (int k = 0; k < nl; ++k) {
    const double* t = h.data() + k * kTotSlots;
    out[k] = HostLevel{t[kTotY2], t[kTotJumps], t[kTotWalks], t[kTotLimit], t[kTotStill],
                       t[kTotSumSq], t[kTotSum]};
  }
  *norm2 = h[nl * kTotSlots];
  return MLMC_OK;
}

// The controller's three targets: the vector x (FULL, error in the 2-norm),
// one entry x_row (ENTRY: only that row walks), or the scalar 1^T x (SUM).
enum Target { kFull = 0, kEntry = 1, kSum = 2 };

// Unbiased V_l of one sample's contribution to the target.  Backward mode:
// rows are independent, so sum_i Var(Y_i) = (sum Y^2 - ||S||^2/M)/(M-1) for
// every target.  Forward mode: one walk adds y to a single entry, so the
// vector target uses the same expression while the scalar target 1^T x has
// Var(y) = (sum Y^2 - (sum_i S_i)^2/M)/(M-1).
static double level_var(const mlmc_plan* p, int k, const HostLevel& h, Target target) {
  const double m = static_cast<double>(p->levels[k].reps);
  if (m < 2) return 0.0;
  const double sq = (p->sched.mode == MLMC_FORWARD && target == kSum) ? h.sum * h.sum : h.sumsq;
  return std::max(0.0, (h.y2 - sq / m) / (m - 1.0));
}

static double level_cost(const mlmc_plan* p, const HostLevel& h) {
  const double per_walk = h.walks > 0 ? 1.0 + h.jumps / h.walks : 1.0;
  if (forward_mode(p)) return per_walk;  // one sample = one walk
  return static_cast<double>(p->ctl_row_count < 0 ? p->n : p->ctl_row_count) * per_walk;
}

}  // namespace mlmc

using namespace mlmc;

namespace mlmc {
int l2_window_attr(const mlmc_plan* p, const void* base, size_t bytes, cudaLaunchAttribute* attr) {
  if (p->l2_persist_bytes == 0 || p->l2_max_window == 0 || !base || bytes == 0) return 0;
  const size_t win = std::min(bytes, p->l2_max_window);
  attr->id = cudaLaunchAttributeAccessPolicyWindow;
  attr->val.accessPolicyWindow.base_ptr = const_cast<void*>(base);
  attr->val.accessPolicyWindow.num_bytes = win;
  attr->val.accessPolicyWindow.hitRatio =
      static_cast<float>(std::min(1.0, static_cast<double>(p->l2_persist_bytes) / static_cast<double>(win)));
  attr->val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  attr->val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  return 1;
}
}  // namespace mlmc

// Saved controller state: a header, per level (M_l, seconds, launches), then
// the level totals, the per-level row sums and v (doubles).
namespace {
constexpr uint64_t kStateMagic = 0x54415453434D4C4Dull;  // "MLMCSTAT"
struct StateHeader {
  uint64_t magic;
  uint32_t version;
  int32_t nl;
  int64_t n, nnz;
  double t;
  int32_t l0, precision, mode, target;
  int64_t row_begin, row_count;
  uint64_t seed;
  int32_t source, proposal;
};
struct StateLevel {
  int64_t reps;
  double seconds;
  int64_t launches;
};
size_t state_bytes(const mlmc_plan* p, int nl) {
  return sizeof(StateHeader) + sizeof(StateLevel) * nl +
         sizeof(double) * (static_cast<size_t>(nl) * kTotSlots + static_cast<size_t>(nl) * p->n + p->n);
}
}  // namespace

extern "C" {

mlmc_status mlmc_schedule_default(mlmc_schedule* s) {
  if (!s) return fail(MLMC_ERR_INVALID_ARG, "mlmc_schedule_default: NULL schedule");
  std::memset(s, 0, sizeof(*s));
  s->l0 = -1;
  s->num_levels = 5;
  s->max_levels = 12;
  s->precision = MLMC_FP64;
  s->mode = MLMC_BACKWARD;
  s->proposal = MLMC_PLAIN;
  s->pilot_walks = 64;
  s->max_jumps_per_walk = 1 << 20;
  s->max_walks_per_row = 1ll << 34;
  s->time_budget_s = 600.0;
  s->walks_per_lane = 0;
  s->block_threads = 0;
  s->l2_persist = 1;
  return MLMC_OK;
}

const char* mlmc_last_error(void) { return g_last_error.c_str(); }

mlmc_status mlmc_plan_create(mlmc_plan** out, int64_t n, int64_t nnz, const int64_t* row_ptr,
                             const int32_t* col, const double* vals, double t,
                             const mlmc_schedule* sched, double rel_tol, void* cuda_stream) {
  g_last_error.clear();
  if (!out) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_create: NULL out");
  *out = nullptr;
  if (!coefficients_ok()) return fail(MLMC_ERR_NUMERIC, "neglog coefficients are not 1/(2k+1)");
  if (n < 1 || n >= (1ll << 31)) return fail(MLMC_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  if (nnz < 0 || nnz >= (1ll << 31)) return fail(MLMC_ERR_INVALID_ARG, "nnz must be in [0, 2^31)");
  if (!row_ptr || (nnz > 0 && (!col || !vals)))
    return fail(MLMC_ERR_INVALID_ARG, "NULL CSR pointer");
  if (!(t >= 0.0) || !std::isfinite(t)) return fail(MLMC_ERR_INVALID_ARG, "t must be finite and >= 0");
  if (!(rel_tol > 0.0) || !std::isfinite(rel_tol))
    return fail(MLMC_ERR_INVALID_ARG, "rel_tol must be finite and > 0");
  mlmc_schedule s;
  if (sched) s = *sched; else mlmc_schedule_default(&s);
  if (s.num_levels < 1 || s.max_levels < s.num_levels || s.max_levels > 32)
    return fail(MLMC_ERR_INVALID_ARG, "need 1 <= num_levels <= max_levels <= 32");
  if (s.precision != MLMC_FP64 && s.precision != MLMC_FP32_KAHAN)
    return fail(MLMC_ERR_INVALID_ARG, "unknown precision");
  if (s.mode != MLMC_BACKWARD && s.mode != MLMC_FORWARD)
    return fail(MLMC_ERR_INVALID_ARG, "mode must be MLMC_BACKWARD or MLMC_FORWARD");
  if (s.proposal != MLMC_PLAIN)
    return fail(MLMC_ERR_INVALID_ARG,
                "create the plan with MLMC_PLAIN; a proposal is set by mlmc_plan_set_proposal");
  if (s.pilot_walks < 2 || s.max_jumps_per_walk < 0 || s.max_jumps_per_walk > 0xFFFFFFF0ll ||
      s.max_walks_per_row < s.pilot_walks || s.max_walks_per_row > (1ll << 55))
    return fail(MLMC_ERR_INVALID_ARG, "bad schedule budgets");
  if (s.l0 > 24 || (s.l0 >= 0 && s.l0 + s.max_levels - 1 > 24))
    return fail(MLMC_ERR_INVALID_ARG, "levels above 24 are not supported");
  if (s.l2_persist != 0 && s.l2_persist != 1)
    return fail(MLMC_ERR_INVALID_ARG, "l2_persist must be 0 or 1");
  if (s.walks_per_lane < 0 || s.block_threads < 0 || s.block_threads % 32 != 0 ||
      s.block_threads > 256)
    return fail(MLMC_ERR_INVALID_ARG, "block_threads must be a multiple of 32 up to 256");
  if (s.launch_reps < 0) return fail(MLMC_ERR_INVALID_ARG, "launch_reps must be >= 0");

  mlmc_plan* p = new mlmc_plan();
  p->n = n;
  p->nnz = nnz;
  p->t = t;
  p->rel_tol = rel_tol;
  p->sched = s;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](mlmc_status st) {
    free_plan(p);
    return st;
  };
#define PLAN_CUDA(call, what)                                  \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, what));   \
  } while (0)
  PLAN_CUDA(cudaGetDevice(&p->device), "cudaGetDevice");
  PLAN_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device),
            "device attribute");
  PLAN_CUDA(dev_alloc(&p->d_row_ptr, n + 1), "alloc row_ptr");
  PLAN_CUDA(dev_alloc(&p->d_col, nnz), "alloc col");
  PLAN_CUDA(dev_alloc(&p->d_val, nnz), "alloc val");
  {
    // [records of the plan's precision | its fused entries | plain alias |
    // records of the other precision | FP32 still thresholds], each part
    // 256-byte aligned: the walk reads the first two parts (one contiguous
    // L2 window) and one threshold per work item.
    auto up = [](size_t b) { return (b + 255) & ~size_t{255}; };
    const bool fp64 = s.precision == MLMC_FP64;
    const size_t ent = static_cast<size_t>(nnz > 0 ? nnz : 1);
    const size_t b32 = up(sizeof(Meta32) * static_cast<size_t>(n));
    const size_t b64 = up(sizeof(Meta64) * static_cast<size_t>(n));
    const size_t ba = up(sizeof(AliasEntry) * ent);
    const size_t bf = up((fp64 ? sizeof(FusedEntry64) : sizeof(FusedEntry32)) * ent);
    const size_t bown = fp64 ? b64 : b32, bother = fp64 ? b32 : b64;
    const size_t bstill = up(sizeof(int32_t) * static_cast<size_t>(n > 0 ? n : 1));
    PLAN_CUDA(dev_alloc(&p->d_tables, bown + bf + ba + bother + bstill), "alloc tables");
    unsigned char* own = p->d_tables;
    p->d_fused = p->d_tables + bown;
    p->d_alias = reinterpret_cast<AliasEntry*>(p->d_tables + bown + bf);
    unsigned char* other = p->d_tables + bown + bf + ba;
    p->d_meta32 = reinterpret_cast<Meta32*>(fp64 ? other : own);
    p->d_meta64 = reinterpret_cast<Meta64*>(fp64 ? own : other);
    p->d_still32 = reinterpret_cast<int32_t*>(other + bother);
    p->l2_base32 = p->d_tables;
    p->l2_bytes32 = bown + bf;
    p->l2_base64 = p->d_tables;
    p->l2_bytes64 = bown + bf;
    if (s.l2_persist) {
      int max_persist = 0, max_window = 0;
      if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, p->device) != cudaSuccess ||
          cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, p->device) != cudaSuccess) {
        max_persist = 0;
        max_window = 0;
        cudaGetLastError();
      }
      const size_t want = s.precision == MLMC_FP64 ? p->l2_bytes64 : p->l2_bytes32;
      const size_t aside = std::min<size_t>(want, static_cast<size_t>(max_persist));
      size_t cur = 0;
      if (aside > 0 && max_window > 0 && cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
        if (cur >= aside || cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, aside) == cudaSuccess) {
          p->l2_persist_bytes = aside;
          p->l2_max_window = static_cast<size_t>(max_window);
        }
      }
      cudaGetLastError();  // a refused set-aside only turns the window off
    }
  }
  PLAN_CUDA(dev_alloc(&p->d_lii, n), "alloc lii");
  PLAN_CUDA(dev_alloc(&p->d_flags, 4), "alloc flags");
  PLAN_CUDA(dev_alloc(&p->d_work, 1), "alloc work");
  PLAN_CUDA(dev_alloc(&p->d_totals, static_cast<size_t>(s.max_levels) * kTotSlots), "alloc totals");
  PLAN_CUDA(dev_alloc(&p->d_v, n), "alloc v");
  PLAN_CUDA(dev_alloc(&p->d_v32, n), "alloc v32");
  PLAN_CUDA(dev_alloc(&p->d_x, n), "alloc x");
  PLAN_CUDA(dev_alloc(&p->d_norm2, 4), "alloc scalars");
  PLAN_CUDA(dev_alloc(&p->d_sumpair, 2), "alloc scalars");
  PLAN_CUDA(dev_alloc(&p->d_red_part, static_cast<size_t>(red_partials(p->num_sms))), "alloc partials");
  PLAN_CUDA(cudaMemsetAsync(p->d_sumpair, 0, 2 * sizeof(double), p->stream), "memset");
  double* sums = nullptr;
  PLAN_CUDA(dev_alloc(&sums, static_cast<size_t>(n) * s.max_levels), "alloc level sums");
  p->levels.resize(s.max_levels);
  for (int k = 0; k < s.max_levels; ++k) {
    p->levels[k].sum_y = sums + static_cast<size_t>(k) * n;
    PLAN_CUDA(cudaEventCreate(&p->levels[k].ev0), "event create");
    PLAN_CUDA(cudaEventCreate(&p->levels[k].ev1), "event create");
  }
  PLAN_CUDA(cudaEventCreate(&p->ev0), "event create");
  PLAN_CUDA(cudaEventCreate(&p->ev1), "event create");

  PLAN_CUDA(cudaMemcpyAsync(p->d_row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault,
                            p->stream), "copy row_ptr");
  if (nnz > 0) {
    PLAN_CUDA(cudaMemcpyAsync(p->d_col, col, sizeof(int32_t) * nnz, cudaMemcpyDefault, p->stream),
              "copy col");
    PLAN_CUDA(cudaMemcpyAsync(p->d_val, vals, sizeof(double) * nnz, cudaMemcpyDefault, p->stream),
              "copy vals");
  }
  PLAN_CUDA(cudaMemsetAsync(p->d_flags, 0, sizeof(uint32_t) * 4, p->stream), "memset flags");
  PLAN_CUDA(launch_validate(p), "validate kernel");
  uint32_t flags = 0;
  {
    mlmc_status st = read_flags(p, &flags);
    if (st != MLMC_OK) return bail(st);
  }
  if (flags) return bail(fail(MLMC_ERR_INVALID_ARG, "invalid CSR:" + flag_text(flags)));
  if (s.mode == MLMC_FORWARD) {
    // Forward mode walks on B = A^T: transpose on the device and keep B as
    // the plan's matrix (tables, proposals and features are built from it).
    int64_t* rp_t = nullptr;
    int32_t* col_t = nullptr;
    double* val_t = nullptr;
    int64_t* work = nullptr;
    const int64_t scan_tmp = n / 256 + 64;
    PLAN_CUDA(dev_alloc(&rp_t, n + 1), "alloc transpose");
    PLAN_CUDA(dev_alloc(&col_t, nnz), "alloc transpose");
    PLAN_CUDA(dev_alloc(&val_t, nnz), "alloc transpose");
    PLAN_CUDA(dev_alloc(&work, 2 * n + scan_tmp), "alloc transpose");
    cudaError_t terr = launch_transpose(p, p->d_row_ptr, p->d_col, p->d_val, rp_t, col_t, val_t, work);
    if (terr == cudaSuccess) terr = cudaStreamSynchronize(p->stream);
    cudaFree(work);
    cudaFree(p->d_row_ptr);
    cudaFree(p->d_col);
    cudaFree(p->d_val);
    p->d_row_ptr = rp_t;
    p->d_col = col_t;
    p->d_val = val_t;
    if (terr != cudaSuccess) return bail(cuda_fail(terr, "transpose"));
    PLAN_CUDA(dev_alloc(&p->d_wstart, n), "alloc start weights");
    PLAN_CUDA(dev_alloc(&p->d_cdf, n), "alloc start cdf");
    PLAN_CUDA(dev_alloc(&p->d_guide, n), "alloc start guide");
    PLAN_CUDA(dev_alloc(&p->d_scan_tmp, scan_tmp), "alloc scan scratch");
  }
  mlmc_status st = mlmc_plan_rebuild(p);
  if (st != MLMC_OK) return bail(st);
  unsigned long long bits = 0;
  PLAN_CUDA(cudaMemcpyAsync(&bits, p->d_norm2, sizeof(bits), cudaMemcpyDeviceToHost, p->stream),
            "read dmax");
  PLAN_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  std::memcpy(&p->dmax_scaled, &bits, sizeof(bits));
  if (s.l0 >= 0) {
    p->l0 = s.l0;
  } else {
    // Eq. 16, l0 = log2(2 t d_max), with d_max = max_i max(|d_i|, L_ii),
    // rounded up (values within 1e-9 of an integer count as that integer).
    const double x = 2.0 * p->dmax_scaled;
    p->l0 = x > 0.0 ? std::max(0, static_cast<int>(std::ceil(std::log2(x) - 1e-9))) : 0;
  }
  if (p->l0 + s.max_levels - 1 > 24) {
    p->sched.max_levels = std::max(s.num_levels, 25 - p->l0);
    if (p->l0 + p->sched.max_levels - 1 > 24)
      return bail(fail(MLMC_ERR_INVALID_ARG, "l0 from Eq. 16 leaves no room for the levels"));
  }
#undef PLAN_CUDA
  *out = p;
  return MLMC_OK;
}

mlmc_status mlmc_plan_rebuild(mlmc_plan* p) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  MLMC_CUDA(launch_build_tables(p), "table build");
  if (p->proposal_active) MLMC_CUDA(launch_build_is_tables(p), "proposal table build");
  return MLMC_OK;
}


mlmc_status mlmc_plan_l2_window(const mlmc_plan* p, int64_t* bytes, double* hit_ratio) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  cudaLaunchAttribute attr;
  const bool fp64 = p->sched.precision == MLMC_FP64;
  const int na = l2_window_attr(p, fp64 ? p->l2_base64 : p->l2_base32,
                                fp64 ? p->l2_bytes64 : p->l2_bytes32, &attr);
  if (bytes) *bytes = na ? static_cast<int64_t>(attr.val.accessPolicyWindow.num_bytes) : 0;
  if (hit_ratio) *hit_ratio = na ? attr.val.accessPolicyWindow.hitRatio : 0.0;
  return MLMC_OK;
}

mlmc_status mlmc_plan_set_source(mlmc_plan* p, const double* f) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (!f) {
    p->source_active = false;
    return MLMC_OK;
  }
  if (forward_mode(p)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_source: backward-mode plans only");
  if (p->proposal_active)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_source: remove the proposal first");
  if (p->l0 < 1)
    return fail(MLMC_ERR_INVALID_ARG,
                "mlmc_plan_set_source: Simpson's rule needs an even number of steps on every "
                "level; create the plan with l0 >= 1");
  if (!p->d_src) {
    MLMC_CUDA(dev_alloc(&p->d_src, static_cast<size_t>(p->n)), "alloc source");
    MLMC_CUDA(dev_alloc(&p->d_src32, static_cast<size_t>(p->n)), "alloc source");
  }
  MLMC_CUDA(cudaMemcpyAsync(p->d_src, f, sizeof(double) * p->n, cudaMemcpyDefault, p->stream),
            "copy source");
  std::vector<double> hf(p->n);
  MLMC_CUDA(cudaMemcpyAsync(hf.data(), p->d_src, sizeof(double) * p->n, cudaMemcpyDeviceToHost,
                            p->stream), "read source");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (double x : hf)
    if (!std::isfinite(x)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_source: f must be finite");
  p->source_active = true;
  return MLMC_OK;
}

mlmc_status mlmc_plan_set_proposal(mlmc_plan* p, const float* h, double alpha) {
  return mlmc_plan_set_tilt(p, h, alpha, MLMC_TILT_JUMPS);
}

namespace {

// mlmc_plan_set_tilt and mlmc_plan_set_tilt_pieces: `pieces` laws, h holding
// pieces x n values (piece k's h at k n).
mlmc_status set_tilt_impl(mlmc_plan* p, const float* h, double alpha, int32_t tilt, int32_t pieces,
                          const char* who) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (!h) {
    p->proposal_active = false;
    p->clock_tilt = false;
    p->pieces = 1;
    p->sched.proposal = MLMC_PLAIN;
    return MLMC_OK;
  }
  if (tilt != MLMC_TILT_JUMPS && tilt != (MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS))
    return fail(MLMC_ERR_INVALID_ARG,
                std::string(who) + ": tilt must be MLMC_TILT_JUMPS or MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS");
  if (p->source_active)
    return fail(MLMC_ERR_INVALID_ARG, std::string(who) + ": the plan has a source term");
  if (!(alpha > 0.0) || !(alpha <= 1.0))
    return fail(MLMC_ERR_INVALID_ARG, "alpha must be in (0, 1]: the proposal mixes in the plain law");
  if (pieces > 1) {
    if (forward_mode(p))
      return fail(MLMC_ERR_INVALID_ARG, std::string(who) + ": time pieces need a backward-mode plan");
    if (pieces > kMaxPieces || (pieces & (pieces - 1)) != 0)
      return fail(MLMC_ERR_INVALID_ARG, std::string(who) + ": pieces must be a power of two <= " +
                                            std::to_string(kMaxPieces));
    if (pieces > (1 << p->l0))
      return fail(MLMC_ERR_INVALID_ARG,
                  std::string(who) + ": every piece boundary must lie on the grid of every level "
                  "walked, so pieces <= 2^l0 (l0 = " + std::to_string(p->l0) + ")");
  }
  const size_t k = static_cast<size_t>(pieces);
  const size_t nh = static_cast<size_t>(p->n) * k;
  // h must be positive and finite on every row (checked on a host copy,
  // taken before anything of the plan changes: h may be the plan's own).
  std::vector<float> hh(nh);
  MLMC_CUDA(cudaMemcpyAsync(hh.data(), h, sizeof(float) * nh, cudaMemcpyDefault, p->stream), "read h");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (size_t i = 0; i < nh; ++i)
    if (!(hh[i] > 0.0f) || !std::isfinite(hh[i]))
      return fail(MLMC_ERR_INVALID_ARG, "h must be positive and finite (row " +
                                            std::to_string(i % static_cast<size_t>(p->n)) +
                                            (pieces > 1 ? ", piece " + std::to_string(i / p->n) : "") + ")");
  if (p->is_pieces_cap < pieces) {
    // [proposal entries | Meta32 | Meta64 | still thresholds | lambda], the
    // entries, records and rates once per piece
    cudaFree(p->d_is_block);
    cudaFree(p->d_h);
    p->d_is_block = nullptr;
    p->d_h = nullptr;
    p->is_pieces_cap = 0;
    p->proposal_active = false;
    p->sched.proposal = MLMC_PLAIN;
    auto up = [](size_t b) { return (b + 255) & ~size_t{255}; };
    const size_t n = static_cast<size_t>(p->n);
    const size_t be = up(sizeof(AliasEntryIS) * static_cast<size_t>(p->nnz > 0 ? p->nnz : 1) * k);
    const size_t b32 = up(sizeof(Meta32) * n * k), b64 = up(sizeof(Meta64) * n * k);
    const size_t bs = up(sizeof(int32_t) * n), bl = up(sizeof(double) * n * k);
    MLMC_CUDA(dev_alloc(&p->d_is_block, be + b32 + b64 + bs + bl), "alloc proposal tables");
    MLMC_CUDA(dev_alloc(&p->d_h, n * k), "alloc h");
    p->d_alias_is = reinterpret_cast<AliasEntryIS*>(p->d_is_block);
    p->d_meta32_t = reinterpret_cast<Meta32*>(p->d_is_block + be);
    p->d_meta64_t = reinterpret_cast<Meta64*>(p->d_is_block + be + b32);
    p->d_still32_t = reinterpret_cast<int32_t*>(p->d_is_block + be + b32 + b64);
    p->d_lam = reinterpret_cast<double*>(p->d_is_block + be + b32 + b64 + bs);
    p->is_pieces_cap = pieces;
  }
  MLMC_CUDA(cudaMemcpyAsync(p->d_h, hh.data(), sizeof(float) * nh, cudaMemcpyHostToDevice, p->stream),
            "copy h");
  p->alpha = alpha;
  p->clock_tilt = (tilt & MLMC_TILT_CLOCKS) != 0;
  p->pieces = pieces;
  MLMC_CUDA(launch_build_is_tables(p), "proposal table build");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");  // hh is read by the copy above
  p->proposal_active = true;
  p->sched.proposal = MLMC_LEARNED;
  return MLMC_OK;
}

}  // namespace

mlmc_status mlmc_plan_set_tilt(mlmc_plan* p, const float* h, double alpha, int32_t tilt) {
  return set_tilt_impl(p, h, alpha, tilt, 1, "mlmc_plan_set_tilt");
}

mlmc_status mlmc_plan_set_tilt_pieces(mlmc_plan* p, const float* h, int32_t pieces, double alpha) {
  if (pieces < 1) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_tilt_pieces: pieces must be >= 1");
  return set_tilt_impl(p, h, alpha, MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS, pieces,
                       "mlmc_plan_set_tilt_pieces");
}

mlmc_status mlmc_export_tilt_piece(const mlmc_plan* pc, int32_t piece, double* lam, double* dl,
                                   double* inv_rate, float* inv_rate32, float* dl32, int32_t* still32) {
  mlmc_plan* p = const_cast<mlmc_plan*>(pc);
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (!p->proposal_active || !p->clock_tilt)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_export_tilt: no proposal with tilted clocks on this plan");
  if (piece < 0 || piece >= p->pieces)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_export_tilt_piece: piece out of range");
  const size_t n = static_cast<size_t>(p->n);
  const size_t k = static_cast<size_t>(p->pieces);
  const size_t off = static_cast<size_t>(piece) * n;
  // the records are state-major (row i's record of piece q at i K + q)
  std::vector<Meta32> m32(n * k);
  std::vector<Meta64> m64(n * k);
  std::vector<double> lm(n);
  std::vector<int32_t> st(n);
  MLMC_CUDA(cudaMemcpyAsync(m32.data(), p->d_meta32_t, sizeof(Meta32) * n * k, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaMemcpyAsync(m64.data(), p->d_meta64_t, sizeof(Meta64) * n * k, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaMemcpyAsync(lm.data(), p->d_lam + off, sizeof(double) * n, cudaMemcpyDeviceToHost, p->stream), "copy");
  if (p->sched.precision != MLMC_FP64)
    MLMC_CUDA(cudaMemcpyAsync(st.data(), p->d_still32_t, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (size_t i = 0; i < n; ++i) {
    const size_t r = i * k + static_cast<size_t>(piece);
    if (lam) lam[i] = lm[i];
    if (dl) dl[i] = m64[r].dl;
    if (inv_rate) inv_rate[i] = m64[r].inv_rate;
    if (inv_rate32) inv_rate32[i] = m32[r].inv_rate;
    if (dl32) dl32[i] = m32[r].dl;
    if (still32) still32[i] = p->sched.precision != MLMC_FP64 ? st[i] : -1;
  }
  return MLMC_OK;
}

mlmc_status mlmc_export_tilt(const mlmc_plan* pc, double* lam, double* dl, double* inv_rate,
                             float* inv_rate32, float* dl32, int32_t* still32) {
  return mlmc_export_tilt_piece(pc, 0, lam, dl, inv_rate, inv_rate32, dl32, still32);
}

mlmc_status mlmc_export_proposal_piece(const mlmc_plan* pc, int32_t piece, uint32_t* thr,
                                       int32_t* keep_col, uint8_t* keep_neg, int32_t* alias_col,
                                       uint8_t* alias_neg, float* lr_keep, float* lr_alias) {
  mlmc_plan* p = const_cast<mlmc_plan*>(pc);
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (!p->proposal_active) return fail(MLMC_ERR_INVALID_ARG, "no proposal set on this plan");
  if (piece < 0 || piece >= p->pieces)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_export_proposal_piece: piece out of range");
  std::vector<Meta32> m32(p->n);
  std::vector<AliasEntryIS> al(p->nnz > 0 ? p->nnz : 1);
  MLMC_CUDA(cudaMemcpyAsync(m32.data(), p->d_meta32, sizeof(Meta32) * p->n, cudaMemcpyDeviceToHost, p->stream), "copy");
  if (p->nnz > 0)
    MLMC_CUDA(cudaMemcpyAsync(al.data(), p->d_alias_is + static_cast<int64_t>(piece) * p->nnz,
                              sizeof(AliasEntryIS) * p->nnz, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (int64_t i = 0; i < p->n; ++i)
    for (int32_t b = 0; b < m32[i].deg; ++b) {
      const int64_t q = m32[i].start + b;
      const AliasEntryIS& e = al[q];
      if (thr) thr[q] = e.thr;
      if (keep_col) keep_col[q] = static_cast<int32_t>(e.keep & kColMask);
      if (keep_neg) keep_neg[q] = static_cast<uint8_t>(e.keep >> 31);
      if (alias_col) alias_col[q] = static_cast<int32_t>(e.alias & kColMask);
      if (alias_neg) alias_neg[q] = static_cast<uint8_t>(e.alias >> 31);
      if (lr_keep) lr_keep[q] = e.lr_keep;
      if (lr_alias) lr_alias[q] = e.lr_alias;
    }
  return MLMC_OK;
}

mlmc_status mlmc_export_proposal(const mlmc_plan* pc, uint32_t* thr, int32_t* keep_col,
                                 uint8_t* keep_neg, int32_t* alias_col, uint8_t* alias_neg,
                                 float* lr_keep, float* lr_alias) {
  return mlmc_export_proposal_piece(pc, 0, thr, keep_col, keep_neg, alias_col, alias_neg, lr_keep,
                                    lr_alias);
}

int32_t mlmc_plan_tilt_pieces(const mlmc_plan* p) {
  if (!p || !p->proposal_active) return 0;
  return p->pieces;
}

mlmc_status mlmc_export_h(const mlmc_plan* pc, float* h) {
  mlmc_plan* p = const_cast<mlmc_plan*>(pc);
  if (!p || !h) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (!p->proposal_active) return fail(MLMC_ERR_INVALID_ARG, "mlmc_export_h: no proposal set on this plan");
  MLMC_CUDA(cudaMemcpyAsync(h, p->d_h, sizeof(float) * p->n * static_cast<size_t>(p->pieces),
                            cudaMemcpyDefault, p->stream), "copy h");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  return MLMC_OK;
}

int64_t mlmc_shard_buffer_doubles(const mlmc_plan* p) {
  if (!p) return -1;
  return static_cast<int64_t>(p->sched.max_levels) * (p->n + kTotSlots) + 1;
}

mlmc_status mlmc_shard_range(int64_t extra, int32_t rank, int32_t world, int64_t* lo, int64_t* hi) {
  if (!lo || !hi) return fail(MLMC_ERR_INVALID_ARG, "mlmc_shard_range: NULL argument");
  if (extra < 0 || world < 1 || world > 65536 || rank < 0 || rank >= world)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_shard_range: need extra >= 0 and 0 <= rank < world <= 65536");
  shard_range(extra, rank, world, lo, hi);
  return MLMC_OK;
}

mlmc_status mlmc_plan_set_shard(mlmc_plan* p, int32_t rank, int32_t world, mlmc_exchange_fn exchange,
                                void* ctx, double* buf, int64_t cap) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (world == 1 || !exchange) {
    p->shard_rank = 0;
    p->shard_world = 1;
    p->exch_fn = nullptr;
    p->exch_ctx = nullptr;
    p->exch_buf = nullptr;
    p->exch_cap = 0;
    return MLMC_OK;
  }
  if (world < 1 || world > 65536 || rank < 0 || rank >= world)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_shard: need 0 <= rank < world <= 65536");
  if (!buf || cap < mlmc_shard_buffer_doubles(p))
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_set_shard: the exchange buffer needs " +
                                          std::to_string(mlmc_shard_buffer_doubles(p)) + " doubles");
  if (!p->d_glob)
    MLMC_CUDA(dev_alloc(&p->d_glob, static_cast<size_t>(p->sched.max_levels) *
                                        static_cast<size_t>(p->n + kTotSlots)),
              "alloc sharded sums");
  p->shard_rank = rank;
  p->shard_world = world;
  p->exch_fn = exchange;
  p->exch_ctx = ctx;
  p->exch_buf = buf;
  p->exch_cap = cap;
  p->shard_stop = false;
  return MLMC_OK;
}

mlmc_status mlmc_plan_info(const mlmc_plan* p, int64_t* n, int64_t* nnz, int32_t* l0, double* t) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  if (n) *n = p->n;
  if (nnz) *nnz = p->nnz;
  if (l0) *l0 = p->l0;
  if (t) *t = p->t;
  return MLMC_OK;
}

int64_t mlmc_launch_count(const mlmc_plan* p) { return p ? p->launches : 0; }

void mlmc_plan_destroy(mlmc_plan* p) {
  // Lines this plan's windows left persisting go back to normal use.
  if (p && p->l2_persist_bytes > 0) {
    cudaStreamSynchronize(p->stream);
    cudaCtxResetPersistingL2Cache();
    cudaGetLastError();
  }
  free_plan(p);
}

mlmc_status mlmc_mlmcl(mlmc_plan* p, int32_t level, int32_t coarse, int64_t rep_begin,
                       int64_t reps, const double* v, uint64_t seed, double* sum_y,
                       double* totals) {
  if (!p || !v || !sum_y || !totals) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (level < 0 || level > 24 || (coarse && level < 1))
    return fail(MLMC_ERR_INVALID_ARG, "level must be in [0,24] (>= 1 when coarse)");
  if (p->source_active && (level < 1 || (coarse && level < 2)))
    return fail(MLMC_ERR_INVALID_ARG, "with a source term the level must be >= 1 (>= 2 when coarse)");
  if (!pieces_fit(p, level, coarse != 0))
    return fail(MLMC_ERR_INVALID_ARG, "the proposal's time pieces need 2^level (coarse: 2^(level-1)) "
                                      "to be a multiple of the piece count");
  if (rep_begin < 0 || reps < 0 || rep_begin > (1ll << 56) || reps > (1ll << 56) - rep_begin)
    return fail(MLMC_ERR_INVALID_ARG, "replica range out of [0, 2^56)");
  WalkLaunch w;
  w.level = level;
  w.coarse = coarse != 0;
  w.rep_begin = rep_begin;
  w.reps = reps;
  w.seed = seed;
  w.v = v;
  w.sum_y = sum_y;
  w.totals = totals;
  if (forward_mode(p)) {
    mlmc_status sst = prepare_starts(p, v);
    if (sst != MLMC_OK) return sst;
  }
  MLMC_CUDA(launch_any(p, w, nullptr), "walk kernel launch");
  return MLMC_OK;
}

// Largest n_times of the plan's walk precision (the kernels' per-lane sums).
static int max_times(const mlmc_plan* p) { return p->sched.precision == MLMC_FP64 ? 8 : 16; }

static mlmc_status check_times(const mlmc_plan* p, int32_t n_times, int32_t level) {
  if (forward_mode(p)) return fail(MLMC_ERR_INVALID_ARG, "intermediate times: backward-mode plans only");
  if (p->source_active) return fail(MLMC_ERR_INVALID_ARG, "intermediate times: remove the source term first");
  if (p->proposal_active && p->pieces > 1)
    return fail(MLMC_ERR_INVALID_ARG, "intermediate times: not with a proposal of time pieces");
  if (n_times < 2 || n_times > max_times(p) || (n_times & (n_times - 1)) != 0)
    return fail(MLMC_ERR_INVALID_ARG, "n_times must be a power of two in [2, " +
                                          std::to_string(max_times(p)) + "]");
  if (n_times > (1 << level))
    return fail(MLMC_ERR_INVALID_ARG, "n_times must not exceed 2^level (2^l0 for a solve)");
  return MLMC_OK;
}

mlmc_status mlmc_trace_times(mlmc_plan* p, int32_t level, int32_t coarse, int64_t rep_begin,
                             int64_t reps, const double* v, uint64_t seed, int32_t n_times,
                             mlmc_walk_record* rec, double* y_times) {
  if (!p || !v || !rec || !y_times) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (level < 0 || level > 24 || (coarse && level < 2))
    return fail(MLMC_ERR_INVALID_ARG, "level must be in [0,24] (>= 2 when coarse)");
  mlmc_status cst = check_times(p, n_times, coarse ? level - 1 : level);
  if (cst != MLMC_OK) return cst;
  if (rep_begin < 0 || reps < 0 || rep_begin > (1ll << 56) || reps > (1ll << 56) - rep_begin)
    return fail(MLMC_ERR_INVALID_ARG, "replica range out of [0, 2^56)");
  double* scratch = nullptr;
  const size_t ns = static_cast<size_t>(p->n) * static_cast<size_t>(n_times);
  MLMC_CUDA(dev_alloc(&scratch, ns + kTotSlots), "alloc trace sums");
  cudaError_t err = cudaMemsetAsync(scratch, 0, sizeof(double) * (ns + kTotSlots), p->stream);
  WalkLaunch w;
  w.level = level;
  w.coarse = coarse != 0;
  w.rep_begin = rep_begin;
  w.reps = reps;
  w.seed = seed;
  w.v = v;
  w.sum_y = scratch;
  w.totals = scratch + ns;
  w.sum_times = scratch + p->n;
  w.n_times = n_times;
  w.trace = rec;
  w.trace_times = y_times;
  if (err == cudaSuccess) err = launch_walk(p, w, nullptr);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  cudaFree(scratch);
  if (err != cudaSuccess) return cuda_fail(err, "trace launch");
  return MLMC_OK;
}

mlmc_status mlmc_trace(mlmc_plan* p, int32_t level, int32_t coarse, int64_t rep_begin,
                       int64_t reps, const double* v, uint64_t seed, mlmc_walk_record* rec) {
  if (!p || !v || !rec) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (level < 0 || level > 24 || (coarse && level < 1))
    return fail(MLMC_ERR_INVALID_ARG, "level must be in [0,24] (>= 1 when coarse)");
  if (p->source_active && (level < 1 || (coarse && level < 2)))
    return fail(MLMC_ERR_INVALID_ARG, "with a source term the level must be >= 1 (>= 2 when coarse)");
  if (!pieces_fit(p, level, coarse != 0))
    return fail(MLMC_ERR_INVALID_ARG, "the proposal's time pieces need 2^level (coarse: 2^(level-1)) "
                                      "to be a multiple of the piece count");
  if (rep_begin < 0 || reps < 0 || rep_begin > (1ll << 56) || reps > (1ll << 56) - rep_begin)
    return fail(MLMC_ERR_INVALID_ARG, "replica range out of [0, 2^56)");
  double* scratch = nullptr;
  MLMC_CUDA(dev_alloc(&scratch, static_cast<size_t>(p->n) + kTotSlots), "alloc trace sums");
  cudaError_t err = cudaMemsetAsync(scratch, 0, sizeof(double) * (p->n + kTotSlots), p->stream);
  WalkLaunch w;
  w.level = level;
  w.coarse = coarse != 0;
  w.rep_begin = rep_begin;
  w.reps = reps;
  w.seed = seed;
  w.v = v;
  w.sum_y = scratch;
  w.totals = scratch + p->n;
  w.trace = rec;
  if (err == cudaSuccess && forward_mode(p)) {
    mlmc_status sst = prepare_starts(p, v);
    if (sst != MLMC_OK) {
      cudaFree(scratch);
      return sst;
    }
  }
  if (err == cudaSuccess) err = launch_any(p, w, nullptr);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  cudaFree(scratch);
  if (err != cudaSuccess) return cuda_fail(err, "trace launch");
  return MLMC_OK;
}

// The controller of Algorithm 1 for one of three targets (Target above).
// They differ in the norm that sets eps, in the bias test and, in forward
// mode, in V_l.

static mlmc_status controller(mlmc_plan* p, const double* v, double* x, double* scalar,
                              uint64_t seed, Target target, bool resume = false) {
  const auto t_start = std::chrono::steady_clock::now();
  NvtxRange whole("mlmc controller");
  const mlmc_schedule& s = p->sched;
  MLMC_CUDA(cudaMemsetAsync(p->d_flags, 0, sizeof(uint32_t) * 4, p->stream), "memset flags");
  if (!resume) {
    MLMC_CUDA(cudaMemcpyAsync(p->d_v, v, sizeof(double) * p->n, cudaMemcpyDefault, p->stream), "copy v");
    MLMC_CUDA(cudaMemsetAsync(p->levels[0].sum_y, 0, sizeof(double) * p->n * s.max_levels, p->stream),
              "memset sums");
    MLMC_CUDA(cudaMemsetAsync(p->d_totals, 0, sizeof(double) * kTotSlots * s.max_levels, p->stream),
              "memset totals");
    if (p->ctl_times > 1)
      MLMC_CUDA(cudaMemsetAsync(p->d_times, 0, sizeof(double) * (kMaxTimesAll - 1) * p->n *
                                                   static_cast<size_t>(s.max_levels), p->stream),
                "memset time sums");
    for (auto& L : p->levels) {
      L.reps = 0;
      L.seconds = 0.0;
      L.launches = 0;
      L.pending = false;
    }
  }
  std::vector<char> timed(s.max_levels, 0);
  // A resumed solve continues the saved levels, sums and sample counts
  // (walk indices continue from M_l, so no walk is repeated).
  int nl = resume ? p->ctl_nl : s.num_levels;
  p->ctl_nl = nl;
  p->ctl_seed = seed;
  p->ctl_target = target;
  // Forward mode counts walks, not walks per row: the pilot and the budget
  // are scaled by n so that both modes spend the same effort.
  const int64_t unit = forward_mode(p) ? p->n : 1;
  const int64_t pilot = s.pilot_walks * unit;
  const double max_reps = static_cast<double>(s.max_walks_per_row) * static_cast<double>(unit);
  if (forward_mode(p)) {
    mlmc_status sst = prepare_starts(p, p->d_v);
    if (sst != MLMC_OK) return sst;
  }
  mlmc_status st = MLMC_OK;
  const auto deadline = t_start + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                      std::chrono::duration<double>(s.time_budget_s));
  bool out_of_time = false;
  for (int k = 0; k < nl && st == MLMC_OK && !resume; ++k)
    st = run_level(p, k, pilot, seed, timed, deadline, nullptr);
  if (st != MLMC_OK) return st;

  std::vector<HostLevel> h;
  double norm2 = 0.0;
  bool converged = false;
  mlmc_status result = MLMC_OK;
  auto past = [&]() { return std::chrono::steady_clock::now() > deadline; };
  for (int iter = 0; iter < 64; ++iter) {
    NvtxRange range("mlmc controller iteration");
    if ((st = collect(p, nl, h, &norm2, past())) != MLMC_OK) return st;
    auto size_of_x = [&]() {
      if (target == kFull) return std::sqrt(norm2);
      double tsum = 0.0;
      for (int k = 0; k < nl; ++k) tsum += h[k].sum / static_cast<double>(p->levels[k].reps);
      return std::fabs(tsum);
    };
    double eps = p->rel_tol * size_of_x();
    // Optimal sample sizes and top-up.
    std::vector<double> V(nl), C(nl);
    double root_sum = 0.0;
    for (int k = 0; k < nl; ++k) {
      V[k] = level_var(p, k, h[k], target);
      C[k] = level_cost(p, h[k]);
      root_sum += std::sqrt(V[k] * C[k]);
    }
    bool topped = false;
    if (eps > 0.0) {
      for (int k = 0; k < nl; ++k) {
        if (V[k] <= 0.0) continue;
        double want_reps = std::ceil(2.0 / (eps * eps) * std::sqrt(V[k] / C[k]) * root_sum);
        want_reps = std::min(want_reps, max_reps);
        const int64_t want = static_cast<int64_t>(want_reps);
        if (want > p->levels[k].reps) {
          if ((st = run_level(p, k, want - p->levels[k].reps, seed, timed, deadline,
                              &out_of_time)) != MLMC_OK)
            return st;
          topped = true;
          if (out_of_time) break;
        }
      }
    }
    if (topped) {
      if ((st = collect(p, nl, h, &norm2, past())) != MLMC_OK) return st;
      eps = p->rel_tol * size_of_x();
    }
    double var = 0.0;
    for (int k = 0; k < nl; ++k) var += level_var(p, k, h[k], target) / static_cast<double>(p->levels[k].reps);
    auto mnorm = [&](int k) {
      const double m = static_cast<double>(p->levels[k].reps);
      return (target == kFull ? std::sqrt(h[k].sumsq) : std::fabs(h[k].sum)) / m;
    };
    const double bias = nl > 1 ? std::max(mnorm(nl - 1), mnorm(nl - 2) / 4.0) / 3.0 : 0.0;
    const bool var_ok = var <= 0.5 * eps * eps * (1.0 + 1e-12);
    const bool bias_ok = bias <= eps / std::sqrt(2.0);
    const double xs = size_of_x();
    p->last_est_rel_err = xs > 0 ? std::sqrt(var) / xs : 0.0;
    if (var_ok && bias_ok) {
      converged = true;
      break;
    }
    // Sharded: the ranks stop together, on the vote of the last exchange.
    if (sharded(p) ? p->shard_stop : (out_of_time || past())) break;
    if (!bias_ok && nl < s.max_levels) {
      if ((st = run_level(p, nl, pilot, seed, timed, deadline, nullptr)) != MLMC_OK)
        return st;
      ++nl;
      p->ctl_nl = nl;
      continue;
    }
    bool capped = true;
    for (int k = 0; k < nl; ++k)
      if (level_var(p, k, h[k], target) > 0.0 && static_cast<double>(p->levels[k].reps) < max_reps)
        capped = false;
    if (capped || !bias_ok) break;
  }
  if (!converged) result = fail(MLMC_ERR_NOT_CONVERGED, "budget exhausted before the tolerance");

  // Final cross-level sum (Eq. 10) in FP64 and copy-out.
  if (target == kFull) {
    MLMC_CUDA(launch_finalize(p, nl, p->d_x, p->d_norm2), "finalize");
    if (p->ctl_times > 1) {
      // x holds n_times rows: the intermediate times first, the final one last
      const int64_t nt = static_cast<int64_t>(p->ctl_times - 1) * p->n;
      MLMC_CUDA(launch_finalize_times(p, nl, p->ctl_times, p->d_xtimes), "finalize times");
      MLMC_CUDA(cudaMemcpyAsync(x, p->d_xtimes, sizeof(double) * nt, cudaMemcpyDefault, p->stream),
                "copy x(t_k)");
      MLMC_CUDA(cudaMemcpyAsync(x + nt, p->d_x, sizeof(double) * p->n, cudaMemcpyDefault, p->stream),
                "copy x");
    } else {
      MLMC_CUDA(cudaMemcpyAsync(x, p->d_x, sizeof(double) * p->n, cudaMemcpyDefault, p->stream), "copy x");
    }
  } else {
    double tsum = 0.0;
    for (int k = 0; k < nl; ++k) tsum += h[k].sum / static_cast<double>(p->levels[k].reps);
    *scalar = tsum;
  }
  uint32_t flags = 0;
  if ((st = read_flags(p, &flags)) != MLMC_OK) return st;
  p->last_stats.clear();
  for (int k = 0; k < nl; ++k) {
    mlmc_level_stats ls{};
    ls.level = p->l0 + k;
    ls.walks_per_row = p->levels[k].reps;
    const double m = static_cast<double>(p->levels[k].reps);
    ls.mean_norm2 = h[k].sumsq / (m * m);
    ls.var = level_var(p, k, h[k], target);
    ls.cost_events_per_walk = h[k].walks > 0 ? 1.0 + h[k].jumps / h[k].walks : 1.0;
    ls.jumps = static_cast<int64_t>(h[k].jumps);
    ls.seconds = p->levels[k].seconds;
    ls.launches = p->levels[k].launches;
    ls.still_walks = static_cast<int64_t>(h[k].still);
    p->last_stats.push_back(ls);
  }
  if (flags & kFlagWalkLimit) return fail(MLMC_ERR_WALK_LIMIT, "walk limit:" + flag_text(flags));
  if (flags & kFlagNonFiniteY) return fail(MLMC_ERR_NUMERIC, "numeric:" + flag_text(flags));
  if (flags & kFlagBounds) return fail(MLMC_ERR_NUMERIC, "tables:" + flag_text(flags));
  return result;
}

mlmc_status mlmc_expmv(mlmc_plan* p, const double* v, double* x, uint64_t seed) {
  g_last_error.clear();
  if (!p || !v || !x) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  p->ctl_row_begin = 0;
  p->ctl_row_count = -1;
  return controller(p, v, x, nullptr, seed, kFull);
}

mlmc_status mlmc_expmv_times(mlmc_plan* p, const double* v, double* x_times, int32_t n_times,
                             uint64_t seed) {
  g_last_error.clear();
  if (!p || !v || !x_times) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  mlmc_status cst = check_times(p, n_times, p->l0);
  if (cst != MLMC_OK) return cst;
  if (sharded(p)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_expmv_times: not available on a sharded plan");
  if (!p->d_times) {
    MLMC_CUDA(dev_alloc(&p->d_times, static_cast<size_t>(kMaxTimesAll - 1) * static_cast<size_t>(p->n) *
                                         static_cast<size_t>(p->sched.max_levels)),
              "alloc time sums");
    MLMC_CUDA(dev_alloc(&p->d_xtimes, static_cast<size_t>(kMaxTimesAll - 1) * static_cast<size_t>(p->n)),
              "alloc x(t_k)");
  }
  p->ctl_row_begin = 0;
  p->ctl_row_count = -1;
  p->ctl_times = n_times;
  const mlmc_status st = controller(p, v, x_times, nullptr, seed, kFull);
  p->ctl_times = 0;
  return st;
}

mlmc_status mlmc_expmv_entry(mlmc_plan* p, int64_t i, const double* v, double* xi, uint64_t seed) {
  g_last_error.clear();
  if (!p || !v || !xi) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (i < 0 || i >= p->n) return fail(MLMC_ERR_INVALID_ARG, "row index out of range");
  if (forward_mode(p))
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_expmv_entry needs an MLMC_BACKWARD plan");
  p->ctl_row_begin = i;
  p->ctl_row_count = 1;
  const mlmc_status st = controller(p, v, nullptr, xi, seed, kEntry);
  p->ctl_row_begin = 0;
  p->ctl_row_count = -1;
  return st;
}

mlmc_status mlmc_expmv_sum(mlmc_plan* p, const double* v, double* total, uint64_t seed) {
  g_last_error.clear();
  if (!p || !v || !total) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  p->ctl_row_begin = 0;
  p->ctl_row_count = -1;
  return controller(p, v, nullptr, total, seed, kSum);
}


// The kind of law a saved state was walked with: 0 plain, 1 tilted jumps,
// 2 tilted clocks, 2 + K tilted clocks with K > 1 time pieces.
static int32_t proposal_code(const mlmc_plan* p) {
  if (!p->proposal_active) return 0;
  if (!p->clock_tilt) return 1;
  return p->pieces > 1 ? 2 + p->pieces : 2;
}

mlmc_status mlmc_plan_save_state(const mlmc_plan* p, void* buf, size_t cap, size_t* bytes) {
  if (!p || !bytes) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (sharded(p)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_save_state: not available on a sharded plan");
  if (p->ctl_target < 0) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_save_state: no solve to save");
  const int nl = p->ctl_nl;
  const size_t need = state_bytes(p, nl);
  *bytes = need;
  if (!buf) return MLMC_OK;
  if (cap < need) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_save_state: buffer too small");
  unsigned char* out = static_cast<unsigned char*>(buf);
  StateHeader h{};
  h.magic = kStateMagic;
  h.version = 1;
  h.nl = nl;
  h.n = p->n;
  h.nnz = p->nnz;
  h.t = p->t;
  h.l0 = p->l0;
  h.precision = p->sched.precision;
  h.mode = p->sched.mode;
  h.target = p->ctl_target;
  h.row_begin = p->ctl_row_begin;
  h.row_count = p->ctl_row_count;
  h.seed = p->ctl_seed;
  h.source = p->source_active ? 1 : 0;
  h.proposal = proposal_code(p);
  std::memcpy(out, &h, sizeof(h));
  out += sizeof(h);
  for (int k = 0; k < nl; ++k) {
    const StateLevel L{p->levels[k].reps, p->levels[k].seconds, p->levels[k].launches};
    std::memcpy(out, &L, sizeof(L));
    out += sizeof(L);
  }
  const size_t nt = static_cast<size_t>(nl) * kTotSlots;
  const size_t ns = static_cast<size_t>(nl) * p->n;
  MLMC_CUDA(cudaMemcpyAsync(out, p->d_totals, sizeof(double) * nt, cudaMemcpyDeviceToHost, p->stream), "save totals");
  out += sizeof(double) * nt;
  if (ns) MLMC_CUDA(cudaMemcpyAsync(out, p->levels[0].sum_y, sizeof(double) * ns, cudaMemcpyDeviceToHost, p->stream), "save sums");
  out += sizeof(double) * ns;
  MLMC_CUDA(cudaMemcpyAsync(out, p->d_v, sizeof(double) * p->n, cudaMemcpyDeviceToHost, p->stream), "save v");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  return MLMC_OK;
}

mlmc_status mlmc_plan_load_state(mlmc_plan* p, const void* buf, size_t bytes) {
  if (!p || !buf) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (sharded(p)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: not available on a sharded plan");
  if (bytes < sizeof(StateHeader)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: truncated state");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != 1)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: not a saved state");
  if (h.n != p->n || h.nnz != p->nnz || h.t != p->t || h.l0 != p->l0 ||
      h.precision != p->sched.precision || h.mode != p->sched.mode ||
      h.source != (p->source_active ? 1 : 0) || h.proposal != proposal_code(p))
    return fail(MLMC_ERR_INVALID_ARG,
                "mlmc_plan_load_state: the plan differs from the saved one (matrix size, t, l0, "
                "precision, mode, source or proposal)");
  if (h.nl < 1 || h.nl > p->sched.max_levels || h.target < 0 || h.target > 2)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: levels or target out of range");
  if (bytes != state_bytes(p, h.nl)) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: size mismatch");
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(h);
  MLMC_CUDA(cudaMemsetAsync(p->levels[0].sum_y, 0, sizeof(double) * p->n * p->sched.max_levels, p->stream),
            "memset sums");
  MLMC_CUDA(cudaMemsetAsync(p->d_totals, 0, sizeof(double) * kTotSlots * p->sched.max_levels, p->stream),
            "memset totals");
  for (auto& L : p->levels) {
    L.reps = 0;
    L.seconds = 0.0;
    L.launches = 0;
    L.pending = false;
  }
  for (int k = 0; k < h.nl; ++k) {
    StateLevel L;
    std::memcpy(&L, in, sizeof(L));
    in += sizeof(L);
    if (L.reps < 0) return fail(MLMC_ERR_INVALID_ARG, "mlmc_plan_load_state: negative sample count");
    p->levels[k].reps = L.reps;
    p->levels[k].seconds = L.seconds;
    p->levels[k].launches = L.launches;
  }
  const size_t nt = static_cast<size_t>(h.nl) * kTotSlots;
  const size_t ns = static_cast<size_t>(h.nl) * p->n;
  MLMC_CUDA(cudaMemcpyAsync(p->d_totals, in, sizeof(double) * nt, cudaMemcpyHostToDevice, p->stream), "load totals");
  in += sizeof(double) * nt;
  if (ns) MLMC_CUDA(cudaMemcpyAsync(p->levels[0].sum_y, in, sizeof(double) * ns, cudaMemcpyHostToDevice, p->stream), "load sums");
  in += sizeof(double) * ns;
  MLMC_CUDA(cudaMemcpyAsync(p->d_v, in, sizeof(double) * p->n, cudaMemcpyHostToDevice, p->stream), "load v");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  p->ctl_nl = h.nl;
  p->ctl_seed = h.seed;
  p->ctl_target = h.target;
  p->ctl_row_begin = h.row_begin;
  p->ctl_row_count = h.row_count;
  return MLMC_OK;
}

mlmc_status mlmc_expmv_resume(mlmc_plan* p, double* x) {
  if (p && sharded(p))
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_expmv_resume: not available on a sharded plan");
  g_last_error.clear();
  if (!p || !x) return fail(MLMC_ERR_INVALID_ARG, "NULL argument");
  if (p->ctl_target != kFull)
    return fail(MLMC_ERR_INVALID_ARG, "mlmc_expmv_resume: the last solve (or loaded state) is not an mlmc_expmv");
  p->ctl_row_begin = 0;
  p->ctl_row_count = -1;
  return controller(p, nullptr, x, nullptr, p->ctl_seed, kFull, true);
}

mlmc_status mlmc_stats(const mlmc_plan* p, mlmc_level_stats* out, int32_t cap, int32_t* n_levels,
                       double* est_rel_err) {
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  const int32_t nl = static_cast<int32_t>(p->last_stats.size());
  if (out)
    for (int32_t k = 0; k < nl && k < cap; ++k) out[k] = p->last_stats[k];
  if (n_levels) *n_levels = nl;
  if (est_rel_err) *est_rel_err = p->last_est_rel_err;
  return MLMC_OK;
}

mlmc_status mlmc_export_tables(const mlmc_plan* pc, double* l_ii, double* dl, double* inv_rate,
                               float* inv_rate32, float* dl32, int32_t* deg, uint32_t* thr,
                               int32_t* keep_col, uint8_t* keep_neg, int32_t* alias_col,
                               uint8_t* alias_neg) {
  mlmc_plan* p = const_cast<mlmc_plan*>(pc);
  if (!p) return fail(MLMC_ERR_INVALID_ARG, "NULL plan");
  std::vector<Meta32> m32(p->n);
  std::vector<Meta64> m64(p->n);
  std::vector<AliasEntry> al(p->nnz > 0 ? p->nnz : 1);
  std::vector<double> lii(p->n);
  MLMC_CUDA(cudaMemcpyAsync(m32.data(), p->d_meta32, sizeof(Meta32) * p->n, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaMemcpyAsync(m64.data(), p->d_meta64, sizeof(Meta64) * p->n, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaMemcpyAsync(lii.data(), p->d_lii, sizeof(double) * p->n, cudaMemcpyDeviceToHost, p->stream), "copy");
  if (p->nnz > 0)
    MLMC_CUDA(cudaMemcpyAsync(al.data(), p->d_alias, sizeof(AliasEntry) * p->nnz, cudaMemcpyDeviceToHost, p->stream), "copy");
  MLMC_CUDA(cudaStreamSynchronize(p->stream), "synchronize");
  for (int64_t i = 0; i < p->n; ++i) {
    if (l_ii) l_ii[i] = lii[i];
    if (dl) dl[i] = m64[i].dl;
    if (inv_rate) inv_rate[i] = m64[i].inv_rate;
    if (inv_rate32) inv_rate32[i] = m32[i].inv_rate;
    if (dl32) dl32[i] = m32[i].dl;
    if (deg) deg[i] = m32[i].deg;
    for (int32_t b = 0; b < m32[i].deg; ++b) {
      const AliasEntry& e = al[m32[i].start + b];
      const int64_t q = m32[i].start + b;
      if (thr) thr[q] = e.thr;
      if (keep_col) keep_col[q] = static_cast<int32_t>(e.keep & kColMask);
      if (keep_neg) keep_neg[q] = static_cast<uint8_t>(e.keep >> 31);
      if (alias_col) alias_col[q] = static_cast<int32_t>(e.alias & kColMask);
      if (alias_neg) alias_neg[q] = static_cast<uint8_t>(e.alias >> 31);
    }
  }
  return MLMC_OK;
}

}  // extern "C"
