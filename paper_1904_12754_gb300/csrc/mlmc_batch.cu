// Batched MLMC: many problems (a plan plus one right-hand side each; plans
// of different sizes, several right-hand sides per plan) solved together.
//
// The controller of Algorithm 1 runs for every problem in lockstep rounds.
// A round is one launch of one captured graph:
//   H2D  the round's segment table (pinned host buffer, fixed size): one
//        segment per (problem, level, replica range) with work to do;
//   k_walk_batch: one persistent walk kernel over every segment, warps
//        pulling (segment, row, chunk of walks) items from a global counter
//        and running the single-plan walk (screening, queues, the problem's
//        Philox keys) on the segment's tables;
//   H2D  reduction tasks; k_batch_reduce: sum_i S_l,i^2 for every active
//        (problem, level) and ||x||^2 for every active problem;
//   D2H  per-(problem, level) totals and per-problem norms (pinned)
// and the host synchronises once.  Between rounds the host applies each
// problem's sample-size rule (the same readings as the single-plan
// controller) and writes the next segment table.
//
// Launch shape (autotuner at batch creation, timed on the batch's own
// problems with the batch kernel): walks per lane of a work item (the item
// is 32 x that many walks of one row) per problem-size bucket from {4, 16,
// 64}, then threads per block from {128, 256} for the round kernel.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr int kRedBlock = 256;
constexpr int kBuckets = 3;  // n < 1e4, 1e4 <= n < 1e5, n >= 1e5
constexpr int64_t kRoundWalks = int64_t{1} << 35;  // walks per round, at most


struct ReduceTask {
  const double* vec;    // level sums S (sumsq task) or unused (norm task)
  double* out;          // where the result goes
  int64_t n;
  int32_t problem;      // norm task: problem index; sumsq task: -1
  int32_t pad;
};

// What the reduction kernels read of a problem: its per-level row sums.
struct BatchProblemDev {
  double* sums;         // [max_levels][n] per-level row sums of Y
  int64_t n;
};

struct BatchTables {
  int32_t ntasks;
  int32_t pad;
};

int bucket_of(int64_t n) { return n < 10000 ? 0 : (n < 100000 ? 1 : 2); }

__global__ void __launch_bounds__(kRedBlock)
    k_batch_reduce(const BatchTables* __restrict__ tab, const ReduceTask* __restrict__ tasks,
                   const BatchProblemDev* __restrict__ probs, const double* __restrict__ inv_m,
                   int max_levels) {
  __shared__ double part[kRedBlock / 32];
  for (int t = blockIdx.x; t < tab->ntasks; t += gridDim.x) {
    const ReduceTask task = tasks[t];
    double acc = 0.0;
    if (task.problem < 0) {
      for (int64_t i = threadIdx.x; i < task.n; i += kRedBlock) {
        const double x = task.vec[i];
        acc += x * x;
      }
    } else {
      const BatchProblemDev pb = probs[task.problem];
      const double* im = inv_m + static_cast<int64_t>(task.problem) * max_levels;
      for (int64_t i = threadIdx.x; i < task.n; i += kRedBlock) {
        double xi = 0.0;
        for (int l = 0; l < max_levels; ++l)
          if (im[l] != 0.0) xi += pb.sums[static_cast<int64_t>(l) * pb.n + i] * im[l];
        acc += xi * xi;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kRedBlock / 32; ++w) s += part[w];
      *task.out = s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRedBlock)
    k_batch_finalize(int nprob, const BatchProblemDev* __restrict__ probs,
                     const double* __restrict__ inv_m, int max_levels,
                     double* const* __restrict__ x_out) {
  for (int k = blockIdx.x; k < nprob; k += gridDim.x) {
    const BatchProblemDev pb = probs[k];
    const double* im = inv_m + static_cast<int64_t>(k) * max_levels;
    double* x = x_out[k];
    for (int64_t i = threadIdx.x; i < pb.n; i += kRedBlock) {
      double xi = 0.0;
      for (int l = 0; l < max_levels; ++l)
        if (im[l] != 0.0) xi += pb.sums[static_cast<int64_t>(l) * pb.n + i] * im[l];
      x[i] = xi;
    }
  }
}

__global__ void k_batch_to_float(int64_t total, const double* __restrict__ in,
                                 float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}

mlmc_status bfail(mlmc_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

mlmc_status bcuda(cudaError_t e, const char* what) {
  return bfail(e == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA,
               std::string("batch ") + what + ": " + cudaGetErrorString(e));
}

#define BATCH_CUDA(call, what)                     \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return bcuda(e_, what); \
  } while (0)

struct ProblemState {
  int nl = 0;
  bool done = false;
  bool converged = false;
  std::vector<int64_t> reps;      // per slot
  std::vector<int64_t> launches;  // per slot
  double est_rel_err = 0.0;
};

}  // namespace
}  // namespace mlmc

using namespace mlmc;

struct mlmc_batch {
  std::vector<mlmc_plan*> plans;   // one per problem
  int nprob = 0;
  int max_levels = 0;
  mlmc_schedule sched{};
  double rel_tol = 0.0;
  bool fp64 = false;
  int num_sms = 0;
  int device = 0;
  cudaStream_t stream = nullptr;   // controller stream: the round graph, copies
  cudaStream_t caller = nullptr;
  int block = 256;                 // threads per block of the round kernel (autotuned)
  std::vector<int64_t> n;          // per problem
  std::vector<int64_t> offset;     // row offset of each problem in the contiguous buffers
  int64_t total_rows = 0;
  int per_lane[kBuckets] = {16, 16, 64};  // candidates of the autotuner

  // Device buffers.
  BatchProblemDev* d_probs = nullptr;
  double* d_sums = nullptr;        // per problem: max_levels * n
  double* d_totals = nullptr;      // nprob * max_levels * kTotSlots
  double* d_norm = nullptr;        // nprob
  double* d_v = nullptr;           // total_rows
  float* d_v32 = nullptr;          // total_rows
  double* d_x = nullptr;           // total_rows
  double** d_xptr = nullptr;       // nprob pointers into d_x
  unsigned long long* d_work = nullptr;  // the round kernel's work counter
  // Segment table of a round (device + pinned host mirror):
  // [BatchRound][max_segs x BatchSeg]
  unsigned char* d_round = nullptr;
  unsigned char* h_round = nullptr;
  size_t round_bytes = 0;
  int max_segs = 0;
  uint32_t* d_flags = nullptr;
  // Round table (device + pinned host mirror): [BatchTables][tasks][inv_m]
  unsigned char* d_tab = nullptr;
  unsigned char* h_tab = nullptr;
  size_t tab_bytes = 0, off_tasks = 0, off_invm = 0;
  int max_tasks = 0;
  double* h_totals = nullptr;      // pinned
  double* h_norm = nullptr;        // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int64_t rounds = 0;
  int64_t launches = 0;            // walk launches of the last mlmc_batch_expmv
  std::vector<ProblemState> state;
  double last_seconds = 0.0;
};

namespace {

void free_batch(mlmc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_probs);
  cudaFree(b->d_sums);
  cudaFree(b->d_totals);
  cudaFree(b->d_norm);
  cudaFree(b->d_v);
  cudaFree(b->d_v32);
  cudaFree(b->d_x);
  cudaFree(b->d_xptr);
  cudaFree(b->d_work);
  cudaFree(b->d_flags);
  cudaFree(b->d_tab);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  if (b->h_totals) cudaFreeHost(b->h_totals);
  if (b->h_norm) cudaFreeHost(b->h_norm);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  cudaFree(b->d_round);
  if (b->h_round) cudaFreeHost(b->h_round);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

BatchTables* tab_hdr(mlmc_batch* b) { return reinterpret_cast<BatchTables*>(b->h_tab); }
ReduceTask* tab_tasks(mlmc_batch* b) { return reinterpret_cast<ReduceTask*>(b->h_tab + b->off_tasks); }
double* tab_invm(mlmc_batch* b) { return reinterpret_cast<double*>(b->h_tab + b->off_invm); }

// The graph of a round's reductions: upload the task table, reduce, read the
// totals and norms back.
mlmc_status capture_round_graph(mlmc_batch* b) {
  const BatchTables* dt = reinterpret_cast<const BatchTables*>(b->d_tab);
  const ReduceTask* dtasks = reinterpret_cast<const ReduceTask*>(b->d_tab + b->off_tasks);
  const double* dinvm = reinterpret_cast<const double*>(b->d_tab + b->off_invm);
  const BatchRound* dround = reinterpret_cast<const BatchRound*>(b->d_round);
  const BatchSeg* dsegs = reinterpret_cast<const BatchSeg*>(b->d_round + 256);
  BATCH_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t err = cudaMemcpyAsync(b->d_round, b->h_round, b->round_bytes, cudaMemcpyHostToDevice,
                                    b->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), b->stream);
  if (err == cudaSuccess)
    err = launch_walk_batch(b->fp64, dround, dsegs, b->d_work, b->d_flags, b->num_sms, b->block,
                            b->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(b->d_tab, b->h_tab, b->tab_bytes, cudaMemcpyHostToDevice, b->stream);
  if (err == cudaSuccess) {
    k_batch_reduce<<<b->num_sms * 8, kRedBlock, 0, b->stream>>>(dt, dtasks, b->d_probs, dinvm,
                                                                  b->max_levels);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(b->h_totals, b->d_totals,
                          sizeof(double) * b->nprob * b->max_levels * kTotSlots,
                          cudaMemcpyDeviceToHost, b->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(b->h_norm, b->d_norm, sizeof(double) * b->nprob, cudaMemcpyDeviceToHost,
                          b->stream);
  cudaGraph_t g = nullptr;
  cudaError_t end = cudaStreamEndCapture(b->stream, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(err, "capture");
  }
  if (end != cudaSuccess) return bcuda(end, "end capture");
  b->graph = g;
  BATCH_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
  return MLMC_OK;
}

BatchRound* round_hdr(mlmc_batch* b) { return reinterpret_cast<BatchRound*>(b->h_round); }
BatchSeg* round_segs(mlmc_batch* b) { return reinterpret_cast<BatchSeg*>(b->h_round + 256); }

// Segment of problem k, level slot l: walks rep_begin .. rep_begin+reps-1 of
// every row, walks per lane of an item per_lane; its items start at `first`.
BatchSeg make_seg(mlmc_batch* b, int k, int l, int64_t rep_begin, int64_t reps, int64_t per_lane,
                  uint64_t seed, unsigned long long first) {
  mlmc_plan* p = b->plans[k];
  const int64_t L = b->max_levels;
  BatchSeg g{};
  g.meta = walk_meta(p, b->fp64);
  g.alias = p->proposal_active ? static_cast<const void*>(p->d_alias_is)
                               : static_cast<const void*>(p->d_fused);
  g.v_walk = b->fp64 ? static_cast<const void*>(b->d_v + b->offset[k])
                     : static_cast<const void*>(b->d_v32 + b->offset[k]);
  g.still32 = walk_still32(p);
  g.sum_y = b->d_sums + b->offset[k] * L + static_cast<int64_t>(l) * b->n[k];
  g.totals = b->d_totals + (static_cast<int64_t>(k) * L + l) * kTotSlots;
  g.n = b->n[k];
  g.nnz = p->nnz;
  g.rep_begin = rep_begin;
  g.reps = reps;
  per_lane = std::max<int64_t>(1, std::min<int64_t>(per_lane, (reps + 31) / 32));
  g.chunk = 32 * per_lane;
  g.chunks_per_row = (reps + g.chunk - 1) / g.chunk;
  g.item_begin = first;
  g.max_jumps = p->sched.max_jumps_per_walk;
  g.level = p->l0 + l;
  g.coarse = l > 0 ? 1 : 0;
  g.is = p->proposal_active ? 1 : 0;
  g.ctr3 = static_cast<uint32_t>(g.level) & 0x3Fu;
  g.rk = philox_round_keys(static_cast<uint32_t>(seed & 0xFFFFFFFFull), static_cast<uint32_t>(seed >> 32));
  return g;
}

unsigned long long seg_items(const BatchSeg& g) {
  return static_cast<unsigned long long>(g.n) * static_cast<unsigned long long>(g.chunks_per_row);
}

// Autotuner trial: one launch of the round kernel over the given problems'
// l0 walks (reps per row each, into the batch's sums, which every
// mlmc_batch_expmv clears), timed with events; ms per walk.
double trial_round(mlmc_batch* b, const std::vector<int>& probs, int64_t reps, int64_t per_lane,
                   int block) {
  BatchSeg* segs = round_segs(b);
  unsigned long long items = 0;
  int nseg = 0;
  int64_t walks = 0;
  for (int k : probs) {
    segs[nseg] = make_seg(b, k, 0, 0, reps, per_lane, 0x5eedull, items);
    items += seg_items(segs[nseg]);
    walks += reps * b->n[k];
    ++nseg;
  }
  round_hdr(b)->total_items = items;
  round_hdr(b)->nseg = nseg;
  const BatchRound* dround = reinterpret_cast<const BatchRound*>(b->d_round);
  const BatchSeg* dsegs = reinterpret_cast<const BatchSeg*>(b->d_round + 256);
  cudaMemcpyAsync(b->d_round, b->h_round, b->round_bytes, cudaMemcpyHostToDevice, b->stream);
  cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long), b->stream);
  cudaEventRecord(b->ev0, b->stream);
  cudaError_t err = launch_walk_batch(b->fp64, dround, dsegs, b->d_work, b->d_flags, b->num_sms,
                                      block, b->stream);
  cudaEventRecord(b->ev1, b->stream);
  cudaEventSynchronize(b->ev1);
  float ms = 0.f;
  if (err != cudaSuccess || cudaEventElapsedTime(&ms, b->ev0, b->ev1) != cudaSuccess) return 1e30;
  return static_cast<double>(ms) / static_cast<double>(walks > 0 ? walks : 1);
}

}  // namespace

extern "C" {

mlmc_status mlmc_batch_create(mlmc_batch** out, mlmc_plan* const* plans, int32_t count,
                              const mlmc_schedule* sched, double rel_tol, void* cuda_stream) {
  if (!out) return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: NULL out");
  *out = nullptr;
  if (!plans || count < 1) return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: need >= 1 plan");
  if (!(rel_tol > 0.0) || !std::isfinite(rel_tol))
    return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: rel_tol must be finite and > 0");
  mlmc_batch* b = new mlmc_batch();
  auto bail = [&](mlmc_status st) {
    free_batch(b);
    return st;
  };
  b->nprob = count;
  b->sched = sched ? *sched : plans[0]->sched;
  b->rel_tol = rel_tol;
  b->caller = static_cast<cudaStream_t>(cuda_stream);
  if (b->sched.num_levels < 1 || b->sched.max_levels < b->sched.num_levels || b->sched.max_levels > 32 ||
      b->sched.pilot_walks < 2)
    return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: bad schedule"));
  b->max_levels = b->sched.max_levels;
  b->fp64 = plans[0]->sched.precision == MLMC_FP64;
  for (int k = 0; k < count; ++k) {
    mlmc_plan* p = plans[k];
    if (!p) return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: NULL plan"));
    if (p->sched.mode != MLMC_BACKWARD)
      return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: backward-mode plans only"));
    if (p->source_active)
      return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: plans with a source term are not batched"));
    if (p->proposal_active && p->pieces > 1)
      return bail(bfail(MLMC_ERR_INVALID_ARG,
                        "mlmc_batch_create: proposals with time pieces are not batched"));
    if ((p->sched.precision == MLMC_FP64) != b->fp64)
      return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: plans differ in precision"));
    if (p->device != plans[0]->device)
      return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: plans on different devices"));
    if (p->l0 + b->max_levels - 1 > 24)
      return bail(bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_create: levels above 24 for a plan"));
    b->plans.push_back(p);
    b->offset.push_back(b->total_rows);
    b->n.push_back(p->n);
    b->total_rows += p->n;
    cudaError_t e = cudaStreamSynchronize(p->stream);  // tables ready
    if (e != cudaSuccess) return bail(bcuda(e, "plan stream"));
  }
  b->device = plans[0]->device;
  b->num_sms = plans[0]->num_sms;
#define BC(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return bail(bcuda(e_, what));  \
  } while (0)
  BC(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
  BC(cudaEventCreate(&b->ev0), "event");
  BC(cudaEventCreate(&b->ev1), "event");
  const int64_t L = b->max_levels;
  BC(cudaMalloc(&b->d_probs, sizeof(BatchProblemDev) * count), "alloc");
  BC(cudaMalloc(&b->d_sums, sizeof(double) * b->total_rows * L), "alloc sums");
  BC(cudaMalloc(&b->d_totals, sizeof(double) * count * L * kTotSlots), "alloc");
  BC(cudaMalloc(&b->d_norm, sizeof(double) * count), "alloc");
  BC(cudaMalloc(&b->d_v, sizeof(double) * b->total_rows), "alloc");
  BC(cudaMalloc(&b->d_v32, sizeof(float) * b->total_rows), "alloc");
  BC(cudaMalloc(&b->d_x, sizeof(double) * b->total_rows), "alloc");
  BC(cudaMalloc(&b->d_xptr, sizeof(double*) * count), "alloc");
  BC(cudaMalloc(&b->d_work, sizeof(unsigned long long)), "alloc");
  b->max_segs = static_cast<int>(count * L);
  b->round_bytes = 256 + sizeof(BatchSeg) * static_cast<size_t>(b->max_segs);
  BC(cudaMalloc(&b->d_round, b->round_bytes), "alloc segment table");
  BC(cudaMallocHost(&b->h_round, b->round_bytes), "alloc pinned segment table");
  std::memset(b->h_round, 0, b->round_bytes);
  BC(cudaMalloc(&b->d_flags, sizeof(uint32_t) * 4), "alloc");
  b->max_tasks = static_cast<int>(count * L + count);
  b->off_tasks = 256;
  b->off_invm = b->off_tasks + ((sizeof(ReduceTask) * b->max_tasks + 255) / 256) * 256;
  b->tab_bytes = b->off_invm + sizeof(double) * count * L;
  BC(cudaMalloc(&b->d_tab, b->tab_bytes), "alloc table");
  BC(cudaMallocHost(&b->h_tab, b->tab_bytes), "alloc pinned table");
  BC(cudaMallocHost(&b->h_totals, sizeof(double) * count * L * kTotSlots), "alloc pinned");
  BC(cudaMallocHost(&b->h_norm, sizeof(double) * count), "alloc pinned");
  std::memset(b->h_tab, 0, b->tab_bytes);
  std::vector<BatchProblemDev> probs(count);
  std::vector<double*> xptr(count);
  for (int k = 0; k < count; ++k) {
    probs[k].sums = b->d_sums + b->offset[k] * L;
    probs[k].n = b->n[k];
    xptr[k] = b->d_x + b->offset[k];
  }
  BC(cudaMemcpy(b->d_probs, probs.data(), sizeof(BatchProblemDev) * count, cudaMemcpyHostToDevice),
     "upload problems");
  BC(cudaMemcpy(b->d_xptr, xptr.data(), sizeof(double*) * count, cudaMemcpyHostToDevice), "upload");

  // Autotuner, timed with the round kernel on this batch's problems at their
  // l0 (zero right-hand sides; the trial's sums are cleared by every solve):
  // walks per lane of a work item per problem-size bucket from {4, 16, 64}
  // (256 walks per row, the bucket's problems only), then threads per block
  // of the round kernel from {128, 256} (every problem).  Blocks of 512 would
  // need the walk's per-warp queues of 16 warps in one block's shared memory
  // (over 48 KB for FP64 walks).
  {
    BC(cudaMemsetAsync(b->d_v, 0, sizeof(double) * b->total_rows, b->stream), "memset");
    BC(cudaMemsetAsync(b->d_v32, 0, sizeof(float) * b->total_rows, b->stream), "memset");
    BC(cudaMemsetAsync(b->d_sums, 0, sizeof(double) * b->total_rows * L, b->stream), "memset");
    BC(cudaMemsetAsync(b->d_totals, 0, sizeof(double) * count * L * kTotSlots, b->stream), "memset");
    std::vector<int> all;
    for (int bk = 0; bk < kBuckets; ++bk) {
      std::vector<int> members;
      for (int k = 0; k < count; ++k)
        if (bucket_of(b->n[k]) == bk) members.push_back(k);
      all.insert(all.end(), members.begin(), members.end());
      if (members.empty()) continue;
      double best = 1e300;
      for (int cand : {4, 16, 64}) {
        trial_round(b, members, 256, cand, 256);  // warm
        const double t = trial_round(b, members, 256, cand, 256);
        if (t < best) {
          best = t;
          b->per_lane[bk] = cand;
        }
      }
    }
    double best = 1e300;
    for (int blk : {128, 256}) {
      BatchSeg* segs = round_segs(b);
      (void)segs;
      // per-bucket walks per lane as tuned: one trial per bucket's problems
      double t = 0.0;
      for (int bk = 0; bk < kBuckets; ++bk) {
        std::vector<int> members;
        for (int k = 0; k < count; ++k)
          if (bucket_of(b->n[k]) == bk) members.push_back(k);
        if (members.empty()) continue;
        trial_round(b, members, 256, b->per_lane[bk], blk);  // warm
        t += trial_round(b, members, 256, b->per_lane[bk], blk);
      }
      if (t < best) {
        best = t;
        b->block = blk;
      }
    }
    BC(cudaStreamSynchronize(b->stream), "autotune");
  }
  {
    mlmc_status st = capture_round_graph(b);
    if (st != MLMC_OK) return bail(st);
  }
#undef BC
  *out = b;
  return MLMC_OK;
}

void mlmc_batch_destroy(mlmc_batch* b) { free_batch(b); }

mlmc_status mlmc_batch_autotune(const mlmc_batch* b, int32_t* walks_per_lane, int32_t cap) {
  if (!b || !walks_per_lane) return bfail(MLMC_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < kBuckets && k < cap; ++k) walks_per_lane[k] = b->per_lane[k];
  if (cap > kBuckets) walks_per_lane[kBuckets] = b->block;
  return MLMC_OK;
}

mlmc_status mlmc_batch_expmv(mlmc_batch* b, const double* const* v, double* const* x,
                             const uint64_t* seeds) {
  if (!b || !v || !x || !seeds) return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_expmv: NULL argument");
  const auto t_start = std::chrono::steady_clock::now();
  const auto deadline = t_start + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                      std::chrono::duration<double>(b->sched.time_budget_s));
  const int K = b->nprob;
  const int64_t L = b->max_levels;
  for (int k = 0; k < K; ++k)
    if (b->plans[k]->proposal_active && b->plans[k]->pieces > 1)
      return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_expmv: proposals with time pieces are not batched");
  BATCH_CUDA(cudaEventRecord(b->ev0, b->caller), "event");
  BATCH_CUDA(cudaStreamWaitEvent(b->stream, b->ev0, 0), "wait");
  for (int k = 0; k < K; ++k) {
    if (!v[k] || !x[k]) return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_expmv: NULL v/x entry");
    BATCH_CUDA(cudaMemcpyAsync(b->d_v + b->offset[k], v[k], sizeof(double) * b->n[k],
                               cudaMemcpyDefault, b->stream), "copy v");
  }
  if (!b->fp64) {
    k_batch_to_float<<<b->num_sms * 8, 256, 0, b->stream>>>(b->total_rows, b->d_v, b->d_v32);
    BATCH_CUDA(cudaGetLastError(), "to float");
  }
  BATCH_CUDA(cudaMemsetAsync(b->d_sums, 0, sizeof(double) * b->total_rows * L, b->stream), "memset");
  BATCH_CUDA(cudaMemsetAsync(b->d_totals, 0, sizeof(double) * K * L * kTotSlots, b->stream), "memset");
  BATCH_CUDA(cudaMemsetAsync(b->d_flags, 0, sizeof(uint32_t) * 4, b->stream), "memset");
  b->state.assign(K, ProblemState());
  for (auto& s : b->state) {
    s.nl = b->sched.num_levels;
    s.reps.assign(L, 0);
    s.launches.assign(L, 0);
  }
  // Pending work per (problem, slot): walks per row still to launch.
  std::vector<int64_t> want(K * L, 0);
  for (int k = 0; k < K; ++k)
    for (int l = 0; l < b->sched.num_levels; ++l) want[k * L + l] = b->sched.pilot_walks;
  b->rounds = 0;
  b->launches = 0;
  double gpu_s = 0.0;
  bool out_of_time = false;
  for (;;) {
    NvtxRange range("mlmc batch round");
    // The round's walks: a table of segments of bounded total size, walked
    // by one launch of the round kernel inside the round graph.
    BATCH_CUDA(cudaEventRecord(b->ev0, b->stream), "event");
    BatchSeg* segs = round_segs(b);
    int nseg = 0;
    int64_t walks = 0;
    unsigned long long items = 0;
    for (int k = 0; k < K; ++k) {
      ProblemState& s = b->state[k];
      if (s.done) continue;
      for (int l = 0; l < s.nl; ++l) {
        int64_t reps = want[k * L + l];
        if (reps <= 0) continue;
        if (walks >= kRoundWalks || nseg >= b->max_segs) break;
        const int64_t room = std::max<int64_t>(1, (kRoundWalks - walks) / b->n[k]);
        reps = std::min(reps, room);
        segs[nseg] = make_seg(b, k, l, s.reps[l], reps, b->per_lane[bucket_of(b->n[k])], seeds[k],
                              items);
        items += seg_items(segs[nseg]);
        ++nseg;
        s.launches[l] += 1;
        walks += reps * b->n[k];
        want[k * L + l] -= reps;
        s.reps[l] += reps;
      }
    }
    round_hdr(b)->total_items = items;
    round_hdr(b)->nseg = nseg;
    if (nseg > 0) ++b->launches;
    // Reduction tasks of every active problem.
    BatchTables* th = tab_hdr(b);
    ReduceTask* tasks = tab_tasks(b);
    double* invm = tab_invm(b);
    int ntask = 0;
    for (int k = 0; k < K; ++k) {
      ProblemState& s = b->state[k];
      for (int l = 0; l < L; ++l)
        invm[k * L + l] = (l < s.nl && s.reps[l] > 0) ? 1.0 / static_cast<double>(s.reps[l]) : 0.0;
      if (s.done) continue;
      for (int l = 0; l < s.nl; ++l) {
        ReduceTask& t = tasks[ntask++];
        t.vec = b->d_sums + b->offset[k] * L + static_cast<int64_t>(l) * b->n[k];
        t.out = b->d_totals + (static_cast<int64_t>(k) * L + l) * kTotSlots + kTotSumSq;
        t.n = b->n[k];
        t.problem = -1;
      }
      ReduceTask& t = tasks[ntask++];
      t.vec = nullptr;
      t.out = b->d_norm + k;
      t.n = b->n[k];
      t.problem = k;
    }
    if (nseg == 0 && ntask == 0) break;
    th->ntasks = ntask;
    BATCH_CUDA(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    BATCH_CUDA(cudaEventRecord(b->ev1, b->stream), "event");
    BATCH_CUDA(cudaStreamSynchronize(b->stream), "sync");
    float ms = 0.f;
    BATCH_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1), "elapsed");
    gpu_s += 1e-3 * ms;
    ++b->rounds;
    if (std::chrono::steady_clock::now() > deadline) out_of_time = true;
    // Controller step for every problem whose pending walks are all done.
    bool any_pending = false;
    for (int k = 0; k < K; ++k) {
      ProblemState& s = b->state[k];
      if (s.done) continue;
      bool pending = false;
      for (int l = 0; l < s.nl; ++l) pending |= want[k * L + l] > 0;
      if (pending) {
        any_pending = true;
        continue;
      }
      const double* tt = b->h_totals + static_cast<int64_t>(k) * L * kTotSlots;
      const double norm2 = b->h_norm[k];
      const double eps = b->rel_tol * std::sqrt(norm2);
      std::vector<double> V(s.nl), C(s.nl);
      double root_sum = 0.0, var = 0.0;
      for (int l = 0; l < s.nl; ++l) {
        const double* t = tt + l * kTotSlots;
        const double m = static_cast<double>(s.reps[l]);
        V[l] = m >= 2 ? std::max(0.0, (t[kTotY2] - t[kTotSumSq] / m) / (m - 1.0)) : 0.0;
        C[l] = static_cast<double>(b->n[k]) * (t[kTotWalks] > 0 ? 1.0 + t[kTotJumps] / t[kTotWalks] : 1.0);
        root_sum += std::sqrt(V[l] * C[l]);
        var += V[l] / m;
      }
      auto mnorm = [&](int l) { return std::sqrt(tt[l * kTotSlots + kTotSumSq]) / static_cast<double>(s.reps[l]); };
      const double bias = s.nl > 1 ? std::max(mnorm(s.nl - 1), mnorm(s.nl - 2) / 4.0) / 3.0 : 0.0;
      s.est_rel_err = norm2 > 0 ? std::sqrt(var / norm2) : 0.0;
      const bool var_ok = var <= 0.5 * eps * eps * (1.0 + 1e-12);
      const bool bias_ok = bias <= eps / std::sqrt(2.0);
      if (var_ok && bias_ok) {
        s.done = true;
        s.converged = true;
        continue;
      }
      if (out_of_time) {
        s.done = true;
        continue;
      }
      bool added = false;
      if (eps > 0.0 && !var_ok) {
        for (int l = 0; l < s.nl; ++l) {
          if (V[l] <= 0.0) continue;
          double target = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * root_sum);
          target = std::min(target, static_cast<double>(b->sched.max_walks_per_row));
          const int64_t w = static_cast<int64_t>(target) - s.reps[l];
          if (w > 0) {
            want[k * L + l] = w;
            added = true;
          }
        }
      }
      if (!added && !bias_ok && s.nl < b->max_levels) {
        want[k * L + s.nl] = b->sched.pilot_walks;
        ++s.nl;
        added = true;
      }
      if (!added) {
        s.done = true;  // budget per row exhausted
        continue;
      }
      any_pending = true;
    }
    if (!any_pending) {
      bool all_done = true;
      for (auto& s : b->state) all_done &= s.done;
      if (all_done) break;
    }
  }
  // Final cross-level sums (FP64) into the caller's buffers.
  {
    double* invm = tab_invm(b);
    for (int k = 0; k < K; ++k)
      for (int l = 0; l < L; ++l)
        invm[k * L + l] = (l < b->state[k].nl && b->state[k].reps[l] > 0)
                              ? 1.0 / static_cast<double>(b->state[k].reps[l]) : 0.0;
    BATCH_CUDA(cudaMemcpyAsync(b->d_tab + b->off_invm, invm, sizeof(double) * K * L,
                               cudaMemcpyHostToDevice, b->stream), "upload inv m");
    k_batch_finalize<<<b->num_sms * 4, kRedBlock, 0, b->stream>>>(
        K, b->d_probs, reinterpret_cast<const double*>(b->d_tab + b->off_invm), b->max_levels,
        b->d_xptr);
    BATCH_CUDA(cudaGetLastError(), "finalize");
    for (int k = 0; k < K; ++k)
      BATCH_CUDA(cudaMemcpyAsync(x[k], b->d_x + b->offset[k], sizeof(double) * b->n[k],
                                 cudaMemcpyDefault, b->stream), "copy x");
    uint32_t flags = 0;
    BATCH_CUDA(cudaMemcpyAsync(&flags, b->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream),
               "flags");
    BATCH_CUDA(cudaStreamSynchronize(b->stream), "sync");
    b->last_seconds = gpu_s;
    if (flags & kFlagWalkLimit) return bfail(MLMC_ERR_WALK_LIMIT, "batch: a walk exceeded max_jumps_per_walk");
    if (flags & kFlagNonFiniteY) return bfail(MLMC_ERR_NUMERIC, "batch: non-finite walk weight");
    if (flags & kFlagBounds) return bfail(MLMC_ERR_NUMERIC, "batch: table index out of range");
  }
  for (auto& s : b->state)
    if (!s.converged) return bfail(MLMC_ERR_NOT_CONVERGED, "batch: budget exhausted before the tolerance");
  return MLMC_OK;
}

mlmc_status mlmc_batch_stats(const mlmc_batch* b, int32_t problem, mlmc_level_stats* out,
                             int32_t cap, int32_t* n_levels, double* est_rel_err) {
  if (!b || problem < 0 || problem >= b->nprob || b->state.empty())
    return bfail(MLMC_ERR_INVALID_ARG, "mlmc_batch_stats: bad batch or problem index");
  const ProblemState& s = b->state[problem];
  const int64_t L = b->max_levels;
  const double* tt = b->h_totals + static_cast<int64_t>(problem) * L * kTotSlots;
  for (int l = 0; l < s.nl && l < cap && out; ++l) {
    const double* t = tt + l * kTotSlots;
    const double m = static_cast<double>(s.reps[l]);
    mlmc_level_stats ls{};
    ls.level = b->plans[problem]->l0 + l;
    ls.walks_per_row = s.reps[l];
    ls.mean_norm2 = m > 0 ? t[kTotSumSq] / (m * m) : 0.0;
    ls.var = m >= 2 ? std::max(0.0, (t[kTotY2] - t[kTotSumSq] / m) / (m - 1.0)) : 0.0;
    ls.cost_events_per_walk = t[kTotWalks] > 0 ? 1.0 + t[kTotJumps] / t[kTotWalks] : 1.0;
    ls.jumps = static_cast<int64_t>(t[kTotJumps]);
    ls.seconds = 0.0;
    ls.launches = s.launches[l];
    ls.still_walks = static_cast<int64_t>(t[kTotStill]);
    out[l] = ls;
  }
  if (n_levels) *n_levels = s.nl;
  if (est_rel_err) *est_rel_err = s.est_rel_err;
  return MLMC_OK;
}

mlmc_status mlmc_batch_info(const mlmc_batch* b, int64_t* rounds, double* gpu_seconds,
                            int32_t* converged) {
  if (!b) return bfail(MLMC_ERR_INVALID_ARG, "NULL batch");
  if (rounds) *rounds = b->rounds;
  if (gpu_seconds) *gpu_seconds = b->last_seconds;
  if (converged) {
    int c = 0;
    for (auto& s : b->state) c += s.converged ? 1 : 0;
    *converged = c;
  }
  return MLMC_OK;
}

}  // extern "C"
