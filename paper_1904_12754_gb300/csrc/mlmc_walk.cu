// The walk kernel: MLMCL of Algorithm 2 for every row, event-driven.
//
// A walk of row i at level l (N = 2^l intervals of scaled time 1/N) is the
// continuous-time Markov chain of Sec. 3 in scaled time s = tau/t: in state j
// it holds for an Exp(t L_jj) time, then jumps to k with probability
// |a_jk|/L_jj (alias table) and multiplies its sign by sign(a_jk).  Instead of
// stepping through the N intervals (the paper's O(N) loop), the kernel visits
// only events and counts grid points in closed form: a jump at time s falls
// after grid point g = floor(s N) (exact: N is a power of two), so the state
// held on (a, b] of grid indices contributes
//   fine   (b - a)              grid points of level l,
//   coarse floor(b/2) - floor(a/2) grid points of level l-1,
//   and to the fine-minus-coarse difference (b mod 2) - (a mod 2),
// with the first segment starting at a = -1 and the last ending at b = N.
// Then, with h = (dl_start + dl_end)/2 (the half-weighted endpoints of Eq. 7),
//   E_f = (acc_f - h)/N,  E_c = (acc_c - h)/(N/2),  E_f - E_c = (acc_d + h)/N
// and the sample is Y = sign v_end e^{E_f} at the coarsest level and
// Y = sign v_end e^{E_c} expm1(E_f - E_c) above it (Fig. 1; no cancellation).
// Draws are Philox4x32-10 blocks, counter (rep_lo, row, draw index, level |
// rep_hi << 8), key = seed.  FP64 walks: draw k gives the k-th holding time
// (words 0-1) and the bucket and alias coin of the jump that ends it (words
// 2-3).  FP32 walks (one word per uniform): draw k gives the (k+1)-th jump
// (words 2-3) and the holding time after it (word 0); the first holding time
// is word 1 of draw 0, or a word of a block shared by four walks in rows
// whose walks rarely jump.  An FP32 walk thus draws once per jump.
//
// Work decomposition: a warp takes one (row, chunk of walks) item at a time
// from a global counter.  Its lanes first screen the chunk's walks (first
// holding time only; FP32: 128 walks per round from 32 Philox blocks, four
// walks per block): walks that never jump are counted, the others go to a
// per-warp queue in shared memory, from which a lane whose walk ends takes
// the next one at once, so lanes stay busy although walk lengths are
// geometric.  Per-row sums are reduced across the warp and added
// with one FP64 atomic per item; totals are flushed once per warp.
// The FP32 variant keeps times, exponents and weights in FP32 and sums Y per
// row with Kahan compensation and sum Y^2 (which sets the sample sizes through
// the variance estimate) as an exact-product FP32 pair; FP64 appears only in
// the per-item warp reductions and the atomics.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Checked build (-DMLMC_CHECKED): every alias-entry index and every state a
// jump picks is compared with the table sizes before it is used; a walk that
// would leave them ends (status 2, sample 0) and sets kFlagBounds.
#ifdef MLMC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

struct WalkArgs {
  const void* meta;
  const void* alias;       // AliasEntry, or AliasEntryIS with a proposal
  const void* v_walk;      // right-hand side in the walk precision
  int64_t n;
  int64_t nnz;
  int64_t rep_begin;
  int64_t reps;
  int64_t chunk;           // walks per item (multiple of 32)
  int64_t chunks_per_row;
  unsigned long long total_items;
  int64_t row_begin;       // first row of the launch
  int level;
  uint32_t ctr3;           // level | stream << 6
  uint32_t key0, key1;
  PhiloxRoundKeys rk;      // round keys of (key0, key1)
  int64_t max_jumps;
  double* sum_y;
  double* totals;
  uint32_t* flags;
  unsigned long long* work;
  mlmc_walk_record* trace;
  int64_t trace_stride;    // records per row (the whole replica range)
  int64_t trace_base;      // offset of this launch's first replica
  const void* f_walk;      // source vector in the walk precision (source walks only)
  double t;                // the time t (source walks only)
  const int32_t* still32;  // FP32: per-row still threshold index (still_index32)
  int pieces;              // proposal walks: time pieces K of the law (1: one law)
  int n_times;             // intermediate-time walks: output times (T), else 0
  double* sum_times;       // [(T-1) x n] per-row sums of the samples at t k/T, k < T
  double* trace_times;     // trace: [(T-1)] samples per record (or null)
};

// Key source of the walk's draws: the round keys of a launch-constant
// parameter, so that every round's key add is an operand of the constant bank.
struct KeysFromParam {
  const PhiloxRoundKeys* rk;
  __device__ __forceinline__ uint4 draw(uint4 c) const { return philox4x32_10(c, *rk); }
};

template <bool FP64>
struct Prec;

template <>
struct Prec<false> {
  using T = float;
  using Meta = Meta32;
  using VT = float;
  __device__ static T uniform(uint4 x) { return uniform32(x.x); }
  __device__ static T neglog(T u) { return neglog32(u); }
  __device__ static T mul(T a, T b) { return __fmul_rn(a, b); }
  __device__ static T add(T a, T b) { return __fadd_rn(a, b); }
  __device__ static T sub(T a, T b) { return __fsub_rn(a, b); }
  __device__ static T fma(T a, T b, T c) { return __fmaf_rn(a, b, c); }
  __device__ static T div(T a, T b) { return __fdiv_rn(a, b); }
  __device__ static T inf() { return __int_as_float(0x7f800000); }
  __device__ static T from_int(int x) { return static_cast<float>(x); }
  __device__ static T ex(T a) { return expf(a); }
  __device__ static T exm1(T a) { return expm1f(a); }
  __device__ static int floor_int(T a) { return static_cast<int>(floorf(a)); }
};

template <>
struct Prec<true> {
  using T = double;
  using Meta = Meta64;
  using VT = double;
  __device__ static T uniform(uint4 x) { return uniform64(x.x, x.y); }
  __device__ static T neglog(T u) { return neglog64(u); }
  __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
  __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
  __device__ static T sub(T a, T b) { return __dsub_rn(a, b); }
  __device__ static T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
  __device__ static T div(T a, T b) { return __ddiv_rn(a, b); }
  __device__ static T inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  __device__ static T from_int(int x) { return static_cast<double>(x); }
  __device__ static T ex(T a) { return exp(a); }
  __device__ static T exm1(T a) { return expm1(a); }
  __device__ static int floor_int(T a) { return static_cast<int>(floor(a)); }
};

// Compensated (Kahan) accumulator.
template <typename T>
struct Kahan {
  T s = 0, c = 0;
  __device__ void add(T y);
};
template <>
__device__ void Kahan<float>::add(float y) {
  const float yy = __fsub_rn(y, c);
  const float tt = __fadd_rn(s, yy);
  c = __fsub_rn(__fsub_rn(tt, s), yy);
  s = tt;
}
template <>
__device__ void Kahan<double>::add(double y) {
  s = __dadd_rn(s, y);
}

// Sum of non-negative terms kept as an unevaluated FP32 pair (hi + lo): each
// y^2 enters as its exact product split (fl(y*y), fma error) and the running
// sum uses Fast2Sum (|hi| >= each term).  Used for sum Y^2, whose
// cancellation against (sum Y)^2/M decides the variance estimate.
template <typename T>
struct SquareSum;
template <>
struct SquareSum<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_square(float y) {
    const float p = __fmul_rn(y, y);
    const float pe = __fmaf_rn(y, y, -p);
    const float t = __fadd_rn(hi, p);
    const float e = __fsub_rn(p, __fsub_rn(t, hi));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};
template <>
struct SquareSum<double> {
  double hi = 0.0;
  __device__ __forceinline__ void add_square(double y) { hi = __dadd_rn(hi, __dmul_rn(y, y)); }
  __device__ __forceinline__ double value() const { return hi; }
};

// Warp sum of a (sum, compensation) pair into one double.
template <typename T>
__device__ __forceinline__ double warp_sum(const Kahan<T>& k) {
  double v = static_cast<double>(k.s) - static_cast<double>(k.c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename Meta>
__device__ __forceinline__ Meta load_meta(const Meta* m, int64_t j);

template <>
__device__ __forceinline__ Meta64 load_meta<Meta64>(const Meta64* m, int64_t j) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(m + j));
  const double2 b = __ldg(reinterpret_cast<const double2*>(m + j) + 1);
  Meta64 out;
  out.start = a.x;
  out.deg = a.y;
  out.pad0 = 0;
  out.pad1 = 0;
  out.inv_rate = b.x;
  out.dl = b.y;
  return out;
}

template <>
__device__ __forceinline__ Meta32 load_meta<Meta32>(const Meta32* m, int64_t j) {
  const int4 r = __ldg(reinterpret_cast<const int4*>(m) + j);
  Meta32 out;
  out.start = r.x;
  out.deg = r.y;
  out.inv_rate = __int_as_float(r.z);
  out.dl = __int_as_float(r.w);
  return out;
}

// Walk-side parameters of one work item's walks (one plan or one batch
// problem).
struct ItemArgs {
  const void* meta;
  const void* alias;      // AliasEntry, or AliasEntryIS with a proposal
  const void* v_walk;
  int level;
  uint32_t ctr3;
  uint32_t key0, key1;
  int64_t max_jumps;
  double* sum_y;
  int64_t rep_begin;
  mlmc_walk_record* trace;
  int64_t trace_stride;
  int64_t trace_base;
  const void* f_walk;     // source vector (source walks only)
  double t;               // the time t (source walks only)
  int64_t n, nnz;         // table sizes (checked build)
  const int32_t* still32; // FP32: per-row still threshold index
  int pieces;             // proposal walks: time pieces K (1: one law)
  int n_times;            // intermediate times (T), 0 without
  double* sum_times;
  double* trace_times;
};

// Per-warp running totals of the walks a warp has finished.
template <typename T>
struct WalkTotals {
  SquareSum<T> y2;
  double y2_fixed = 0.0;  // per-item constant part (walks without a jump)
  unsigned long long jumps = 0, walks = 0, limit = 0, still = 0;
  uint32_t bad = 0;
};

// Add a warp's totals into totals[] (one lane) and clear them.
template <typename T>
__device__ __forceinline__ void flush_totals(WalkTotals<T>& t, double* totals, uint32_t* flags,
                                             int lane) {
  double y2 = t.y2.value() + t.y2_fixed;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y2 += __shfl_xor_sync(kFull, y2, o);
  const unsigned long long jw = warp_sum_u64(t.jumps);
  const unsigned long long ww = warp_sum_u64(t.walks);
  const unsigned long long lw = warp_sum_u64(t.limit);
  const unsigned long long sw = warp_sum_u64(t.still);
  const uint32_t bad = __reduce_or_sync(kFull, t.bad);
  if (lane == 0) {
    if (ww) {
      atomicAdd(totals + kTotY2, y2);
      atomicAdd(totals + kTotJumps, static_cast<double>(jw));
      atomicAdd(totals + kTotWalks, static_cast<double>(ww));
      if (lw) atomicAdd(totals + kTotLimit, static_cast<double>(lw));
      if (sw) atomicAdd(totals + kTotStill, static_cast<double>(sw));
    }
    if (bad) atomicOr(flags, bad);
  }
  t = WalkTotals<T>();
}

// Totals of the backward walk kernels, split by who updates them: the sum
// of Y^2 and the error flags per lane (registers), the counters per warp
// (shared memory, written by lane 0 after a warp reduction per item).
template <typename T>
struct LaneTotals {
  SquareSum<T> y2;
  uint32_t bad = 0;
};
struct WarpCounters {
  double y2_fixed;  // walks without a jump: count x y_still^2 per item
  unsigned long long jumps, walks, limit, still;
};

// Add a warp's totals into totals[] (one lane) and clear them.
template <typename T>
__device__ __forceinline__ void flush_warp(LaneTotals<T>& t, WarpCounters* wc, double* totals,
                                           uint32_t* flags, int lane) {
  double y2 = t.y2.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y2 += __shfl_xor_sync(kFull, y2, o);
  const uint32_t bad = __reduce_or_sync(kFull, t.bad);
  __syncwarp();
  if (lane == 0) {
    if (wc->walks) {
      atomicAdd(totals + kTotY2, y2 + wc->y2_fixed);
      atomicAdd(totals + kTotJumps, static_cast<double>(wc->jumps));
      atomicAdd(totals + kTotWalks, static_cast<double>(wc->walks));
      if (wc->limit) atomicAdd(totals + kTotLimit, static_cast<double>(wc->limit));
      if (wc->still) atomicAdd(totals + kTotStill, static_cast<double>(wc->still));
    }
    if (bad) atomicOr(flags, bad);
    wc->y2_fixed = 0.0;
    wc->jumps = wc->walks = wc->limit = wc->still = 0;
  }
  __syncwarp();
  t = LaneTotals<T>();
}

// Per-warp queue of screened walks that jump at least once, a ring of
// WarpQueue<FP64>::kCap slots.  A screening round runs only while fewer than
// 32 walks are queued, so the queue never holds more than 31 plus one round's
// walks.  FP32: replica offset and the Philox word of the first holding time
// (the first jump's words come from the walk's own draw 0 when it is taken);
// a round screens 32 blocks of 4 walks, at most 128 entries, so never more
// than 159 are queued.  FP64: replica offset, the first holding time and the
// first jump's bucket and coin words; a round screens kWays = 2 walks per
// lane, at most 64 entries, never more than 95.
template <bool FP64>
struct WarpQueue;
template <>
struct WarpQueue<false> {
  static constexpr uint32_t kCap = 256;
  uint32_t r[kCap];
  uint32_t first[kCap];
};
template <>
struct WarpQueue<true> {
  static constexpr uint32_t kCap = 128;
  uint32_t r[kCap];
  uint32_t xz[kCap];
  uint32_t xw[kCap];
  double first[kCap];
};
// Screening rounds: FP32 32 blocks of 4 walks, FP64 kScreenWays walks per
// lane; the bound above must fit the rings, whose sizes are powers of two
// (slots are taken modulo the size).
constexpr uint32_t kScreenWalks32 = 32u * 4u;
constexpr uint32_t kScreenWays = 2u;
static_assert(31u + kScreenWalks32 <= WarpQueue<false>::kCap, "FP32 screening queue too small");
static_assert(31u + 32u * kScreenWays <= WarpQueue<true>::kCap, "FP64 screening queue too small");
static_assert((WarpQueue<false>::kCap & (WarpQueue<false>::kCap - 1)) == 0, "ring size");
static_assert((WarpQueue<true>::kCap & (WarpQueue<true>::kCap - 1)) == 0, "ring size");
constexpr uint32_t kQueueCap = 64;  // the end queue's ring
// FP32 walks of rows that are not screened (long walks): jumps a lane makes
// per iteration of the one-wave loop before the warp's claim and end votes.
#ifndef MLMC_LONG_EVENTS
#define MLMC_LONG_EVENTS 2
#endif
constexpr int kLongEvents = MLMC_LONG_EVENTS;
static_assert(kLongEvents >= 1 && kLongEvents <= 8, "jumps per iteration");

// Per-warp queue of walks that ended at s = 1 (their samples are evaluated 32
// at a time): the exponents and the end state with the sign in bit 31.  At
// most 32 are added per iteration and fewer than 32 are left after one, so
// it never holds more than 63.
template <bool FP64>
struct EndQueue {
  typename std::conditional<FP64, double, float>::type x1[kQueueCap];
  typename std::conditional<FP64, double, float>::type x2[kQueueCap];
  uint32_t js[kQueueCap];
};
constexpr int kMaxWarps = 8;  // blocks of at most 256 threads

// Intermediate times (mlmc_expmv_times): a walk also samples x(t k/T) at the
// fine grid points g_k = k N/T, k = 1..T-1, from its prefix; each lane sums
// its walks' samples per time here (per warp: [T-1][32]) and the warp adds
// them to the row's sums once per work item.
// At most 16 output times for FP32 walks and 8 for FP64 walks (the block's
// static shared memory stays below 48 KB).
constexpr int kMaxTimes32 = 16;
constexpr int kMaxTimes64 = 8;
template <bool FP64, bool TIMES>
struct TimesAcc {
  typename std::conditional<FP64, double, float>::type
      v[TIMES ? (FP64 ? kMaxTimes64 : kMaxTimes32) - 1 : 1][32];
};

// Source term (Algorithm 3, Simpson's rule on a grid of K steps, K even): the
// weighted sum over grid points k in (a, b] of w_k e^{W_k / K}, where the walk
// holds one state (scaled rate term dl) on (a, b], W_k = P_a + (k - a) dl -
// (dl0 + dl)/2 is the Strang exponent at grid point k (P_a: the sum of the
// scaled d of the states at grid points 0..a, dl0: the start state's), and
// w_k = 1 at k = 0 and k = K, 4 at odd k, 2 at even k in between.  With
// r = e^{dl/K} the terms are geometric: sum_k (3 - (-1)^k) r^k in closed
// form, minus one term at each end point of the grid that (a, b] contains.
template <bool FP64>
__device__ __forceinline__ typename Prec<FP64>::T simpson_segment(
    int a, int b, int K, typename Prec<FP64>::T inv_k, typename Prec<FP64>::T pa,
    typename Prec<FP64>::T dl, typename Prec<FP64>::T dl0) {
  using P = Prec<FP64>;
  using T = typename P::T;
  const int L = b - a;
  if (L <= 0) return static_cast<T>(0);
  const T h = P::mul(dl, inv_k);  // exponent step per grid step
  // exponent at grid point a + 1
  const T e1 = P::mul(P::add(P::sub(pa, P::mul(dl0, static_cast<T>(0.5))),
                             P::mul(dl, static_cast<T>(0.5))), inv_k);
  const T em1 = P::exm1(P::mul(P::from_int(L), h));           // r^L - 1
  // sum_{q < L} r^q and sum_{q < L} (-r)^q = (1 - (-r)^L) / (1 + r)
  const T g1 = (h == static_cast<T>(0)) ? P::from_int(L) : em1 / P::exm1(h);
  const T rl = P::add(em1, static_cast<T>(1));
  const T g2 = ((L & 1) ? P::add(static_cast<T>(1), rl) : P::sub(static_cast<T>(1), rl)) /
               P::add(static_cast<T>(1), P::ex(h));
  // (3 - (-1)^k) r^k summed over k = a+1 .. b, divided by r^{a+1}
  const T sgeo = ((a + 1) & 1) ? P::add(P::mul(static_cast<T>(3), g1), g2)
                               : P::sub(P::mul(static_cast<T>(3), g1), g2);
  T total = P::mul(P::ex(e1), sgeo);
  if (a < 0) total = P::sub(total, static_cast<T>(1));       // k = 0: weight 1, e^0
  if (b == K)                                                 // k = K: weight 1
    total = P::sub(total, P::ex(P::add(e1, P::mul(P::from_int(K - a - 1), h))));
  return total;
}

// One work item: walks r_lo .. r_hi-1 (replica offsets relative to
// a.rep_begin) of row `row`, run by the whole warp in two interleaved stages.
//   screen  the 32 lanes draw the first holding time of 64 (FP64) or 128
//           (FP32) new walks; a walk whose first time reaches s = 1 never
//           leaves the row (its sample is the same for every such walk: it is
//           only counted), the others are queued;
//   walk    lanes without a walk take queued ones.  FP64: an iteration has
//           two waves: the refilled lanes make their first jump with the
//           queued draw, then every live lane draws its next holding time and
//           jumps or ends.  FP32: every live lane takes its pending jump with
//           one draw, which also gives the holding time after the jump, and
//           ends if that time reaches s = 1.  Either way most walks finish in
//           one iteration with the draw on (nearly) all lanes.
// Rows whose walks are long (t L_row > 1) are not screened: an iteration is
// one event per lane, a lane whose walk ends claims the next walk index at
// once (ballot + prefix count), and the samples of ended walks are evaluated
// 32 at a time from a second queue (few lanes end per iteration).
// Screening runs whenever fewer than 32 walks are queued, so every lane of
// the walk stage has work while any is left, and walks that never jump (most
// of them when t L_ii is small) cost one draw at full SIMD width instead of a
// pass through the jump and end paths.  A walk's draws depend only on its own
// counter, so the trajectories are those of the walk-by-walk definition.
// Adds the item's sum of Y to a.sum_y[row] (one atomic) and its totals to
// `tot`.
template <bool FP64, bool COARSE, bool TRACE, bool IS, class Keys, bool SRC = false,
          bool TIMES = false, bool PIECES = false>
__device__ __forceinline__ void walk_item(const ItemArgs& a, const Keys& keys, int64_t row,
                                          int64_t r_lo, int64_t r_hi,
                                          LaneTotals<typename Prec<FP64>::T>& tot,
                                          WarpCounters* __restrict__ wc,
                                          WarpQueue<FP64>* __restrict__ q,
                                          EndQueue<FP64>* __restrict__ eq,
                                          TimesAcc<FP64, TIMES>* __restrict__ ta, int lane) {
  using P = Prec<FP64>;
  using T = typename P::T;
  using Meta = typename P::Meta;
  using VT = typename P::VT;
  const Meta* __restrict__ meta = static_cast<const Meta*>(a.meta);
  const VT* __restrict__ vv = static_cast<const VT*>(a.v_walk);
  const int n_grid = 1 << a.level;                 // fine grid points 0..N
  const T n_fine = P::from_int(n_grid);
  const T inv_n = static_cast<T>(1.0 / n_grid);  // exact: a power of two
  const int n_coarse = n_grid >> 1;
  // Time pieces (proposal walks, R19): piece p's alias entries follow
  // piece p-1's, nnz apart; the row records are state-major, state j's record
  // of piece p at j K + p (one cache line for a state's pieces); a pending
  // jump time that reaches the current piece's end b_next is carried into
  // the next piece.
  static_assert(!PIECES || (IS && !SRC && !TIMES), "time pieces: proposal walks without source or times");
  const int n_pieces = PIECES ? a.pieces : 1;
  const Meta m0 = load_meta(meta, row * n_pieces);
  const T dl0 = static_cast<T>(m0.dl);
  const T inv_rate0 = static_cast<T>(m0.inv_rate);
  const int g_per = n_grid / n_pieces;  // fine grid points per piece (K divides N)
  const T inv_pieces = P::div(static_cast<T>(1), P::from_int(n_pieces));  // exact: K = 2^k
  const T b_first = n_pieces > 1 ? inv_pieces : P::inf();
  // Rows whose walks are short (t L_row <= 1: few events per walk, the
  // first jump and the end usually fall in the same iteration) are screened;
  // the others run one event per lane per iteration without screening.
  // (FP64 walks with time pieces are not screened: their screening tests
  // the first holding time before any carry-over.)
  constexpr int kWays = static_cast<int>(kScreenWays);  // FP64 screening: walks per lane per round
  const bool screened_row = static_cast<T>(m0.inv_rate) >= static_cast<T>(1) &&
                            !(FP64 && n_pieces > 1);
  // FP32: a screened walk never jumps exactly when its first uniform's index
  // is <= the row's threshold index (computed once per row with the tables).
  const int32_t still_max = (FP64 || !screened_row) ? 0 : __ldg(a.still32 + row);
  // A walk that never jumps stays at the row for the whole interval: its
  // sample is 0 above l0 and v_row e^{dl_row} at l0 (E_f = dl_row exactly
  // as the grid weights sum to 1), the same for every such walk.
  // With time pieces E_f is the mean of the row's d over the pieces (every
  // boundary is a grid point).
  T y_still = 0;
  if (!COARSE) {
    T dl_still = dl0;
    if (PIECES && n_pieces > 1) {
      T sum = dl0;
      for (int pp = 1; pp < n_pieces; ++pp)
        sum = P::add(sum, static_cast<T>(load_meta(meta, row * n_pieces + pp).dl));
      dl_still = P::mul(sum, inv_pieces);
    }
    y_still = P::mul(static_cast<T>(__ldg(vv + row)), P::ex(dl_still));
  }
  // Source term: the sample also gets t/(3N) times the fine Simpson sum
  // minus, above l0, 2t/(3N) times the coarse one (level l-1's rule on the
  // even grid points).  A walk that never jumps has a fixed source part.
  const VT* __restrict__ ff = static_cast<const VT*>(a.f_walk);
  const T src_scale_f = SRC ? static_cast<T>(a.t / (3.0 * n_grid)) : static_cast<T>(0);
  const T src_scale_c = SRC ? static_cast<T>(2.0 * a.t / (3.0 * n_grid)) : static_cast<T>(0);
  const T inv_nc = P::mul(inv_n, static_cast<T>(2));
  if (SRC) {
    const T fr = static_cast<T>(__ldg(ff + row));
    T ys = P::mul(src_scale_f,
                  P::mul(fr, simpson_segment<FP64>(-1, n_grid, n_grid, inv_n, static_cast<T>(0),
                                                   dl0, dl0)));
    if (COARSE)
      ys = P::sub(ys, P::mul(src_scale_c,
                             P::mul(fr, simpson_segment<FP64>(-1, n_coarse, n_coarse, inv_nc,
                                                              static_cast<T>(0), dl0, dl0))));
    y_still = P::add(y_still, ys);
  }
  if (!isfinite(y_still)) {
    tot.bad |= kFlagNonFiniteY;
    y_still = 0;
  }

  Kahan<T> acc_y;
  uint32_t item_jumps = 0;  // this lane's jumps in this item (< 2^32)
  uint32_t n_still = 0;     // walks of one-wave rows that ended without a jump
  uint32_t n_limit = 0;     // this lane's walks stopped at the jump limit
  const uint32_t row32 = static_cast<uint32_t>(row);
  const uint32_t span = static_cast<uint32_t>(r_hi - r_lo);
  const uint64_t rep_base = static_cast<uint64_t>(a.rep_begin + r_lo);
  const unsigned lanes_below = (1u << lane) - 1u;
  uint32_t screened = 0;           // warp-uniform: walks screened so far
  uint32_t qhead = 0, qtail = 0;   // warp-uniform queue positions
  uint32_t ehead = 0, etail = 0;   // warp-uniform end-queue positions
  uint32_t claimed = 0;            // warp-uniform: walks claimed (one-wave rows)
  bool live = false;               // this lane holds a walk
  // Walk state.
  uint32_t r = 0, c_lo = 0, c_hi = 0;  // replica offset and its counter words
  Meta m = m0;
  int32_t j = static_cast<int32_t>(row);
  uint32_t e = 0;          // jumps taken (= Philox draw index)
  uint32_t neg = 0;        // sign bit of the product of jump signs
  T s = 0;                 // current time in [0,1)
  T acc = 0;               // coarse: acc_c; coarsest: acc_f
  T acc_d = 0;             // coarse only
  int kprev = -1;          // grid index of the segment start (fine)
  T lw = 0;                // proposal only: sum of log(k/q) over the jumps
  uint32_t hash = 2166136261u;
  T src_f = 0, src_c = 0;  // source only: fine and coarse Simpson sums so far
  // FP32: the walk's next jump time (< 1), known before the draw that gives
  // the jump's words; `fresh`: claimed, first holding time not drawn yet.
  T s_pend = 0;
  bool fresh = false;
  int pc = 0;          // time piece of the walk (proposal walks)
  T b_next = b_first;  // its end (infinite in the last piece)
  // Intermediate times: output k < T at fine grid point k * t_stride.
  const int t_stride = TIMES ? n_grid / a.n_times : 1;
  const int n_out = TIMES ? a.n_times - 1 : 0;

  // Start walk r of the item (state at s = 0 in the row).
  auto start_walk = [&](uint32_t r_new) {
    r = r_new;
    const uint64_t rep = rep_base + r;
    c_lo = static_cast<uint32_t>(rep);
    c_hi = a.ctr3 | (static_cast<uint32_t>(rep >> 32) << 8);
    m = m0;
    j = static_cast<int32_t>(row);
    e = 0;
    neg = 0;
    s = 0;
    acc = 0;
    acc_d = 0;
    kprev = -1;
    lw = 0;
    hash = 2166136261u;
    src_f = 0;
    src_c = 0;
    pc = 0;
    b_next = b_first;
  };
  // Source term: add the Simpson sums of the segment (kprev, b] held in
  // state j (sign neg) before the exponent sums move past it.
  auto source_segment = [&](int b) {
    const T fj = static_cast<T>(__ldg(ff + j));
    const T sfj = neg ? -fj : fj;
    const T dlj = static_cast<T>(m.dl);
    const T pa = COARSE ? P::add(P::add(acc, acc), acc_d) : acc;  // fine prefix at kprev
    src_f = P::add(src_f, P::mul(sfj, simpson_segment<FP64>(kprev, b, n_grid, inv_n, pa, dlj, dl0)));
    if (COARSE)
      src_c = P::add(src_c, P::mul(sfj, simpson_segment<FP64>(kprev >> 1, b >> 1, n_coarse, inv_nc,
                                                             acc, dlj, dl0)));
  };
  // Intermediate times: the samples at the output grid points in (kprev, g],
  // all held in the current state j (prefix exponents as in exponents()
  // with the grid ending at the output point), added to this lane's sums.
  auto emit_times = [&](int g) {
    if constexpr (TIMES) {
      const T dlj = static_cast<T>(m.dl);
      const T vj = static_cast<T>(__ldg(vv + j));
      const T h = P::mul(P::add(dl0, dlj), static_cast<T>(0.5));
      // the first output after grid point kprev (kprev = -1 before the first
      // jump: C++ division truncates toward zero, so that case is explicit)
      int k = kprev < 0 ? 1 : kprev / t_stride + 1;
      const int k_hi = min(g / t_stride, n_out);
      for (; k <= k_hi; ++k) {
        const int gk = k * t_stride;
        T y;
        if (COARSE) {
          const T acc_c = P::fma(P::from_int((gk >> 1) - (kprev >> 1)), dlj, acc);
          const T accd = P::fma(P::from_int(-(kprev & 1)), dlj, acc_d);
          T x1 = P::mul(P::sub(acc_c, h), P::mul(inv_n, static_cast<T>(2)));
          if (IS) x1 = P::add(x1, lw);
          const T x2 = P::mul(P::add(accd, h), inv_n);
          y = P::mul(vj, P::mul(P::ex(x1), P::exm1(x2)));
        } else {
          const T acc_f = P::fma(P::from_int(gk - kprev), dlj, acc);
          T x1 = P::mul(P::sub(acc_f, h), inv_n);
          if (IS) x1 = P::add(x1, lw);
          y = P::mul(vj, P::ex(x1));
        }
        if (neg) y = -y;
        if (!isfinite(y)) {
          tot.bad |= kFlagNonFiniteY;
          y = 0;
        }
        ta->v[k - 1][lane] = P::add(ta->v[k - 1][lane], y);
        if (TRACE)
          a.trace_times[(row * a.trace_stride + a.trace_base + (r_lo + r)) * n_out + (k - 1)] =
              static_cast<double>(y);
      }
    }
  };
  // The still sample at output k (a walk that never leaves the row).
  auto still_time = [&](int k) -> T {
    if (COARSE) return static_cast<T>(0);
    return P::mul(static_cast<T>(__ldg(vv + row)),
                  P::ex(P::mul(P::mul(P::from_int(k * t_stride), dl0), inv_n)));
  };
  // Jump at time s_new (after fine grid point g) with bucket word xz and
  // alias coin xw: count the grid points of the segment that ends, pick the
  // next state from the alias table of the current one.
  auto jump = [&](T s_new, uint32_t xz, uint32_t xw) -> bool {
    const int g = P::floor_int(P::mul(s_new, n_fine));
    if (SRC) source_segment(g);
    if (TIMES) emit_times(g);
    const T dlj = static_cast<T>(m.dl);
    if (COARSE) {
      const int kc_prev = kprev >> 1;   // floor(a/2), also for a = -1
      acc = P::fma(P::from_int((g >> 1) - kc_prev), dlj, acc);
      acc_d = P::fma(P::from_int((g & 1) - (kprev & 1)), dlj, acc_d);
    } else {
      acc = P::fma(P::from_int(g - kprev), dlj, acc);
    }
    kprev = g;
    const uint32_t bucket = __umulhi(xz, static_cast<uint32_t>(m.deg));
    if (kChecked && (m.start < 0 || static_cast<int64_t>(m.start) + bucket >= a.nnz)) return false;
    uint32_t pick;
    Meta mnext{};
    if (IS) {
      const uint4* ep = reinterpret_cast<const uint4*>(
          static_cast<const AliasEntryIS*>(a.alias) + (PIECES ? static_cast<int64_t>(pc) * a.nnz : 0) +
          m.start + bucket);
      const uint4 e0 = __ldg(ep);
      const uint2 e1 = __ldg(reinterpret_cast<const uint2*>(ep + 1));
      const bool keep = xw < e0.x;
      pick = keep ? e0.y : e0.z;
      lw = P::add(lw, static_cast<T>(__uint_as_float(keep ? e1.x : e1.y)));
    } else {
      // the fused entry: both candidates' row records arrive with it
      using Fused = typename std::conditional<FP64, FusedEntry64, FusedEntry32>::type;
      const Fused* fe = static_cast<const Fused*>(a.alias) + m.start + bucket;
      const uint4 ent = __ldg(reinterpret_cast<const uint4*>(fe));
      const Meta mk = load_meta(&fe->mk, 0);
      const Meta ma = load_meta(&fe->ma, 0);
      const bool keep = xw < ent.x;
      pick = keep ? ent.y : ent.z;
      mnext = keep ? mk : ma;
    }
    if (kChecked && static_cast<int64_t>(pick & kColMask) >= a.n) return false;
    neg ^= pick >> 31;
    j = static_cast<int32_t>(pick & kColMask);
    if (TRACE) hash = (hash ^ static_cast<uint32_t>(j)) * 16777619u;
    m = IS ? load_meta(meta, PIECES ? static_cast<int64_t>(j) * n_pieces + pc : static_cast<int64_t>(j))
           : mnext;
    s = s_new;
    ++e;
    return true;
  };
  // R19: carry the pending jump time s_at over every piece boundary it
  // reaches: s_at = b + (s_at - b) * (1/rate_next) / (1/rate_now) (infinite
  // when either rate is 0), the grid points up to b count with the piece's
  // d and the boundary point gets the mean of both pieces' d.
  auto carry = [&](T& s_at) {
    if constexpr (PIECES) {
      while (pc + 1 < n_pieces && s_at >= b_next) {
        const Meta mn = load_meta(meta, static_cast<int64_t>(j) * n_pieces + pc + 1);
        const T ir = static_cast<T>(m.inv_rate), irn = static_cast<T>(mn.inv_rate);
        s_at = (isinf(ir) || isinf(irn)) ? P::inf()
                                          : P::fma(P::sub(s_at, b_next), P::div(irn, ir), b_next);
        const int gb = (pc + 1) * g_per;
        const T dlo = static_cast<T>(m.dl);
        const T half = P::mul(P::sub(static_cast<T>(mn.dl), dlo), static_cast<T>(0.5));
        if (COARSE) {
          // gb is even: K divides the coarse grid too
          acc = P::add(P::fma(P::from_int((gb >> 1) - (kprev >> 1)), dlo, acc), half);
          acc_d = P::sub(P::fma(P::from_int(-(kprev & 1)), dlo, acc_d), half);
        } else {
          acc = P::add(P::fma(P::from_int(gb - kprev), dlo, acc), half);
        }
        kprev = gb;
        m = mn;
        ++pc;
        b_next = pc + 1 < n_pieces ? P::mul(P::from_int(pc + 1), inv_pieces) : P::inf();
      }
    }
  };
  // Sample of a walk that ended at s = 1 after e >= 1 jumps, from its
  // exponents: x1 = E_f (l0) or E_c (above), plus the proposal's log-ratio;
  // x2 = E_f - E_c (above l0); js = end state | sign << 31.
  auto sample = [&](T x1, T x2, uint32_t js, T extra) {
    const T vend = static_cast<T>(__ldg(vv + (js & kColMask)));
    T y = COARSE ? P::mul(vend, P::mul(P::ex(x1), P::exm1(x2))) : P::mul(vend, P::ex(x1));
    if (js >> 31) y = -y;
    if (SRC) y = P::add(y, extra);
    if (!isfinite(y)) {
      tot.bad |= kFlagNonFiniteY;
      y = 0;
    }
    acc_y.add(y);
    tot.y2.add_square(y);
    return y;
  };
  // The exponents of the walk that ends at state j (s = 1).
  auto exponents = [&](T& x1, T& x2) {
    const T dle = static_cast<T>(m.dl);
    const T h = P::mul(P::add(dl0, dle), static_cast<T>(0.5));
    if (COARSE) {
      const T acc_c = P::fma(P::from_int(n_coarse - (kprev >> 1)), dle, acc);
      const T accd = P::fma(P::from_int(-(kprev & 1)), dle, acc_d);
      const T ec = P::mul(P::sub(acc_c, h), P::mul(inv_n, static_cast<T>(2)));
      x1 = IS ? P::add(ec, lw) : ec;
      x2 = P::mul(P::add(accd, h), inv_n);
    } else {
      const T acc_f = P::fma(P::from_int(n_grid - kprev), dle, acc);
      const T ef = P::mul(P::sub(acc_f, h), inv_n);
      x1 = IS ? P::add(ef, lw) : ef;
      x2 = 0;
    }
  };
  // The walk ends at state j: at s = 1 after e >= 1 jumps (status 0), or at
  // the jump limit (status 1, sample 0).  A deferred status-0 end (no trace)
  // only records its exponents (ending = true); the samples are evaluated
  // 32 at a time from the warp's end queue.
  bool ending = false;
  T end_x1 = 0, end_x2 = 0;
  auto finish = [&](int status, bool defer) {
    item_jumps += e;
    live = false;
    if (status == 0 && e == 0) {
      // never jumped: counted, its sample y_still is added per item
      ++n_still;
      if (TRACE && TIMES)
        for (int k = 1; k <= n_out; ++k)
          a.trace_times[(row * a.trace_stride + a.trace_base + (r_lo + r)) * n_out + (k - 1)] =
              static_cast<double>(still_time(k));
      if (TRACE) {
        mlmc_walk_record rec;
        rec.end = j;
        rec.jumps = 0;
        rec.sign = 1;
        rec.hash = hash;
        rec.y = static_cast<double>(y_still);
        rec.status = 0;
        rec.pad = 0;
        a.trace[row * a.trace_stride + a.trace_base + (r_lo + r)] = rec;
      }
      return;
    }
    if (status != 0) {
      tot.bad |= (status == 2) ? kFlagBounds : kFlagWalkLimit;
      ++n_limit;
      acc_y.add(static_cast<T>(0));
      tot.y2.add_square(static_cast<T>(0));
    } else if (!TRACE && !SRC && !TIMES && defer) {
      exponents(end_x1, end_x2);
      ending = true;
      return;
    }
    T y = 0;
    if (status == 0) {
      if (TIMES) emit_times(n_grid);
      T x1, x2;
      exponents(x1, x2);
      T extra = 0;
      if (SRC) {
        source_segment(n_grid);
        extra = P::sub(P::mul(src_scale_f, src_f), COARSE ? P::mul(src_scale_c, src_c) : static_cast<T>(0));
      }
      y = sample(x1, x2, static_cast<uint32_t>(j) | (neg << 31), extra);
    }
    if (TRACE) {
      mlmc_walk_record rec;
      rec.end = j;
      rec.jumps = static_cast<int32_t>(e);
      rec.sign = neg ? -1 : 1;
      rec.hash = hash;
      rec.y = static_cast<double>(y);
      rec.status = status;
      rec.pad = 0;
      a.trace[row * a.trace_stride + a.trace_base + (r_lo + r)] = rec;
    }
  };
  // Move this iteration's ended walks into the end queue; evaluate 32
  // samples at once when at least 32 are queued, or all of them at the end
  // of the item (drain).  Called by the whole warp.
  auto settle_ends = [&](bool drain) {
    if (TRACE) return;
    const unsigned em = __ballot_sync(kFull, ending);
    if (ending) {
      const uint32_t slot = (etail + static_cast<uint32_t>(__popc(em & lanes_below))) & (kQueueCap - 1);
      eq->x1[slot] = end_x1;
      eq->x2[slot] = end_x2;
      eq->js[slot] = static_cast<uint32_t>(j) | (neg << 31);
      ending = false;
    }
    etail += static_cast<uint32_t>(__popc(em));
    while (etail - ehead >= 32u || (drain && etail != ehead)) {
      __syncwarp();
      const uint32_t k = ehead + static_cast<uint32_t>(lane);
      if (k < etail) {
        const uint32_t slot = k & (kQueueCap - 1);
        sample(eq->x1[slot], eq->x2[slot], eq->js[slot], static_cast<T>(0));
      }
      ehead = min(ehead + 32u, etail);
      __syncwarp();
    }
  };

  // A walk stopped at the jump limit with its pending jump at time s_at: the
  // output times it passed keep their samples, the final time gets 0.
  auto stop_limit = [&](T s_at, bool defer) {
    if (TIMES) emit_times(P::floor_int(P::mul(s_at, n_fine)));
    finish(1, defer);
  };
  // Record of a walk screened as never jumping (trace only).
  auto trace_still = [&](uint32_t rs) {
    if (TIMES)
      for (int k = 1; k <= n_out; ++k)
        a.trace_times[(row * a.trace_stride + a.trace_base + (r_lo + rs)) * n_out + (k - 1)] =
            static_cast<double>(still_time(k));
    mlmc_walk_record rec;
    rec.end = static_cast<int32_t>(row);
    rec.jumps = 0;
    rec.sign = 1;
    rec.hash = 2166136261u;
    rec.y = static_cast<double>(y_still);
    rec.status = 0;
    rec.pad = 0;
    a.trace[row * a.trace_stride + a.trace_base + (r_lo + rs)] = rec;
  };
  // FP32 screening: the blocks of four walks (groups rep/4) that meet the
  // item's replica range [rep_base, rep_base + span).
  uint64_t gnext = rep_base >> 2;
  const uint64_t g_end = (rep_base + span + 3) >> 2;

  for (;;) {
    if (screened_row) {
      constexpr uint32_t kCap = WarpQueue<FP64>::kCap;
      // Screen first holding times while fewer than 32 walks are queued.
      if constexpr (FP64) {
        // 64 walks per round (two per lane: independent Philox chains that
        // the lane's instructions interleave), each from its own draw 0.
        while (qtail - qhead < 32u && screened < span) {
          uint4 x[kWays];
          T h1[kWays] = {};
          bool push[kWays];
#pragma unroll
          for (int w = 0; w < kWays; ++w) {
            const uint64_t rep = rep_base + screened + static_cast<uint32_t>(32 * w + lane);
            x[w] = keys.draw(make_uint4(static_cast<uint32_t>(rep), row32, 0u,
                                        a.ctr3 | (static_cast<uint32_t>(rep >> 32) << 8)));
          }
#pragma unroll
          for (int w = 0; w < kWays; ++w) {
            const uint32_t rs = screened + static_cast<uint32_t>(32 * w + lane);
            h1[w] = P::mul(P::neglog(P::uniform(x[w])), inv_rate0);
            push[w] = rs < span && h1[w] < static_cast<T>(1);
            if (TRACE && rs < span && !push[w]) trace_still(rs);
            const unsigned pm = __ballot_sync(kFull, push[w]);
            if (push[w]) {
              const uint32_t slot = (qtail + static_cast<uint32_t>(__popc(pm & lanes_below))) & (kCap - 1);
              q->r[slot] = rs;
              q->xz[slot] = x[w].z;
              q->xw[slot] = x[w].w;
              q->first[slot] = h1[w];
            }
            qtail += static_cast<uint32_t>(__popc(pm));
          }
          screened += 32u * kWays;
        }
      } else {
        // 32 blocks of four walks per round: walk rep takes word (rep mod 4)
        // of the block of group rep/4 (draw index 0xFFFFFFFE); the still test
        // is the uniform's index against the row's threshold index.
        while (qtail - qhead < 32u && gnext < g_end) {
          const uint64_t g = gnext + static_cast<uint32_t>(lane);
          uint4 xg = make_uint4(0u, 0u, 0u, 0u);
          if (g < g_end)
            xg = keys.draw(make_uint4(static_cast<uint32_t>(g), row32, 0xFFFFFFFEu,
                                      a.ctr3 | (static_cast<uint32_t>(g >> 32) << 8)));
          // offset of the block's first walk in the item (wraps below 0: the
          // unsigned compare with span rejects it)
          const uint32_t rs0 = 4u * static_cast<uint32_t>(g - (rep_base >> 2)) -
                               static_cast<uint32_t>(rep_base & 3u);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t rs = rs0 + static_cast<uint32_t>(k);
            const bool valid = rs < span;
            const uint32_t word = k == 0 ? xg.x : (k == 1 ? xg.y : (k == 2 ? xg.z : xg.w));
            const bool push = valid && static_cast<int32_t>(word >> 9) > still_max;
            if (TRACE && valid && !push) trace_still(rs);
            const unsigned pm = __ballot_sync(kFull, push);
            if (push) {
              const uint32_t slot = (qtail + static_cast<uint32_t>(__popc(pm & lanes_below))) & (kCap - 1);
              q->r[slot] = rs;
              q->first[slot] = word;
            }
            qtail += static_cast<uint32_t>(__popc(pm));
          }
          gnext += 32u;
        }
      }
      __syncwarp();
      if constexpr (FP64) {
        // Refill wave: lanes without a walk take queued ones and make their
        // first jump.
        const unsigned idle = __ballot_sync(kFull, !live);
        if (!live) {
          const uint32_t k = qhead + static_cast<uint32_t>(__popc(idle & lanes_below));
          if (k < qtail) {
            const uint32_t slot = k & (kCap - 1);
            start_walk(q->r[slot]);
            const T s1 = q->first[slot];  // drawn at screening
            if (static_cast<int64_t>(e) >= a.max_jumps) {
              stop_limit(s1, false);
            } else if (jump(s1, q->xz[slot], q->xw[slot])) {
              live = true;
            } else {
              finish(2, false);
            }
          }
        }
        qhead = min(qhead + static_cast<uint32_t>(__popc(idle)), qtail);
        __syncwarp();  // queue slots read above are free for the next screening
        if (!__any_sync(kFull, live)) break;  // queue empty and every walk screened
        // Draw wave: every live lane draws its next holding time, then jumps
        // or ends (short walks: most lanes end here together, so the sample
        // is evaluated at once).
        if (live) {
          const uint4 x = keys.draw(make_uint4(c_lo, row32, e, c_hi));
          const T s_new = P::add(s, P::mul(P::neglog(P::uniform(x)), static_cast<T>(m.inv_rate)));
          if (!(s_new < static_cast<T>(1))) {
            finish(0, false);
          } else if (static_cast<int64_t>(e) >= a.max_jumps) {
            stop_limit(s_new, false);
          } else if (!jump(s_new, x.z, x.w)) {
            finish(2, false);
          }
        }
      } else {
        // Lanes without a walk take queued ones: the first jump time from
        // the queued word (s = 0, m = m0).
        const unsigned idle = __ballot_sync(kFull, !live);
        if (!live) {
          const uint32_t k = qhead + static_cast<uint32_t>(__popc(idle & lanes_below));
          if (k < qtail) {
            const uint32_t slot = k & (kCap - 1);
            start_walk(q->r[slot]);
            s_pend = P::mul(neglog32(uniform32(q->first[slot])), static_cast<T>(m0.inv_rate));
            carry(s_pend);
            live = true;
          }
        }
        qhead = min(qhead + static_cast<uint32_t>(__popc(idle)), qtail);
        __syncwarp();  // queue slots read above are free for the next screening
        if (!__any_sync(kFull, live)) break;  // queue empty and every walk screened
        // Every live lane takes its pending jump with draw e (words 2, 3)
        // and draws the holding time after it (word 0): one Philox call per
        // jump.  Short walks: most lanes end here together, so the sample
        // is evaluated at once.
        if (live) {
          if (static_cast<int64_t>(e) >= a.max_jumps) {
            stop_limit(s_pend, false);
          } else {
            const uint4 x = keys.draw(make_uint4(c_lo, row32, e, c_hi));
            if (!jump(s_pend, x.z, x.w)) {
              finish(2, false);
            } else {
              s_pend = P::add(s, P::mul(neglog32(uniform32(x.x)), static_cast<T>(m.inv_rate)));
              carry(s_pend);
              if (!(s_pend < static_cast<T>(1))) finish(0, false);
            }
          }
        }
      }
    } else {
      // One wave (rows whose walks are long: no screening): lanes without a
      // walk claim the next unclaimed walks of the item and every live lane
      // makes one event; few lanes end per iteration, so the samples of
      // ended walks go to the end queue.
      const unsigned idle = __ballot_sync(kFull, !live);
      if (!live) {
        const uint32_t k = claimed + static_cast<uint32_t>(__popc(idle & lanes_below));
        if (k < span) {
          start_walk(k);
          live = true;
          fresh = true;
        }
      }
      claimed = min(claimed + static_cast<uint32_t>(__popc(idle)), span);
      if (!__any_sync(kFull, live)) break;  // every walk of the item done
      if (live) {
        const uint4 x = keys.draw(make_uint4(c_lo, row32, e, c_hi));
        if constexpr (FP64) {
          T s_new = P::add(s, P::mul(P::neglog(P::uniform(x)), static_cast<T>(m.inv_rate)));
          carry(s_new);
          if (!(s_new < static_cast<T>(1))) {
            finish(0, true);
          } else if (static_cast<int64_t>(e) >= a.max_jumps) {
            stop_limit(s_new, true);
          } else if (!jump(s_new, x.z, x.w)) {
            finish(2, true);
          }
        } else {
          // Up to kLongEvents jumps per lane per iteration: the claim, the
          // end bookkeeping and the warp votes around them are paid once for
          // both.  Draw e gives the pending jump (words 2, 3) and the holding
          // time after it (word 0); a fresh walk first takes its first
          // holding time from word 1 (rows with 1/(tL) < 1: no shared block
          // word).  One end site: status -1 while the walk goes on.
          // (one per iteration with a source term or output times: their
          // per-segment sums need the registers)
          constexpr int kEvents = (SRC || TIMES) ? 1 : kLongEvents;
          int status = -1;
          for (int k = 0; k < kEvents; ++k) {
            const uint4 xk = k == 0 ? x : keys.draw(make_uint4(c_lo, row32, e, c_hi));
            if (fresh) {
              s_pend = P::add(s, P::mul(neglog32(uniform32(xk.y)), static_cast<T>(m.inv_rate)));
              carry(s_pend);
              fresh = false;
            }
            if (!(s_pend < static_cast<T>(1))) {
              status = 0;  // never jumped
              break;
            }
            if (static_cast<int64_t>(e) >= a.max_jumps) {
              status = 1;
              break;
            }
            if (!jump(s_pend, xk.z, xk.w)) {
              status = 2;
              break;
            }
            s_pend = P::add(s, P::mul(neglog32(uniform32(xk.x)), static_cast<T>(m.inv_rate)));
            carry(s_pend);
            if (!(s_pend < static_cast<T>(1))) {
              status = 0;
              break;
            }
          }
          if (status == 1) {
            stop_limit(s_pend, true);
          } else if (status >= 0) {
            finish(status, true);
          }
        }
      }
      settle_ends(false);
    }
  }
  settle_ends(true);
  double ys = warp_sum(acc_y);
  const unsigned long long jumps = warp_sum_u64(item_jumps);
  // Screened rows: every screened walk that was not queued never jumps
  // (qtail counts the queued ones); other rows count them as they end.
  const unsigned long long still =
      warp_sum_u64(n_still) + (screened_row ? static_cast<unsigned long long>(span - qtail) : 0ull);
  const unsigned long long limit = warp_sum_u64(n_limit);
  // Walks that never jump: y_still each (0 above l0 unless a source term
  // adds its fixed Simpson part).
  const double yc = static_cast<double>(y_still);
  if (!COARSE || SRC) ys += static_cast<double>(still) * yc;
  if (lane == 0) {
    wc->walks += static_cast<unsigned long long>(r_hi - r_lo);
    wc->jumps += jumps;
    wc->still += still;
    wc->limit += limit;
    if (!COARSE || SRC) wc->y2_fixed += static_cast<double>(still) * (yc * yc);
  }
  if (lane == 0 && ys != 0.0) atomicAdd(a.sum_y + row, ys);
  if constexpr (TIMES) {
    // per output time: the lanes' sums plus the walks that never jumped
    for (int k = 1; k <= n_out; ++k) {
      double yk = static_cast<double>(ta->v[k - 1][lane]);
      ta->v[k - 1][lane] = 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) yk += __shfl_xor_sync(kFull, yk, o);
      if (!COARSE) yk += static_cast<double>(still) * static_cast<double>(still_time(k));
      if (lane == 0 && yk != 0.0) atomicAdd(a.sum_times + static_cast<int64_t>(k - 1) * a.n + row, yk);
    }
  }
}

template <bool FP64, bool COARSE, bool TRACE, bool IS, bool SRC = false, bool TIMES = false,
          bool PIECES = false>
__global__ void __launch_bounds__(256, FP64 ? 3 : 4) k_walk(const __grid_constant__ WalkArgs a) {
  using T = typename Prec<FP64>::T;
  const int lane = threadIdx.x & 31;
  ItemArgs ia;
  ia.meta = a.meta;
  ia.alias = a.alias;
  ia.v_walk = a.v_walk;
  ia.level = a.level;
  ia.ctr3 = a.ctr3;
  ia.key0 = a.key0;
  ia.key1 = a.key1;
  ia.max_jumps = a.max_jumps;
  ia.sum_y = a.sum_y;
  ia.rep_begin = a.rep_begin;
  ia.trace = a.trace;
  ia.trace_stride = a.trace_stride;
  ia.trace_base = a.trace_base;
  ia.f_walk = a.f_walk;
  ia.t = a.t;
  ia.n = a.n;
  ia.nnz = a.nnz;
  ia.still32 = a.still32;
  ia.pieces = a.pieces;
  ia.n_times = a.n_times;
  ia.sum_times = a.sum_times;
  ia.trace_times = a.trace_times;
  __shared__ WarpQueue<FP64> queues[kMaxWarps];
  __shared__ WarpCounters counters[kMaxWarps];
  __shared__ EndQueue<FP64> ends[kMaxWarps];
  __shared__ TimesAcc<FP64, TIMES> tacc[TIMES ? kMaxWarps : 1];
  WarpQueue<FP64>* q = &queues[threadIdx.x >> 5];
  EndQueue<FP64>* eq = &ends[threadIdx.x >> 5];
  WarpCounters* wc = &counters[threadIdx.x >> 5];
  TimesAcc<FP64, TIMES>* ta = &tacc[TIMES ? (threadIdx.x >> 5) : 0];
  if (lane == 0) *wc = WarpCounters{};
  if constexpr (TIMES) {
    constexpr int kOut = (FP64 ? kMaxTimes64 : kMaxTimes32) - 1;
    for (int k = 0; k < kOut; ++k) ta->v[k][lane] = 0;
  }
  __syncwarp();
  LaneTotals<T> tot;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.work, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= a.total_items) break;
    const int64_t rel = static_cast<int64_t>(item / static_cast<unsigned long long>(a.chunks_per_row));
    const int64_t chunk = static_cast<int64_t>(item) - rel * a.chunks_per_row;
    const int64_t r_lo = chunk * a.chunk;
    const int64_t r_hi = min(r_lo + a.chunk, a.reps);
    walk_item<FP64, COARSE, TRACE, IS, KeysFromParam, SRC, TIMES, PIECES>(ia, KeysFromParam{&a.rk},
                                                                       a.row_begin + rel, r_lo,
                                                                       r_hi, tot, wc, q, eq, ta,
                                                                       lane);
  }
  flush_warp(tot, wc, a.totals, a.flags, lane);
}

// ---------------------------------------------------------------------------
// Batched rounds: one persistent launch walks every segment of a round.  A
// warp takes the next global work item, finds its segment (binary search of
// the segments' first items), and runs the same walk_item as the single-plan
// kernel with the segment's tables, right-hand side and Philox round keys
// (copied to shared memory when the warp changes segment); its totals go to
// the segment's (problem, level) after every item.
// ---------------------------------------------------------------------------
// Round keys of the segment a warp is walking, interleaved (k0, k1) per
// round so that each Philox round reads its pair with one shared load.
struct SharedRoundKeys {
  uint2 k[10];
};
struct KeysFromShared {
  const SharedRoundKeys* rk;  // in shared memory
  __device__ __forceinline__ uint4 draw(uint4 c) const {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      const uint2 kr = rk->k[r];
      const unsigned long long p0 = static_cast<unsigned long long>(kPhiloxM0) * c.x;
      const unsigned long long p1 = static_cast<unsigned long long>(kPhiloxM1) * c.z;
      c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ kr.x, static_cast<uint32_t>(p1),
                     static_cast<uint32_t>(p0 >> 32) ^ c.w ^ kr.y, static_cast<uint32_t>(p0));
    }
    return c;
  }
};

template <bool FP64>
__global__ void __launch_bounds__(256, FP64 ? 3 : 4)
    k_walk_batch(const BatchRound* __restrict__ round, const BatchSeg* __restrict__ segs,
                 unsigned long long* __restrict__ work, uint32_t* __restrict__ flags) {
  using T = typename Prec<FP64>::T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  __shared__ WarpQueue<FP64> queues[kMaxWarps];
  __shared__ WarpCounters counters[kMaxWarps];
  __shared__ EndQueue<FP64> ends[kMaxWarps];
  __shared__ SharedRoundKeys keys[kMaxWarps];
  WarpQueue<FP64>* q = &queues[warp];
  EndQueue<FP64>* eq = &ends[warp];
  WarpCounters* wc = &counters[warp];
  if (lane == 0) *wc = WarpCounters{};
  __syncwarp();
  const unsigned long long total = round->total_items;
  const int nseg = round->nseg;
  LaneTotals<T> tot;
  int loaded = -1;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(work, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    // the last segment whose first item is <= item
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    const BatchSeg& sg = segs[lo];
    if (lo != loaded) {
      __syncwarp();  // the previous item's draws are done with the keys
      if (lane < 10) keys[warp].k[lane] = make_uint2(sg.rk.k0[lane], sg.rk.k1[lane]);
      __syncwarp();
      loaded = lo;
    }
    ItemArgs ia;
    ia.meta = sg.meta;
    ia.alias = sg.alias;
    ia.v_walk = sg.v_walk;
    ia.level = sg.level;
    ia.ctr3 = sg.ctr3;
    ia.key0 = sg.rk.k0[0];
    ia.key1 = sg.rk.k1[0];
    ia.max_jumps = sg.max_jumps;
    ia.sum_y = sg.sum_y;
    ia.rep_begin = sg.rep_begin;
    ia.trace = nullptr;
    ia.trace_stride = 0;
    ia.trace_base = 0;
    ia.f_walk = nullptr;
    ia.t = 0.0;
    ia.n = sg.n;
    ia.nnz = sg.nnz;
    ia.still32 = sg.still32;
    ia.pieces = 1;
    ia.n_times = 0;
    ia.sum_times = nullptr;
    ia.trace_times = nullptr;
    const unsigned long long local = item - sg.item_begin;
    const int64_t row = static_cast<int64_t>(local / static_cast<unsigned long long>(sg.chunks_per_row));
    const int64_t chunk = static_cast<int64_t>(local) - row * sg.chunks_per_row;
    const int64_t r_lo = chunk * sg.chunk;
    const int64_t r_hi = min(r_lo + sg.chunk, sg.reps);
    const KeysFromShared kk{&keys[warp]};
    TimesAcc<FP64, false>* ta = nullptr;
    if (sg.is) {
      if (sg.coarse)
        walk_item<FP64, true, false, true, KeysFromShared>(ia, kk, row, r_lo, r_hi, tot, wc, q, eq, ta, lane);
      else
        walk_item<FP64, false, false, true, KeysFromShared>(ia, kk, row, r_lo, r_hi, tot, wc, q, eq, ta, lane);
    } else {
      if (sg.coarse)
        walk_item<FP64, true, false, false, KeysFromShared>(ia, kk, row, r_lo, r_hi, tot, wc, q, eq, ta, lane);
      else
        walk_item<FP64, false, false, false, KeysFromShared>(ia, kk, row, r_lo, r_hi, tot, wc, q, eq, ta, lane);
    }
    flush_warp(tot, wc, sg.totals, flags, lane);
  }
}

// ---------------------------------------------------------------------------
// Forward mode (Eq. 5): walk g starts at s ~ w_s / W (integer weights, see
// mlmc_forward.cu), runs on the tables of B = A^T, and adds
// y = (v_s W / w_s) sign e^{E} (level l0) or ... e^{E_c} expm1(E_f - E_c)
// (above l0) to x[end].  Counter words: (g bits 0-31, g bits 32-63, draw
// index, level | 1 << 6); the start draw uses draw index 0xFFFFFFFF.  Lanes
// that end in the same iteration on the same state add their values with
// one atomic (match_any + shuffles).
// ---------------------------------------------------------------------------
struct FwdArgs {
  const void* meta;
  const void* alias;
  const double* v;              // right-hand side (start weights use FP64 v)
  const int64_t* cdf;           // inclusive prefix sums of the integer weights
  const int32_t* guide;         // guide table (cutpoints) over cdf
  int64_t nnz;                  // alias entries (checked build)
  const int64_t* w;             // integer weights
  int64_t n;
  unsigned long long W;         // cdf[n-1]
  int64_t walk_begin;
  int64_t walks;
  int64_t chunk;
  unsigned long long total_items;
  int level;
  uint32_t ctr3;                // level | 1 << 6
  uint32_t key0, key1;
  PhiloxRoundKeys rk;           // round keys of (key0, key1)
  int64_t max_jumps;
  double* sum_x;
  double* totals;
  uint32_t* flags;
  unsigned long long* work;
  mlmc_walk_record* trace;      // index g - walk_begin
};

template <bool FP64, bool COARSE, bool TRACE, bool IS>
__global__ void __launch_bounds__(256, FP64 ? 3 : 4) k_walk_fwd(const __grid_constant__ FwdArgs a) {
  using P = Prec<FP64>;
  using T = typename P::T;
  using Meta = typename P::Meta;
  const Meta* __restrict__ meta = static_cast<const Meta*>(a.meta);
  const int lane = threadIdx.x & 31;
  const int n_grid = 1 << a.level;
  const T n_fine = P::from_int(n_grid);
  const T inv_n = static_cast<T>(1.0 / n_grid);
  const int n_coarse = n_grid >> 1;
  WalkTotals<T> tot;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.work, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= a.total_items) break;
    const int64_t w_lo = static_cast<int64_t>(item) * a.chunk;
    const uint32_t span = static_cast<uint32_t>(min(a.chunk, a.walks - w_lo));
    if (lane == 0) tot.walks += span;
    uint32_t next = 32;
    uint32_t r = static_cast<uint32_t>(lane);
    bool live = r < span;
    Kahan<T> acc_unused;
    uint32_t item_jumps = 0;
    // Walk state.
    uint64_t g = 0;
    Meta m{};
    int32_t j = 0;
    T dl0 = 0, f = 0;
    uint32_t e = 0, neg = 0;
    T s = 0, acc = 0, acc_d = 0, lw = 0;
    int kprev = -1;
    int32_t start = 0;
    uint32_t hash = 2166136261u;
    // FP32: the next jump time, drawn with the previous jump (word 0) or,
    // for a fresh walk, from word 1 of draw 0.
    T s_pend = 0;
    bool fresh = false;
    auto begin_walk = [&]() {
      g = static_cast<uint64_t>(a.walk_begin + w_lo + r);
      const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(g), static_cast<uint32_t>(g >> 32),
                                               0xFFFFFFFFu, a.ctr3),
                                    a.rk);
      const unsigned long long u = (static_cast<unsigned long long>(x.x) << 32) | x.y;
      const unsigned long long rr = __umul64hi(u, a.W);
      // smallest index with cdf > rr: from the guide table's cutpoint for
      // bucket floor(u n / 2^64), scanning forward
      int64_t k = __ldg(a.guide + __umul64hi(u, static_cast<unsigned long long>(a.n)));
      while (static_cast<unsigned long long>(__ldg(a.cdf + k)) <= rr) ++k;
      start = static_cast<int32_t>(k);
      j = start;
      m = load_meta(meta, j);
      dl0 = static_cast<T>(m.dl);
      const double fd = __ldg(a.v + j) * (static_cast<double>(a.W) / static_cast<double>(__ldg(a.w + j)));
      f = static_cast<T>(fd);
      e = 0;
      neg = 0;
      s = 0;
      acc = 0;
      acc_d = 0;
      lw = 0;
      kprev = -1;
      hash = 2166136261u;
      fresh = true;
    };
    if (live) begin_walk();
    while (__any_sync(kFull, live)) {
      bool fin = false;
      T y = 0;
      if (live) {
        const uint4 x = philox4x32_10(
            make_uint4(static_cast<uint32_t>(g), static_cast<uint32_t>(g >> 32), e, a.ctr3), a.rk);
        T s_new;
        if constexpr (FP64) {
          // draw e: the holding time (words 0, 1) and the jump after it
          s_new = P::add(s, P::mul(P::neglog(P::uniform(x)), static_cast<T>(m.inv_rate)));
        } else {
          // draw e: the pending jump (words 2, 3) and the holding time after
          // it (word 0); a fresh walk's first holding time is word 1
          if (fresh) {
            s_pend = P::add(s, P::mul(neglog32(uniform32(x.y)), static_cast<T>(m.inv_rate)));
            fresh = false;
          }
          s_new = s_pend;
        }
        bool done = !(s_new < static_cast<T>(1));
        int status = 0;
        if (!done && static_cast<int64_t>(e) >= a.max_jumps) {
          done = true;
          status = 1;
        }
        if (kChecked && !done) {
          // the alias entry and the state it picks must lie inside the tables
          const uint32_t bk = __umulhi(x.z, static_cast<uint32_t>(m.deg));
          if (m.start < 0 || static_cast<int64_t>(m.start) + bk >= a.nnz) {
            done = true;
            status = 2;
          } else {
            using Fused = typename std::conditional<FP64, FusedEntry64, FusedEntry32>::type;
            const uint4 ent = IS ? __ldg(reinterpret_cast<const uint4*>(
                                       static_cast<const AliasEntryIS*>(a.alias) + m.start + bk))
                                 : __ldg(reinterpret_cast<const uint4*>(
                                       static_cast<const Fused*>(a.alias) + m.start + bk));
            const uint32_t pk = (x.w < ent.x) ? ent.y : ent.z;
            if (static_cast<int64_t>(pk & kColMask) >= a.n) {
              done = true;
              status = 2;
            }
          }
        }
        if (!done) {
          const int gi = P::floor_int(P::mul(s_new, n_fine));
          const T dlj = static_cast<T>(m.dl);
          if (COARSE) {
            const int kc_prev = kprev >> 1;
            acc = P::fma(P::from_int((gi >> 1) - kc_prev), dlj, acc);
            acc_d = P::fma(P::from_int((gi & 1) - (kprev & 1)), dlj, acc_d);
          } else {
            acc = P::fma(P::from_int(gi - kprev), dlj, acc);
          }
          kprev = gi;
          const uint32_t bucket = __umulhi(x.z, static_cast<uint32_t>(m.deg));
          uint32_t pick;
          Meta mnext{};
          if (IS) {
            const uint4* ep = reinterpret_cast<const uint4*>(
                static_cast<const AliasEntryIS*>(a.alias) + m.start + bucket);
            const uint4 e0 = __ldg(ep);
            const uint2 e1 = __ldg(reinterpret_cast<const uint2*>(ep + 1));
            const bool keep = x.w < e0.x;
            pick = keep ? e0.y : e0.z;
            lw = P::add(lw, static_cast<T>(__uint_as_float(keep ? e1.x : e1.y)));
          } else {
            using Fused = typename std::conditional<FP64, FusedEntry64, FusedEntry32>::type;
            const Fused* fe = static_cast<const Fused*>(a.alias) + m.start + bucket;
            const uint4 ent = __ldg(reinterpret_cast<const uint4*>(fe));
            const Meta mk = load_meta(&fe->mk, 0);
            const Meta ma = load_meta(&fe->ma, 0);
            const bool keep = x.w < ent.x;
            pick = keep ? ent.y : ent.z;
            mnext = keep ? mk : ma;
          }
          neg ^= pick >> 31;
          j = static_cast<int32_t>(pick & kColMask);
          if (TRACE) hash = (hash ^ static_cast<uint32_t>(j)) * 16777619u;
          m = IS ? load_meta(meta, j) : mnext;
          s = s_new;
          ++e;
          if constexpr (!FP64) {
            s_pend = P::add(s, P::mul(neglog32(uniform32(x.x)), static_cast<T>(m.inv_rate)));
            done = !(s_pend < static_cast<T>(1));
          }
        }
        if (done) {
          fin = true;
          if (status == 0) {
            const T dle = static_cast<T>(m.dl);
            const T h = P::mul(P::add(dl0, dle), static_cast<T>(0.5));
            if (COARSE) {
              if (e != 0) {
                const T acc_c = P::fma(P::from_int(n_coarse - (kprev >> 1)), dle, acc);
                const T accd = P::fma(P::from_int(-(kprev & 1)), dle, acc_d);
                const T ec = P::mul(P::sub(acc_c, h), P::mul(inv_n, static_cast<T>(2)));
                const T diff = P::mul(P::add(accd, h), inv_n);
                y = P::mul(f, P::mul(P::ex(IS ? P::add(ec, lw) : ec), P::exm1(diff)));
              }
            } else {
              const T acc_f = P::fma(P::from_int(n_grid - kprev), dle, acc);
              const T ef = P::mul(P::sub(acc_f, h), inv_n);
              y = P::mul(f, P::ex(IS ? P::add(ef, lw) : ef));
            }
            if (neg) y = -y;
            if (!isfinite(y)) {
              tot.bad |= kFlagNonFiniteY;
              y = 0;
            }
          } else {
            tot.bad |= (status == 2) ? kFlagBounds : kFlagWalkLimit;
            ++tot.limit;
          }
          if (e == 0) ++tot.still;
          tot.y2.add_square(y);
          item_jumps += e;
          if (TRACE) {
            mlmc_walk_record rec;
            rec.end = j;
            rec.jumps = static_cast<int32_t>(e);
            rec.sign = neg ? -1 : 1;
            rec.hash = hash;
            rec.y = static_cast<double>(y);
            rec.status = status;
            rec.pad = start;
            a.trace[g - a.walk_begin] = rec;
          }
        }
      }
      const unsigned fmask = __ballot_sync(kFull, fin);
      if (fin) {
        // Add y to x[end], one atomic per distinct end state of the warp.
        const unsigned peers = __match_any_sync(fmask, j);
        double total = 0.0;
        for (unsigned mm = peers; mm; mm &= mm - 1) {
          const int src = __ffs(mm) - 1;
          total += __shfl_sync(peers, static_cast<double>(y), src);
        }
        if (lane == __ffs(peers) - 1 && total != 0.0) atomicAdd(a.sum_x + j, total);
        r = next + static_cast<uint32_t>(__popc(fmask & ((1u << lane) - 1u)));
        live = r < span;
        if (live) begin_walk();
      }
      next += static_cast<uint32_t>(__popc(fmask));
    }
    tot.jumps += item_jumps;
    (void)acc_unused;
  }
  flush_totals(tot, a.totals, a.flags, lane);
}

__global__ void k_to_float(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}

cudaError_t launch_to_float(mlmc_plan* p, const double* in, float* out) {
  const int64_t want = (p->n + 255) / 256;
  const int grid = static_cast<int>(want < p->num_sms * 8 ? want : p->num_sms * 8);
  k_to_float<<<grid, 256, 0, p->stream>>>(p->n, in, out);
  p->launches++;
  return cudaGetLastError();
}

template <bool FP64, bool COARSE, bool TRACE, bool IS, bool SRC, bool TIMES = false,
          bool PIECES = false>
cudaError_t launch_one(mlmc_plan* p, const WalkArgs& args, int block, cudaStream_t stream) {
  auto kern = k_walk<FP64, COARSE, TRACE, IS, SRC, TIMES, PIECES>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
  if (err != cudaSuccess) return err;
  const unsigned long long warps_needed = args.total_items;
  const int warps_per_block = block / 32;
  unsigned long long grid = static_cast<unsigned long long>(p->num_sms) * (per_sm > 0 ? per_sm : 1);
  const unsigned long long need = (warps_needed + warps_per_block - 1) / warps_per_block;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  // The tables this walk reads, through the plan's L2 access-policy window.
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(block));
  cfg.stream = stream;
  cfg.attrs = attr;
  if (IS)
    cfg.numAttrs = l2_window_attr(p, p->d_alias_is, is_window_bytes(p, FP64), attr);
  else
    cfg.numAttrs = FP64 ? l2_window_attr(p, p->l2_base64, p->l2_bytes64, attr)
                        : l2_window_attr(p, p->l2_base32, p->l2_bytes32, attr);
  err = cudaLaunchKernelEx(&cfg, kern, args);
  p->launches++;
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

// Proposal and source term are exclusive (checked when either is set), and
// so are the source term and intermediate times.
template <bool FP64, bool COARSE, bool TRACE>
cudaError_t dispatch_is(mlmc_plan* p, const WalkArgs& a, int block, bool is, bool src,
                        cudaStream_t st) {
  if (src) return launch_one<FP64, COARSE, TRACE, false, true>(p, a, block, st);
  if (a.n_times > 1)
    return is ? launch_one<FP64, COARSE, TRACE, true, false, true>(p, a, block, st)
              : launch_one<FP64, COARSE, TRACE, false, false, true>(p, a, block, st);
  if (is && a.pieces > 1) return launch_one<FP64, COARSE, TRACE, true, false, false, true>(p, a, block, st);
  return is ? launch_one<FP64, COARSE, TRACE, true, false>(p, a, block, st)
            : launch_one<FP64, COARSE, TRACE, false, false>(p, a, block, st);
}

cudaError_t dispatch_walk(mlmc_plan* p, const WalkArgs& a, int block, bool fp64, bool coarse,
                          bool trace, bool is, bool src, cudaStream_t st) {
  if (fp64) {
    if (coarse) return trace ? dispatch_is<true, true, true>(p, a, block, is, src, st) : dispatch_is<true, true, false>(p, a, block, is, src, st);
    return trace ? dispatch_is<true, false, true>(p, a, block, is, src, st) : dispatch_is<true, false, false>(p, a, block, is, src, st);
  }
  if (coarse) return trace ? dispatch_is<false, true, true>(p, a, block, is, src, st) : dispatch_is<false, true, false>(p, a, block, is, src, st);
  return trace ? dispatch_is<false, false, true>(p, a, block, is, src, st) : dispatch_is<false, false, false>(p, a, block, is, src, st);
}

template <bool FP64, bool COARSE, bool TRACE, bool IS>
cudaError_t launch_fwd_one(mlmc_plan* p, const FwdArgs& args, int block) {
  auto kern = k_walk_fwd<FP64, COARSE, TRACE, IS>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
  if (err != cudaSuccess) return err;
  unsigned long long grid = static_cast<unsigned long long>(p->num_sms) * (per_sm > 0 ? per_sm : 1);
  const unsigned long long need = (args.total_items + block / 32 - 1) / (block / 32);
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(block));
  cfg.stream = p->stream;
  cfg.attrs = attr;
  if (IS)
    cfg.numAttrs = l2_window_attr(p, p->d_alias_is, is_window_bytes(p, FP64), attr);
  else
    cfg.numAttrs = FP64 ? l2_window_attr(p, p->l2_base64, p->l2_bytes64, attr)
                        : l2_window_attr(p, p->l2_base32, p->l2_bytes32, attr);
  err = cudaLaunchKernelEx(&cfg, kern, args);
  if (err != cudaSuccess) return err;
  p->launches++;
  return cudaGetLastError();
}

template <bool FP64, bool COARSE, bool TRACE>
cudaError_t fwd_is(mlmc_plan* p, const FwdArgs& a, int block, bool is) {
  return is ? launch_fwd_one<FP64, COARSE, TRACE, true>(p, a, block)
            : launch_fwd_one<FP64, COARSE, TRACE, false>(p, a, block);
}

cudaError_t dispatch_fwd(mlmc_plan* p, const FwdArgs& a, int block, bool fp64, bool coarse,
                         bool trace, bool is) {
  if (fp64) {
    if (coarse) return trace ? fwd_is<true, true, true>(p, a, block, is) : fwd_is<true, true, false>(p, a, block, is);
    return trace ? fwd_is<true, false, true>(p, a, block, is) : fwd_is<true, false, false>(p, a, block, is);
  }
  if (coarse) return trace ? fwd_is<false, true, true>(p, a, block, is) : fwd_is<false, true, false>(p, a, block, is);
  return trace ? fwd_is<false, false, true>(p, a, block, is) : fwd_is<false, false, false>(p, a, block, is);
}

}  // namespace

// Forward-mode walks: w.rep_begin = first walk index, w.reps = walks; the
// start table (cdf, weights, W) must be current for w.v (launch_start_table).
cudaError_t launch_walk_forward(mlmc_plan* p, const WalkLaunch& w, int64_t* launches) {
  if (launches) *launches = 0;
  // v = 0 (W = 0): every sample is 0 and no walk is made
  if (w.reps <= 0 || p->n <= 0 || p->start_total == 0) return cudaSuccess;
  const bool fp64 = p->sched.precision == MLMC_FP64;
  FwdArgs a{};
  a.meta = walk_meta(p, fp64);
  a.alias = p->proposal_active ? static_cast<const void*>(p->d_alias_is)
                               : static_cast<const void*>(p->d_fused);
  a.v = w.v;
  a.cdf = p->d_cdf;
  a.guide = p->d_guide;
  a.nnz = p->nnz;
  a.w = p->d_wstart;
  a.n = p->n;
  a.W = p->start_total;
  a.level = w.level;
  a.ctr3 = (static_cast<uint32_t>(w.level) & 0x3Fu) | (1u << 6);
  a.key0 = static_cast<uint32_t>(w.seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(w.seed >> 32);
  a.rk = philox_round_keys(a.key0, a.key1);
  a.max_jumps = p->sched.max_jumps_per_walk;
  a.sum_x = w.sum_y;
  a.totals = w.totals;
  a.flags = p->d_flags;
  a.work = p->d_work;
  a.trace = w.trace;
  const int block = p->sched.block_threads > 0 ? p->sched.block_threads : 256;
  const int64_t per_lane = p->sched.walks_per_lane > 0 ? p->sched.walks_per_lane : 64;
  a.chunk = 32 * per_lane;
  const int64_t cap = p->sched.launch_reps > 0 ? p->sched.launch_reps : int64_t{1} << 31;
  for (int64_t done = 0; done < w.reps; done += cap) {
    const int64_t walks = std::min(cap, w.reps - done);
    a.walk_begin = w.rep_begin + done;
    a.walks = walks;
    a.total_items = static_cast<unsigned long long>((walks + a.chunk - 1) / a.chunk);
    if (w.trace) a.trace = w.trace + done;
    cudaError_t err = cudaMemsetAsync(p->d_work, 0, sizeof(unsigned long long), p->stream);
    if (err != cudaSuccess) return err;
    err = dispatch_fwd(p, a, block, fp64, w.coarse, w.trace != nullptr, p->proposal_active);
    if (err != cudaSuccess) return err;
    if (launches) ++*launches;
  }
  return cudaSuccess;
}

namespace {

// The launches of one walk request on `stream`: bounded launches of about
// 2^31 walks (tens of milliseconds each: the controller checks its time
// budget between them and no kernel runs for seconds), each after resetting
// the work counter `work`.  v_walk / f_walk: right-hand side and source in
// the walk precision; per_lane_fixed > 0 fixes the walks per lane of an item.
cudaError_t launch_walk_core(mlmc_plan* p, const WalkLaunch& w, const void* v_walk,
                             const void* f_walk, unsigned long long* work, uint32_t* flags,
                             int64_t per_lane_fixed, cudaStream_t stream, int64_t* launches) {
  const bool fp64 = p->sched.precision == MLMC_FP64;
  WalkArgs a{};
  a.meta = walk_meta(p, fp64);
  a.alias = p->proposal_active ? static_cast<const void*>(p->d_alias_is)
                               : static_cast<const void*>(p->d_fused);
  a.v_walk = v_walk;
  a.still32 = walk_still32(p);
  a.pieces = p->proposal_active ? p->pieces : 1;
  const bool src = f_walk != nullptr;
  if (src) {
    a.f_walk = f_walk;
    a.t = p->t;
  }
  a.n = p->n;
  a.nnz = p->nnz;
  a.level = w.level;
  a.ctr3 = static_cast<uint32_t>(w.level) & 0x3Fu;
  a.key0 = static_cast<uint32_t>(w.seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(w.seed >> 32);
  a.rk = philox_round_keys(a.key0, a.key1);
  a.max_jumps = p->sched.max_jumps_per_walk;
  a.sum_y = w.sum_y;
  a.totals = w.totals;
  a.flags = flags;
  a.work = work;
  a.trace = w.trace;
  a.trace_stride = w.reps;
  a.n_times = w.n_times > 1 ? w.n_times : 0;
  a.sum_times = w.sum_times;
  a.trace_times = w.trace_times;
  const int block = p->sched.block_threads > 0 ? p->sched.block_threads : 256;
  const bool trace = w.trace != nullptr;
  const int64_t cap = p->sched.launch_reps > 0 ? p->sched.launch_reps
                                               : std::max<int64_t>(32, (int64_t{1} << 31) / p->n);
  for (int64_t done = 0; done < w.reps; done += cap) {
    const int64_t reps = std::min(cap, w.reps - done);
    a.rep_begin = w.rep_begin + done;
    a.reps = reps;
    a.trace_base = done;
    int64_t per_lane = per_lane_fixed;
    if (per_lane <= 0) {
      // Enough walks per item to amortise the item fetch and each item's
      // tail (its last iterations on few lanes): up to 256 per lane, which
      // measured 1.4-2.8% faster than 128 on launches of 21504 walks per row
      // and still leaves every warp dozens of items per launch.
      per_lane = (reps + 31) / 32;
      if (per_lane > 256) per_lane = 256;
    }
    a.chunk = 32 * per_lane;
    a.chunks_per_row = (reps + a.chunk - 1) / a.chunk;
    a.row_begin = w.row_count < 0 ? 0 : w.row_begin;
    a.total_items = static_cast<unsigned long long>(w.row_count < 0 ? p->n : w.row_count) *
                    static_cast<unsigned long long>(a.chunks_per_row);
    cudaError_t err = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (err != cudaSuccess) return err;
    err = dispatch_walk(p, a, block, fp64, w.coarse, trace, p->proposal_active, src, stream);
    if (err != cudaSuccess) return err;
    if (launches) ++*launches;
  }
  return cudaSuccess;
}

// The source term in the walk precision (FP32 walks: converted into the
// plan's buffer), or null without one.
cudaError_t source_for_walk(mlmc_plan* p, const WalkLaunch& w, const void** f_walk) {
  *f_walk = nullptr;
  if (!p->source_active) return cudaSuccess;
  if (w.level < 1 || (w.coarse && w.level < 2)) return cudaErrorInvalidValue;
  if (p->sched.precision == MLMC_FP64) {
    *f_walk = p->d_src;
    return cudaSuccess;
  }
  cudaError_t err = launch_to_float(p, p->d_src, p->d_src32);
  *f_walk = p->d_src32;
  return err;
}

}  // namespace

cudaError_t launch_walk(mlmc_plan* p, const WalkLaunch& w, int64_t* launches) {
  if (launches) *launches = 0;
  if (w.reps <= 0 || p->n <= 0) return cudaSuccess;
  const void* v_walk = w.v;
  if (p->sched.precision != MLMC_FP64) {
    cudaError_t err = launch_to_float(p, w.v, p->d_v32);
    if (err != cudaSuccess) return err;
    v_walk = p->d_v32;
  }
  const void* f_walk = nullptr;
  cudaError_t err = source_for_walk(p, w, &f_walk);
  if (err != cudaSuccess) return err;
  return launch_walk_core(p, w, v_walk, f_walk, p->d_work, p->d_flags, p->sched.walks_per_lane,
                          p->stream, launches);
}

// The same launch sequence as launch_walk, with the work counter and the FP32
// copy of v taken from caller-supplied device memory instead of the plan's
// buffers (used by the entry point whose scratch is static device memory).
cudaError_t launch_walk_scratch(mlmc_plan* p, const WalkLaunch& w, unsigned long long* work,
                                float* v32, int64_t* launches) {
  if (launches) *launches = 0;
  if (w.reps <= 0 || p->n <= 0) return cudaSuccess;
  const void* v_walk = w.v;
  if (p->sched.precision != MLMC_FP64) {
    cudaError_t err = launch_to_float(p, w.v, v32);
    if (err != cudaSuccess) return err;
    v_walk = v32;
  }
  const void* f_walk = nullptr;
  cudaError_t err = source_for_walk(p, w, &f_walk);
  if (err != cudaSuccess) return err;
  return launch_walk_core(p, w, v_walk, f_walk, work, p->d_flags, p->sched.walks_per_lane,
                          p->stream, launches);
}

cudaError_t launch_walk_batch(bool fp64, const BatchRound* round, const BatchSeg* segs,
                              unsigned long long* work, uint32_t* flags, int num_sms, int block,
                              cudaStream_t stream) {
  int per_sm = 0;
  cudaError_t err = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_batch<true>, block, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_batch<false>, block, 0);
  if (err != cudaSuccess) return err;
  const unsigned grid = static_cast<unsigned>(num_sms * (per_sm > 0 ? per_sm : 1));
  if (fp64)
    k_walk_batch<true><<<grid, block, 0, stream>>>(round, segs, work, flags);
  else
    k_walk_batch<false><<<grid, block, 0, stream>>>(round, segs, work, flags);
  return cudaGetLastError();
}


}  // namespace mlmc
