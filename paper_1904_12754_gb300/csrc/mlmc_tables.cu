// Table build on the device: CSR validation, the split A = D - T of Sec. 2.1
// (Eq. 1) and per-row Vose alias tables for the jump law of Eq. 12.
//
// One thread owns one row and scans it in stored order, so every sum and
// every alias decision is a fixed sequence of IEEE operations (explicit
// round-to-nearest, no contraction): the tables are identical bit for bit to
// any implementation that performs the same sequence.
#include <cmath>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr int kTableBlock = 256;
// Rows with kHeavyLo..kHeavyHi stored entries are built by a block each
// (k_build_tables_heavy, k_build_is_tables_heavy); the others by a thread.
// The thread-per-row build's time is set by its longest rows (their FP64
// divisions and logarithms and the Vose pass run one after another), so
// everything past a few dozen entries goes to the blocks.
constexpr int kHeavyLo = 32;
constexpr int kHeavyHi = 8192;
__host__ __device__ __forceinline__ bool heavy_len(int64_t len) {
  return len >= kHeavyLo && len <= kHeavyHi;
}

__global__ void k_validate(int64_t n, int64_t nnz, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           uint32_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = row_ptr[i];
    const int64_t e = row_ptr[i + 1];
    uint32_t f = 0;
    if ((i == 0 && b != 0) || e < b || e > nnz || b < 0) {
      atomicOr(flags, kFlagBadRowPtr);
      continue;
    }
    if (i == n - 1 && e != nnz) f |= kFlagBadRowPtr;
    int64_t prev = -1;
    for (int64_t q = b; q < e; ++q) {
      const int64_t c = col[q];
      if (c < 0 || c >= n) f |= kFlagBadCol;
      if (c <= prev) f |= kFlagUnsorted;
      prev = c;
      if (!isfinite(val[q])) f |= kFlagNonFinite;
    }
    if (f) atomicOr(flags, f);
  }
}

// Per row i (one thread):
//   pass 1  a_ii, L_ii = sum_{j != i} |a_ij| (stored order), deg_i; the
//           scaled rate t L_ii and dl_i = t (a_ii + L_ii); both meta records.
//   pass 2  p_b = (|a_b| deg) / L_ii for bucket b (the b-th off-diagonal),
//           kept in the bucket's own entry with a FIFO link (small queue:
//           p < 1, large queue: p >= 1, both in ascending b).
//   pass 3  Vose: pop l from small and g from large; finalise l with
//           threshold floor(p_l 2^32) and alias g; p_g = (p_g + p_l) - 1;
//           append g to small (p_g < 1) or large.  Leftovers keep themselves.
// A finalised entry overwrites its working values; at that point the bucket
// is in no queue and its probability is no longer needed, so the build uses
// no memory beyond the table itself.
__global__ void k_build_tables(int64_t n, double t, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               Meta32* __restrict__ meta32, Meta64* __restrict__ meta64,
                               double* __restrict__ lii_out, AliasEntry* __restrict__ alias,
                               unsigned long long* __restrict__ dmax_bits) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rb = row_ptr[i];
    const int64_t re = row_ptr[i + 1];
    if (heavy_len(re - rb)) continue;  // k_build_tables_heavy
    double diag = 0.0, lsum = 0.0;
    int64_t dpos = -1;
    for (int64_t q = rb; q < re; ++q) {
      if (col[q] == i) {
        diag = val[q];
        dpos = q - rb;
      } else {
        lsum = __dadd_rn(lsum, fabs(val[q]));
      }
    }
    const int32_t k = static_cast<int32_t>((re - rb) - (dpos >= 0 ? 1 : 0));
    const double rate = __dmul_rn(t, lsum);
    const double dl = __dmul_rn(t, __dadd_rn(diag, lsum));
    const double inv_rate = rate > 0.0 ? __ddiv_rn(1.0, rate) : __longlong_as_double(0x7ff0000000000000ll);
    Meta32 m32;
    m32.start = static_cast<int32_t>(rb);
    m32.deg = k;
    m32.inv_rate = __double2float_rn(inv_rate);
    m32.dl = __double2float_rn(dl);
    meta32[i] = m32;
    Meta64 m64;
    m64.start = static_cast<int32_t>(rb);
    m64.deg = k;
    m64.pad0 = 0;
    m64.pad1 = 0;
    m64.inv_rate = inv_rate;
    m64.dl = dl;
    meta64[i] = m64;
    lii_out[i] = lsum;
    const double dm = fmax(fabs(dl), rate);
    atomicMax(dmax_bits, static_cast<unsigned long long>(__double_as_longlong(dm)));
    if (k == 0) continue;

    // Bucket b lives at alias[rb + b]; its CSR position skips the diagonal.
    AliasEntry* row = alias + rb;
    auto csr_of = [&](int32_t b) -> int64_t { return rb + b + ((dpos >= 0 && b >= dpos) ? 1 : 0); };
    auto col_word = [&](int32_t b) -> uint32_t {
      const int64_t q = csr_of(b);
      return static_cast<uint32_t>(col[q]) | (val[q] < 0.0 ? kSignBit : 0u);
    };
    auto p_of = [&](int32_t b) -> double& { return *reinterpret_cast<double*>(&row[b]); };
    auto next_of = [&](int32_t b) -> int32_t& { return *reinterpret_cast<int32_t*>(&row[b].alias); };
    auto finalise = [&](int32_t b, double prob, int32_t alias_b) {
      const double scaled = floor(__dmul_rn(prob, 4294967296.0));
      AliasEntry e;
      e.thr = scaled >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(scaled);
      e.keep = col_word(b);
      e.alias = col_word(alias_b);
      e.pad = 0u;
      row[b] = e;
    };

    const double kd = static_cast<double>(k);
    int32_t s_head = -1, s_tail = -1, g_head = -1, g_tail = -1;
    auto push = [&](int32_t& head, int32_t& tail, int32_t b) {
      next_of(b) = -1;
      if (tail < 0) head = b; else next_of(tail) = b;
      tail = b;
    };
    auto pop = [&](int32_t& head, int32_t& tail) -> int32_t {
      const int32_t b = head;
      head = next_of(b);
      if (head < 0) tail = -1;
      return b;
    };
    for (int32_t b = 0; b < k; ++b) {
      const double w = fabs(val[csr_of(b)]);
      const double p = lsum > 0.0 ? __ddiv_rn(__dmul_rn(w, kd), lsum) : 1.0;
      p_of(b) = p;
      if (p < 1.0) push(s_head, s_tail, b); else push(g_head, g_tail, b);
    }
    while (s_head >= 0 && g_head >= 0) {
      const int32_t l = pop(s_head, s_tail);
      const int32_t g = pop(g_head, g_tail);
      const double pl = p_of(l);
      const double pg = __dsub_rn(__dadd_rn(p_of(g), pl), 1.0);
      finalise(l, pl, g);
      p_of(g) = pg;
      if (pg < 1.0) push(s_head, s_tail, g); else push(g_head, g_tail, g);
    }
    while (g_head >= 0) {
      const int32_t g = pop(g_head, g_tail);
      finalise(g, 1.0, g);
    }
    while (s_head >= 0) {
      const int32_t l = pop(s_head, s_tail);
      finalise(l, 1.0, l);
    }
  }
}

// Proposal tables: per row i with h > 0 on the columns,
//   q_b = (1 - alpha) (|a_b| h(col_b)) / sum_c |a_c| h(col_c) + alpha |a_b| / L_ii
// (a defensive mixture with the paper's law k_b = |a_b| / L_ii),
// p_b = q_b deg, then the same Vose construction as k_build_tables; each
// entry also stores lr = log(k/q) of its kept and alias columns.  During the
// build an entry holds its working probability (bytes 0-7), its FIFO link
// (bytes 8-11) and its own lr (bytes 16-19, which is also its final lr_keep).
// Tilted clocks (clocks = true, the h-transform): the row's rate becomes
//   lambda_i = sum_{j != i} |a_ij| h_j / h_i, clamped to
//   [L_ii/1024, max(L_ii, 2/t)] (0 where L_ii = 0: a clock runs faster than
//   the paper's only while its scaled rate t lambda stays below 2), its records m32t/m64t get rate t lambda_i and
// dl_i = t (a_ii + lambda_i) (the split D' = diag(a + lambda),
// T' = diag(lambda) - N, whose Strang product the walk then estimates), and
// every entry's lr gains log(L_ii / lambda_i), the clock's likelihood ratio
// per jump.  The same IEEE operations in the same order as the host
// definition, so the records are identical bit for bit.
__global__ void k_build_is_tables(int64_t n, int64_t nnz, const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  const double* __restrict__ lii, const float* __restrict__ h,
                                  double alpha, AliasEntryIS* __restrict__ alias, bool clocks,
                                  double t, Meta32* __restrict__ m32t, Meta64* __restrict__ m64t,
                                  double* __restrict__ lam_out) {
  // grid.y: the time piece (reading R19).  Its h, entries and rates sit
  // piece n (entries: piece nnz) after piece 0's; the row records are
  // state-major, row i's record of piece kp at i K + kp (K = gridDim.y), so
  // that a walk's later pieces of one state share its cache line.
  const int64_t kp = blockIdx.y, kk = gridDim.y;
  h += kp * n;
  alias += kp * nnz;
  if (lam_out) lam_out += kp * n;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rb = row_ptr[i];
    const int64_t re = row_ptr[i + 1];
    if (heavy_len(re - rb)) continue;  // k_build_is_tables_heavy
    int64_t dpos = -1;
    double hsum = 0.0, diag = 0.0;
    for (int64_t q = rb; q < re; ++q) {
      if (col[q] == i) {
        dpos = q - rb;
        diag = val[q];
      } else {
        hsum = __dadd_rn(hsum, __dmul_rn(fabs(val[q]), static_cast<double>(h[col[q]])));
      }
    }
    const int32_t k = static_cast<int32_t>((re - rb) - (dpos >= 0 ? 1 : 0));
    const double L = lii[i];
    double lr_clock = 0.0;
    if (clocks) {
      double lam = 0.0;
      if (L > 0.0) {
        const double r = __ddiv_rn(hsum, static_cast<double>(h[i]));
        const double lo = __dmul_rn(L, 1.0 / 1024.0);
        const double cap = t > 0.0 ? __ddiv_rn(2.0, t) : 0.0;
        const double hi = L > cap ? L : cap;
        lam = r < lo ? lo : (r > hi ? hi : r);
        lr_clock = lam > 0.0 ? log(L / lam) : 0.0;
      }
      const double rate = __dmul_rn(t, lam);
      const double dl = __dmul_rn(t, __dadd_rn(diag, lam));
      const double inv_rate =
          rate > 0.0 ? __ddiv_rn(1.0, rate) : __longlong_as_double(0x7ff0000000000000ll);
      Meta32 m32;
      m32.start = static_cast<int32_t>(rb);
      m32.deg = k;
      m32.inv_rate = __double2float_rn(inv_rate);
      m32.dl = __double2float_rn(dl);
      m32t[i * kk + kp] = m32;
      Meta64 m64;
      m64.start = static_cast<int32_t>(rb);
      m64.deg = k;
      m64.pad0 = 0;
      m64.pad1 = 0;
      m64.inv_rate = inv_rate;
      m64.dl = dl;
      m64t[i * kk + kp] = m64;
      lam_out[i] = lam;
    }
    if (k == 0) continue;
    AliasEntryIS* row = alias + rb;
    auto csr_of = [&](int32_t b) -> int64_t { return rb + b + ((dpos >= 0 && b >= dpos) ? 1 : 0); };
    auto col_word = [&](int32_t b) -> uint32_t {
      const int64_t q = csr_of(b);
      return static_cast<uint32_t>(col[q]) | (val[q] < 0.0 ? kSignBit : 0u);
    };
    auto p_of = [&](int32_t b) -> double& { return *reinterpret_cast<double*>(&row[b]); };
    auto next_of = [&](int32_t b) -> int32_t& { return *reinterpret_cast<int32_t*>(&row[b].alias); };
    auto finalise = [&](int32_t b, double prob, int32_t alias_b) {
      const double scaled = floor(__dmul_rn(prob, 4294967296.0));
      const float lr_alias = row[alias_b].lr_keep;  // alias_b's own lr
      row[b].thr = scaled >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(scaled);
      row[b].keep = col_word(b);
      row[b].alias = col_word(alias_b);
      row[b].pad = 0u;
      row[b].lr_alias = lr_alias;
      row[b].pad1 = 0u;
      row[b].pad2 = 0u;
    };
    const double kd = static_cast<double>(k);
    const double keep_mix = __dsub_rn(1.0, alpha);
    int32_t s_head = -1, s_tail = -1, g_head = -1, g_tail = -1;
    auto push = [&](int32_t& head, int32_t& tail, int32_t b) {
      next_of(b) = -1;
      if (tail < 0) head = b; else next_of(tail) = b;
      tail = b;
    };
    auto pop = [&](int32_t& head, int32_t& tail) -> int32_t {
      const int32_t b = head;
      head = next_of(b);
      if (head < 0) tail = -1;
      return b;
    };
    for (int32_t b = 0; b < k; ++b) {
      const int64_t q = csr_of(b);
      const double w = fabs(val[q]);
      double p = 1.0, lr = 0.0;
      if (L > 0.0) {
        if (hsum > 0.0) {
          const double kb = __ddiv_rn(w, L);
          const double qb = __dadd_rn(
              __dmul_rn(keep_mix, __ddiv_rn(__dmul_rn(w, static_cast<double>(h[col[q]])), hsum)),
              __dmul_rn(alpha, kb));
          p = __dmul_rn(qb, kd);
          lr = __dadd_rn(qb > 0.0 ? log(kb / qb) : 0.0, lr_clock);
        } else {
          p = __ddiv_rn(__dmul_rn(w, kd), L);
          lr = lr_clock;
        }
      }
      p_of(b) = p;
      row[b].lr_keep = static_cast<float>(lr);
      if (p < 1.0) push(s_head, s_tail, b); else push(g_head, g_tail, b);
    }
    while (s_head >= 0 && g_head >= 0) {
      const int32_t l = pop(s_head, s_tail);
      const int32_t g = pop(g_head, g_tail);
      const double pl = p_of(l);
      const double pg = __dsub_rn(__dadd_rn(p_of(g), pl), 1.0);
      finalise(l, pl, g);
      p_of(g) = pg;
      if (pg < 1.0) push(s_head, s_tail, g); else push(g_head, g_tail, g);
    }
    while (g_head >= 0) {
      const int32_t g = pop(g_head, g_tail);
      finalise(g, 1.0, g);
    }
    while (s_head >= 0) {
      const int32_t l = pop(s_head, s_tail);
      finalise(l, 1.0, l);
    }
  }
}

// ---------------------------------------------------------------------------
// Long rows (kHeavyLo <= row length <= kHeavyHi: the hubs of a scale-free
// graph and the rows around them): one block per row instead of one thread, with the row's working
// values in shared memory.  The sums stay sequential in stored order and the
// Vose pairing stays one sequence of pops and pushes (thread 0), so the
// tables are the same bits as the one-thread build; the per-entry arithmetic
// and the final writes run on all the block's threads.  Without this a hub
// row's thread walks its entries through global memory alone, which set the
// build's time (a 1241-entry row: about 4 ms).
// ---------------------------------------------------------------------------
constexpr int kHeavyBlock = 256;
// Shared memory per entry of the longest listed row (cap entries): p (8
// bytes), queue link (4), alias bucket (4), and for proposal tables lr (4).
constexpr size_t heavy_smem_plain(int cap) { return static_cast<size_t>(cap) * 16; }
constexpr size_t heavy_smem_is(int cap) { return static_cast<size_t>(cap) * 20; }

// Rows whose length is in [kHeavyLo, kHeavyHi] (any order); count[0] gets
// their number, count[1] the longest of them.
__global__ void k_heavy_rows(int64_t n, const int64_t* __restrict__ row_ptr,
                             int32_t* __restrict__ list, uint32_t* __restrict__ count) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t len = row_ptr[i + 1] - row_ptr[i];
    if (heavy_len(len)) {
      list[atomicAdd(count, 1u)] = static_cast<int32_t>(i);
      atomicMax(count + 1, static_cast<uint32_t>(len));
    }
  }
}

// The Vose pairing of k buckets with probabilities p (thread 0): ali[b] gets
// bucket b's alias, p[b] its final probability (1 for the leftovers).
__device__ void vose_shared(int32_t k, double* p, int32_t* nxt, int32_t* ali) {
  int32_t s_head = -1, s_tail = -1, g_head = -1, g_tail = -1;
  auto push = [&](int32_t& head, int32_t& tail, int32_t b) {
    nxt[b] = -1;
    if (tail < 0) head = b; else nxt[tail] = b;
    tail = b;
  };
  auto pop = [&](int32_t& head, int32_t& tail) -> int32_t {
    const int32_t b = head;
    head = nxt[b];
    if (head < 0) tail = -1;
    return b;
  };
  for (int32_t b = 0; b < k; ++b) {
    if (p[b] < 1.0) push(s_head, s_tail, b); else push(g_head, g_tail, b);
  }
  while (s_head >= 0 && g_head >= 0) {
    const int32_t l = pop(s_head, s_tail);
    const int32_t g = pop(g_head, g_tail);
    const double pl = p[l];
    const double pg = __dsub_rn(__dadd_rn(p[g], pl), 1.0);
    ali[l] = g;
    p[g] = pg;
    if (pg < 1.0) push(s_head, s_tail, g); else push(g_head, g_tail, g);
  }
  while (g_head >= 0) {
    const int32_t g = pop(g_head, g_tail);
    p[g] = 1.0;
    ali[g] = g;
  }
  while (s_head >= 0) {
    const int32_t l = pop(s_head, s_tail);
    p[l] = 1.0;
    ali[l] = l;
  }
}

// The stored position of the diagonal in row [rb, re) (cols strictly
// increasing), or -1.
__device__ __forceinline__ int64_t diag_pos(const int32_t* __restrict__ col, int64_t rb, int64_t re,
                                            int64_t i) {
  int64_t lo = rb, hi = re - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t c = col[mid];
    if (c == i) return mid - rb;
    if (c < i) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__global__ void __launch_bounds__(kHeavyBlock)
    k_build_tables_heavy(const int32_t* __restrict__ list, const uint32_t* __restrict__ count, int cap,
                         double t, const int64_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, const double* __restrict__ val,
                         Meta32* __restrict__ meta32, Meta64* __restrict__ meta64,
                         double* __restrict__ lii_out, AliasEntry* __restrict__ alias,
                         unsigned long long* __restrict__ dmax_bits) {
  extern __shared__ __align__(16) unsigned char hs[];
  double* p = reinterpret_cast<double*>(hs);
  int32_t* nxt = reinterpret_cast<int32_t*>(hs + cap * 8);
  int32_t* ali = reinterpret_cast<int32_t*>(hs + cap * 12);
  __shared__ double s_lsum;
  const uint32_t rows = *count;
  for (uint32_t it = blockIdx.x; it < rows; it += gridDim.x) {
    const int64_t i = list[it];
    const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
    const int64_t dpos = diag_pos(col, rb, re, i);
    const int32_t k = static_cast<int32_t>((re - rb) - (dpos >= 0 ? 1 : 0));
    auto csr_of = [&](int32_t b) -> int64_t { return rb + b + ((dpos >= 0 && b >= dpos) ? 1 : 0); };
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x) p[b] = fabs(val[csr_of(b)]);
    __syncthreads();
    if (threadIdx.x == 0) {
      double lsum = 0.0;
      for (int32_t b = 0; b < k; ++b) lsum = __dadd_rn(lsum, p[b]);
      const double diag = dpos >= 0 ? val[rb + dpos] : 0.0;
      const double rate = __dmul_rn(t, lsum);
      const double dl = __dmul_rn(t, __dadd_rn(diag, lsum));
      const double inv_rate =
          rate > 0.0 ? __ddiv_rn(1.0, rate) : __longlong_as_double(0x7ff0000000000000ll);
      Meta32 m32;
      m32.start = static_cast<int32_t>(rb);
      m32.deg = k;
      m32.inv_rate = __double2float_rn(inv_rate);
      m32.dl = __double2float_rn(dl);
      meta32[i] = m32;
      Meta64 m64;
      m64.start = static_cast<int32_t>(rb);
      m64.deg = k;
      m64.pad0 = 0;
      m64.pad1 = 0;
      m64.inv_rate = inv_rate;
      m64.dl = dl;
      meta64[i] = m64;
      lii_out[i] = lsum;
      const double dm = fmax(fabs(dl), rate);
      atomicMax(dmax_bits, static_cast<unsigned long long>(__double_as_longlong(dm)));
      s_lsum = lsum;
    }
    __syncthreads();
    const double lsum = s_lsum;
    const double kd = static_cast<double>(k);
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x)
      p[b] = lsum > 0.0 ? __ddiv_rn(__dmul_rn(p[b], kd), lsum) : 1.0;
    __syncthreads();
    if (threadIdx.x == 0) vose_shared(k, p, nxt, ali);
    __syncthreads();
    auto col_word = [&](int32_t b) -> uint32_t {
      const int64_t q = csr_of(b);
      return static_cast<uint32_t>(col[q]) | (val[q] < 0.0 ? kSignBit : 0u);
    };
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x) {
      const double scaled = floor(__dmul_rn(p[b], 4294967296.0));
      AliasEntry e;
      e.thr = scaled >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(scaled);
      e.keep = col_word(b);
      e.alias = col_word(ali[b]);
      e.pad = 0u;
      alias[rb + b] = e;
    }
    __syncthreads();  // the next row reuses the shared arrays
  }
}

__global__ void __launch_bounds__(kHeavyBlock)
    k_build_is_tables_heavy(const int32_t* __restrict__ list, const uint32_t* __restrict__ count,
                            int cap, int64_t n, int64_t nnz, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ lii,
                            const float* __restrict__ h, double alpha,
                            AliasEntryIS* __restrict__ alias, bool clocks, double t,
                            Meta32* __restrict__ m32t, Meta64* __restrict__ m64t,
                            double* __restrict__ lam_out) {
  extern __shared__ __align__(16) unsigned char hs[];
  double* p = reinterpret_cast<double*>(hs);
  int32_t* nxt = reinterpret_cast<int32_t*>(hs + cap * 8);
  int32_t* ali = reinterpret_cast<int32_t*>(hs + cap * 12);
  float* lrs = reinterpret_cast<float*>(hs + cap * 16);
  __shared__ double s_hsum, s_lr_clock;
  // grid.y: the time piece, as in k_build_is_tables (records state-major)
  const int64_t kp = blockIdx.y, kk = gridDim.y;
  h += kp * n;
  alias += kp * nnz;
  if (lam_out) lam_out += kp * n;
  const uint32_t rows = *count;
  for (uint32_t it = blockIdx.x; it < rows; it += gridDim.x) {
    const int64_t i = list[it];
    const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
    const int64_t dpos = diag_pos(col, rb, re, i);
    const int32_t k = static_cast<int32_t>((re - rb) - (dpos >= 0 ? 1 : 0));
    auto csr_of = [&](int32_t b) -> int64_t { return rb + b + ((dpos >= 0 && b >= dpos) ? 1 : 0); };
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x) {
      const int64_t q = csr_of(b);
      p[b] = __dmul_rn(fabs(val[q]), static_cast<double>(h[col[q]]));
    }
    __syncthreads();
    const double L = lii[i];
    if (threadIdx.x == 0) {
      double hsum = 0.0;
      for (int32_t b = 0; b < k; ++b) hsum = __dadd_rn(hsum, p[b]);
      const double diag = dpos >= 0 ? val[rb + dpos] : 0.0;
      double lr_clock = 0.0;
      if (clocks) {
        double lam = 0.0;
        if (L > 0.0) {
          const double r = __ddiv_rn(hsum, static_cast<double>(h[i]));
          const double lo = __dmul_rn(L, 1.0 / 1024.0);
          const double cap = t > 0.0 ? __ddiv_rn(2.0, t) : 0.0;
          const double hi = L > cap ? L : cap;
          lam = r < lo ? lo : (r > hi ? hi : r);
          lr_clock = lam > 0.0 ? log(L / lam) : 0.0;
        }
        const double rate = __dmul_rn(t, lam);
        const double dl = __dmul_rn(t, __dadd_rn(diag, lam));
        const double inv_rate =
            rate > 0.0 ? __ddiv_rn(1.0, rate) : __longlong_as_double(0x7ff0000000000000ll);
        Meta32 m32;
        m32.start = static_cast<int32_t>(rb);
        m32.deg = k;
        m32.inv_rate = __double2float_rn(inv_rate);
        m32.dl = __double2float_rn(dl);
        m32t[i * kk + kp] = m32;
        Meta64 m64;
        m64.start = static_cast<int32_t>(rb);
        m64.deg = k;
        m64.pad0 = 0;
        m64.pad1 = 0;
        m64.inv_rate = inv_rate;
        m64.dl = dl;
        m64t[i * kk + kp] = m64;
        lam_out[i] = lam;
      }
      s_hsum = hsum;
      s_lr_clock = lr_clock;
    }
    __syncthreads();
    const double hsum = s_hsum, lr_clock = s_lr_clock;
    const double kd = static_cast<double>(k);
    const double keep_mix = __dsub_rn(1.0, alpha);
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x) {
      const int64_t q = csr_of(b);
      const double w = fabs(val[q]);
      double pb = 1.0, lr = 0.0;
      if (L > 0.0) {
        if (hsum > 0.0) {
          const double kb = __ddiv_rn(w, L);
          const double qb = __dadd_rn(
              __dmul_rn(keep_mix, __ddiv_rn(__dmul_rn(w, static_cast<double>(h[col[q]])), hsum)),
              __dmul_rn(alpha, kb));
          pb = __dmul_rn(qb, kd);
          lr = __dadd_rn(qb > 0.0 ? log(kb / qb) : 0.0, lr_clock);
        } else {
          pb = __ddiv_rn(__dmul_rn(w, kd), L);
          lr = lr_clock;
        }
      }
      p[b] = pb;
      lrs[b] = static_cast<float>(lr);
    }
    __syncthreads();
    if (threadIdx.x == 0) vose_shared(k, p, nxt, ali);
    __syncthreads();
    auto col_word = [&](int32_t b) -> uint32_t {
      const int64_t q = csr_of(b);
      return static_cast<uint32_t>(col[q]) | (val[q] < 0.0 ? kSignBit : 0u);
    };
    AliasEntryIS* row = alias + rb;
    for (int32_t b = threadIdx.x; b < k; b += blockDim.x) {
      const double scaled = floor(__dmul_rn(p[b], 4294967296.0));
      AliasEntryIS e;
      e.thr = scaled >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(scaled);
      e.keep = col_word(b);
      e.alias = col_word(ali[b]);
      e.pad = 0u;
      e.lr_keep = lrs[b];
      e.lr_alias = lrs[ali[b]];
      e.pad1 = 0u;
      e.pad2 = 0u;
      row[b] = e;
    }
    __syncthreads();
  }
}

int grid_for(const mlmc_plan* p, int64_t items, int block) {
  const int64_t want = (items + block - 1) / block;
  const int64_t cap = static_cast<int64_t>(p->num_sms) * 16;
  return static_cast<int>(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_validate(mlmc_plan* p) {
  k_validate<<<grid_for(p, p->n, kTableBlock), kTableBlock, 0, p->stream>>>(
      p->n, p->nnz, p->d_row_ptr, p->d_col, p->d_val, p->d_flags);
  p->launches++;
  return cudaGetLastError();
}

// Fused entries (the walk's table): each row's alias entries followed by the
// row records of their kept and alias columns.  One warp per row, its lanes
// over the row's entries (a hub row is not left to one thread).
template <typename Fused, typename Meta>
__global__ void k_fuse(int64_t n, const Meta* __restrict__ meta, const AliasEntry* __restrict__ alias,
                       Fused* __restrict__ fused) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    const int64_t start = meta[i].start;
    const int32_t deg = meta[i].deg;
    for (int32_t b = lane; b < deg; b += 32) {
      const AliasEntry e = alias[start + b];
      Fused f;
      f.thr = e.thr;
      f.keep = e.keep;
      f.alias = e.alias;
      f.pad = 0;
      f.mk = meta[e.keep & kColMask];
      f.ma = meta[e.alias & kColMask];
      fused[start + b] = f;
    }
  }
}

// FP32 walks: per row with 1/(t L) >= 1 (the rows the walk kernel screens),
// the largest first-uniform index whose holding time reaches s = 1
// (still_index32); other rows get -1 (never read).  One warp per row.
__global__ void __launch_bounds__(256) k_still_index(int64_t n, const Meta32* __restrict__ meta,
                                                     int32_t* __restrict__ still) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    const float ir = meta[i].inv_rate;
    const int32_t k = ir >= 1.0f ? still_index32(ir, lane) : -1;  // warp-uniform branch
    if (lane == 0) still[i] = k;
  }
}

// The same with time pieces (reading R19): row i's records of the K pieces
// are meta[i K + p]; screened rows are those whose first piece has
// 1/(t lambda) >= 1.
__global__ void __launch_bounds__(256) k_still_index_pieces(int64_t n, const Meta32* __restrict__ meta,
                                                            int k_pieces, int32_t* __restrict__ still) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const float inv_k = __fdiv_rn(1.0f, static_cast<float>(k_pieces));
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    float ir[kMaxPieces];
#pragma unroll
    for (int p = 0; p < kMaxPieces; ++p) ir[p] = p < k_pieces ? meta[i * k_pieces + p].inv_rate : 1.0f;
    const int32_t k = ir[0] >= 1.0f ? still_index32_pieces(ir, k_pieces, inv_k, lane) : -1;
    if (lane == 0) still[i] = k;
  }
}

// The plan's long rows (once: the matrix structure does not change).
cudaError_t classify_heavy_rows(mlmc_plan* p) {
  if (p->heavy_count >= 0) return cudaSuccess;
  cudaError_t err = cudaMalloc(&p->d_heavy, sizeof(int32_t) * static_cast<size_t>(p->n > 0 ? p->n : 1) +
                                                2 * sizeof(uint32_t));
  if (err != cudaSuccess) return err;
  uint32_t* count = reinterpret_cast<uint32_t*>(p->d_heavy + (p->n > 0 ? p->n : 1));
  if ((err = cudaMemsetAsync(count, 0, 2 * sizeof(uint32_t), p->stream)) != cudaSuccess) return err;
  k_heavy_rows<<<grid_for(p, p->n, kTableBlock), kTableBlock, 0, p->stream>>>(p->n, p->d_row_ptr,
                                                                              p->d_heavy, count);
  p->launches++;
  uint32_t h[2] = {0, 0};
  if ((err = cudaMemcpyAsync(h, count, sizeof(h), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
    return err;
  if ((err = cudaStreamSynchronize(p->stream)) != cudaSuccess) return err;
  p->d_heavy_count = count;
  p->heavy_count = h[0];
  p->heavy_cap = static_cast<int>((h[1] + 3u) & ~3u);
  return cudaSuccess;
}

int heavy_grid(const mlmc_plan* p) {
  const int64_t cap = static_cast<int64_t>(p->num_sms) * 8;
  return static_cast<int>(p->heavy_count < cap ? p->heavy_count : cap);
}

cudaError_t launch_build_tables(mlmc_plan* p) {
  cudaError_t err = cudaMemsetAsync(p->d_norm2, 0, sizeof(double), p->stream);
  if (err != cudaSuccess) return err;
  if ((err = classify_heavy_rows(p)) != cudaSuccess) return err;
  // Narrow blocks: the work per row is as uneven as the degree distribution.
  constexpr int kBuildBlock = 64;
  k_build_tables<<<grid_for(p, p->n, kBuildBlock), kBuildBlock, 0, p->stream>>>(
      p->n, p->t, p->d_row_ptr, p->d_col, p->d_val, p->d_meta32, p->d_meta64, p->d_lii,
      p->d_alias, reinterpret_cast<unsigned long long*>(p->d_norm2));
  p->launches++;
  if (p->heavy_count > 0) {
    static std::atomic<uint64_t> attr{0};
    err = ensure_dynamic_smem(k_build_tables_heavy, static_cast<int>(heavy_smem_plain(kHeavyHi)), attr);
    if (err != cudaSuccess) return err;
    k_build_tables_heavy<<<heavy_grid(p), kHeavyBlock, heavy_smem_plain(p->heavy_cap), p->stream>>>(
        p->d_heavy, p->d_heavy_count, p->heavy_cap, p->t, p->d_row_ptr, p->d_col, p->d_val, p->d_meta32,
        p->d_meta64, p->d_lii, p->d_alias, reinterpret_cast<unsigned long long*>(p->d_norm2));
    p->launches++;
  }
  // k_fuse: one warp per row, 8 rows per block of 256
  const int fuse_grid = grid_for(p, (p->n + 7) / 8, 1);
  if (p->sched.precision == MLMC_FP64)
    k_fuse<<<fuse_grid, 256, 0, p->stream>>>(p->n, p->d_meta64, p->d_alias,
                                             static_cast<FusedEntry64*>(p->d_fused));
  else
    k_fuse<<<fuse_grid, 256, 0, p->stream>>>(p->n, p->d_meta32, p->d_alias,
                                             static_cast<FusedEntry32*>(p->d_fused));
  p->launches++;
  if (p->sched.precision != MLMC_FP64) {
    const int64_t blocks = (p->n + 7) / 8;
    const int grid = static_cast<int>(blocks < p->num_sms * 16 ? blocks : p->num_sms * 16);
    k_still_index<<<grid > 0 ? grid : 1, 256, 0, p->stream>>>(p->n, p->d_meta32, p->d_still32);
    p->launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_is_tables(mlmc_plan* p) {
  constexpr int kBuildBlock = 64;
  cudaError_t err = classify_heavy_rows(p);
  if (err != cudaSuccess) return err;
  // One table set per time piece (one piece without a time-dependent law):
  // piece k's h, entries, records and rates sit k n (k nnz) after piece 0's.
  // (all pieces in one launch: grid.y = pieces)
  const int pieces = p->clock_tilt ? p->pieces : 1;
  k_build_is_tables<<<dim3(grid_for(p, p->n, kBuildBlock), pieces), kBuildBlock, 0, p->stream>>>(
      p->n, p->nnz, p->d_row_ptr, p->d_col, p->d_val, p->d_lii, p->d_h, p->alpha, p->d_alias_is,
      p->clock_tilt, p->t, p->d_meta32_t, p->d_meta64_t, p->d_lam);
  p->launches++;
  if (p->heavy_count > 0) {
    static std::atomic<uint64_t> attr{0};
    err = ensure_dynamic_smem(k_build_is_tables_heavy, static_cast<int>(heavy_smem_is(kHeavyHi)), attr);
    if (err != cudaSuccess) return err;
    k_build_is_tables_heavy<<<dim3(heavy_grid(p), pieces), kHeavyBlock, heavy_smem_is(p->heavy_cap),
                              p->stream>>>(
        p->d_heavy, p->d_heavy_count, p->heavy_cap, p->n, p->nnz, p->d_row_ptr, p->d_col, p->d_val,
        p->d_lii, p->d_h, p->alpha, p->d_alias_is, p->clock_tilt, p->t, p->d_meta32_t, p->d_meta64_t,
        p->d_lam);
    p->launches++;
  }
  if (p->clock_tilt && p->sched.precision != MLMC_FP64) {
    const int64_t blocks = (p->n + 7) / 8;
    const int grid = static_cast<int>(blocks < p->num_sms * 16 ? blocks : p->num_sms * 16);
    if (pieces > 1)
      k_still_index_pieces<<<grid > 0 ? grid : 1, 256, 0, p->stream>>>(p->n, p->d_meta32_t, pieces,
                                                                      p->d_still32_t);
    else
      k_still_index<<<grid > 0 ? grid : 1, 256, 0, p->stream>>>(p->n, p->d_meta32_t, p->d_still32_t);
    p->launches++;
  }
  return cudaGetLastError();
}

}  // namespace mlmc
