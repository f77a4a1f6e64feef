// FP64 reductions of the controller: sum and sum of squares of a level's
// per-row sums (for V_l and ||m_l||), and the final cross-level sum
// x = sum_l S_l / M_l (Eq. 10) with ||x||^2.
#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr int kRedBlock = 256;
constexpr int kMaxLevels = 32;

struct FinalizeArgs {
  const double* s[kMaxLevels];
  double inv_m[kMaxLevels];
  int count;
};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[kRedBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  v = threadIdx.x < kRedBlock / 32 ? part[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  }
  return v;
}

// Per-block partial sums of a and a^2: part[b], part[gridDim.x + b].
__global__ void __launch_bounds__(kRedBlock) k_sum_sumsq(int64_t n, const double* __restrict__ a,
                                                         double* __restrict__ part) {
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedBlock) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kRedBlock) {
    const double x = a[i];
    s1 += x;
    s2 += x * x;
  }
  s1 = block_sum(s1);
  __syncthreads();
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

// out[k] = the sum of parts[k * g .. k * g + g) for k < count, in a fixed
// order (lane j adds partials j, j + 32, ...; then a fixed shuffle tree): the
// controller's sums are the same bits on every run and on every rank of a
// sharded solve, so every rank takes the same decisions.  One warp.
__global__ void k_combine(int g, int count, const double* __restrict__ parts,
                          double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < count; ++k) {
    double v = 0.0;
    for (int b = lane; b < g; b += 32) v += parts[static_cast<int64_t>(k) * g + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) out[k] = v;
  }
}

// x = sum_l S_l / M_l and per-block partials of ||x||^2 (part[b]).
__global__ void __launch_bounds__(kRedBlock) k_finalize(int64_t n, FinalizeArgs f,
                                                        double* __restrict__ x,
                                                        double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kRedBlock) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kRedBlock) {
    double xi = 0.0;
    for (int l = 0; l < f.count; ++l) xi += f.s[l][i] * f.inv_m[l];
    if (x) x[i] = xi;
    acc += xi * xi;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

int red_grid(const mlmc_plan* p) {
  const int64_t want = (p->n + kRedBlock - 1) / kRedBlock;
  const int64_t cap = static_cast<int64_t>(p->num_sms) * 8;
  return static_cast<int>(want < 1 ? 1 : (want > cap ? cap : want));
}

struct FinalizeTimesArgs {
  const double* s[kMaxLevels];  // level sums [(T-1) x n]
  double inv_m[kMaxLevels];
  int count;
};

__global__ void __launch_bounds__(kRedBlock) k_finalize_times(int64_t total, FinalizeTimesArgs f,
                                                              double* __restrict__ x) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(kRedBlock) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * kRedBlock) {
    double xe = 0.0;
    for (int l = 0; l < f.count; ++l) xe += f.s[l][e] * f.inv_m[l];
    x[e] = xe;
  }
}

}  // namespace

cudaError_t launch_finalize_times(mlmc_plan* p, int num_levels, int n_times, double* x_times) {
  if (num_levels > kMaxLevels || n_times < 2) return cudaErrorInvalidValue;
  FinalizeTimesArgs f{};
  const int64_t per_level = static_cast<int64_t>(kMaxTimesAll - 1) * p->n;
  for (int k = 0; k < num_levels; ++k) {
    f.s[k] = p->d_times + k * per_level;
    const int64_t m = p->levels[k].reps;
    f.inv_m[k] = m > 0 ? 1.0 / static_cast<double>(m) : 0.0;
  }
  f.count = num_levels;
  const int64_t total = static_cast<int64_t>(n_times - 1) * p->n;
  const int64_t want = (total + kRedBlock - 1) / kRedBlock;
  const int64_t cap = static_cast<int64_t>(p->num_sms) * 8;
  k_finalize_times<<<static_cast<int>(want < 1 ? 1 : (want > cap ? cap : want)), kRedBlock, 0,
                     p->stream>>>(total, f, x_times);
  p->launches++;
  return cudaGetLastError();
}

cudaError_t launch_sum_sumsq(mlmc_plan* p, const double* a, double* out) {
  const int g = red_grid(p);
  k_sum_sumsq<<<g, kRedBlock, 0, p->stream>>>(p->n, a, p->d_red_part);
  k_combine<<<1, 32, 0, p->stream>>>(g, 2, p->d_red_part, out);
  p->launches += 2;
  return cudaGetLastError();
}

int64_t red_partials(int num_sms) { return 2 * static_cast<int64_t>(num_sms) * 8; }

cudaError_t launch_finalize(mlmc_plan* p, int num_levels, double* x, double* norm2) {
  if (num_levels > kMaxLevels) return cudaErrorInvalidValue;
  FinalizeArgs f{};
  for (int k = 0; k < num_levels; ++k) {
    const LevelAcc& L = p->levels[k];
    f.s[k] = level_sums(p, k);
    f.inv_m[k] = L.reps > 0 ? 1.0 / static_cast<double>(L.reps) : 0.0;
  }
  f.count = num_levels;
  const int g = red_grid(p);
  k_finalize<<<g, kRedBlock, 0, p->stream>>>(p->n, f, x, p->d_red_part);
  k_combine<<<1, 32, 0, p->stream>>>(g, 1, p->d_red_part, norm2);
  p->launches += 2;
  return cudaGetLastError();
}

}  // namespace mlmc
