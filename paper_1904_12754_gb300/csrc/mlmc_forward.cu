// Forward mode (the full-vector representation of Sec. 2.1, Eq. 5): walks
// run on B = A^T from a start s drawn with probability ~ |v_s| and add
// sign(v_s) (W / w_s) |v_s| e^{E} to x[end].
//
//   transpose  canonical CSR of A^T on the device: column counts, an
//              exclusive scan, a scatter, then each row sorted by column
//              (keys are unique, so the result does not depend on the order
//              the scatter's atomics happened to take);
//   starts     integer weights w_s = ceil(|v_s| / max|v| * 2^20) (0 where
//              v_s = 0), their inclusive int64 prefix sum C (exact, order
//              independent) and W = C[n-1].  Walk g draws r = floor(u W / 2^64)
//              from the 64-bit word u of its Philox block at draw index
//              0xFFFFFFFF and starts at the smallest s with C[s] > r, found
//              from a guide table of n cutpoints and a short forward scan;
//              its weight is v_s W / w_s, so E[weight * f(walk from s)] =
//              sum_s v_s f(s) exactly for any positive w.
#include <algorithm>
#include <cmath>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr int kBlock = 256;

__global__ void k_count_cols(int64_t nnz, const int32_t* __restrict__ col,
                             int64_t* __restrict__ cnt) {
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < nnz;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + col[q]), 1ull);
}

// Inclusive scan of int64 values, one block per 1024-element tile; tile sums
// go to `part`.
__global__ void k_scan_tile(int64_t n, const int64_t* __restrict__ in, int64_t* __restrict__ out,
                            int64_t* __restrict__ part) {
  __shared__ int64_t s[1024];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * 1024;
  for (int k = threadIdx.x; k < 1024; k += blockDim.x)
    s[k] = base + k < n ? in[base + k] : 0;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t add[4];
    for (int r = 0; r < 4; ++r) {
      const int k = threadIdx.x + r * 256;
      add[r] = k >= off ? s[k - off] : 0;
    }
    __syncthreads();
    for (int r = 0; r < 4; ++r) s[threadIdx.x + r * 256] += add[r];
    __syncthreads();
  }
  for (int k = threadIdx.x; k < 1024; k += blockDim.x)
    if (base + k < n) out[base + k] = s[k];
  if (threadIdx.x == 0) part[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ part_scan) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * 1024;
  if (blockIdx.x == 0) return;
  const int64_t add = part_scan[blockIdx.x - 1];
  for (int k = threadIdx.x; k < 1024; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

__global__ void k_scatter_t(int64_t n, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            const int64_t* __restrict__ rp_t, int64_t* __restrict__ fill,
                            int32_t* __restrict__ col_t, double* __restrict__ val_t) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int64_t j = col[q];
      const int64_t pos =
          rp_t[j] + static_cast<int64_t>(atomicAdd(reinterpret_cast<unsigned long long*>(fill + j), 1ull));
      col_t[pos] = static_cast<int32_t>(i);
      val_t[pos] = val[q];
    }
}

// Shell sort of each row segment by column (gaps n/2, n/4, ..., 1).
__global__ void k_sort_rows(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                            double* __restrict__ val) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b = rp[i], len = rp[i + 1] - rp[i];
    for (int64_t gap = len / 2; gap > 0; gap /= 2)
      for (int64_t k = gap; k < len; ++k) {
        const int32_t c = col[b + k];
        const double v = val[b + k];
        int64_t m = k;
        while (m >= gap && col[b + m - gap] > c) {
          col[b + m] = col[b + m - gap];
          val[b + m] = val[b + m - gap];
          m -= gap;
        }
        col[b + m] = c;
        val[b + m] = v;
      }
  }
}

__global__ void k_absmax(int64_t n, const double* __restrict__ v, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = fmax(m, fabs(v[i]));
  atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
}

// w_s = ceil(|v_s| / vmax * 2^20) (0 where v_s = 0), IEEE operations only.
__global__ void k_start_weights(int64_t n, const double* __restrict__ v,
                                const unsigned long long* __restrict__ vmax_bits,
                                int64_t* __restrict__ w) {
  const double vmax = __longlong_as_double(static_cast<long long>(*vmax_bits));
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double a = fabs(v[i]);
    w[i] = a > 0.0 ? static_cast<int64_t>(ceil(__dmul_rn(__ddiv_rn(a, vmax), 1048576.0))) : 0;
  }
}

// Guide table of the start draw (the cutpoint method of Chen and Asau):
// bucket b < n holds the answer for r = floor(b W / n).  A draw whose 64-bit
// word is u has r = floor(u W / 2^64) >= floor(b W / n) for b = floor(u n /
// 2^64), so its start is found by scanning forward from guide[b]; with n
// buckets the scan takes one or two steps on average.
__global__ void k_start_guide(int64_t n, const int64_t* __restrict__ cdf, unsigned long long W,
                              int32_t* __restrict__ guide) {
  for (int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; b < n;
       b += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long r = static_cast<unsigned long long>(
        (static_cast<unsigned __int128>(b) * W) / static_cast<unsigned __int128>(n));
    int64_t lo = 0, hi = n - 1;  // smallest s with cdf[s] > r
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (static_cast<unsigned long long>(cdf[mid]) > r) hi = mid; else lo = mid + 1;
    }
    guide[b] = static_cast<int32_t>(lo);
  }
}

int grid_of(const mlmc_plan* p, int64_t items) {
  const int64_t want = (items + kBlock - 1) / kBlock;
  const int64_t cap = static_cast<int64_t>(p->num_sms) * 16;
  return static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
}

}  // namespace

cudaError_t scan_int64(mlmc_plan* p, int64_t n, const int64_t* in, int64_t* out, int64_t* tmp) {
  // tmp: at least 2 * ceil(n / 1024) + 2 entries.
  const int64_t tiles = (n + 1023) / 1024;
  k_scan_tile<<<static_cast<unsigned>(tiles), 256, 0, p->stream>>>(n, in, out, tmp);
  if (tiles > 1) {
    cudaError_t err = scan_int64(p, tiles, tmp, tmp + tiles, tmp + 2 * tiles);
    if (err != cudaSuccess) return err;
    k_scan_add<<<static_cast<unsigned>(tiles), 256, 0, p->stream>>>(n, out, tmp + tiles);
  }
  p->launches += tiles > 1 ? 2 : 1;
  return cudaGetLastError();
}

cudaError_t launch_transpose(mlmc_plan* p, const int64_t* rp, const int32_t* col, const double* val,
                             int64_t* rp_t, int32_t* col_t, double* val_t, int64_t* work) {
  // work: n counts + n fill + scan scratch
  const int64_t n = p->n;
  int64_t* cnt = work;
  int64_t* fill = work + n;
  int64_t* tmp = work + 2 * n;
  cudaError_t err = cudaMemsetAsync(work, 0, sizeof(int64_t) * 2 * n, p->stream);
  if (err != cudaSuccess) return err;
  k_count_cols<<<grid_of(p, p->nnz), kBlock, 0, p->stream>>>(p->nnz, col, cnt);
  // rp_t[0] = 0, rp_t[1..n] = inclusive scan of counts
  err = cudaMemsetAsync(rp_t, 0, sizeof(int64_t), p->stream);
  if (err != cudaSuccess) return err;
  err = scan_int64(p, n, cnt, rp_t + 1, tmp);
  if (err != cudaSuccess) return err;
  k_scatter_t<<<grid_of(p, n), kBlock, 0, p->stream>>>(n, rp, col, val, rp_t, fill, col_t, val_t);
  k_sort_rows<<<grid_of(p, n), 64, 0, p->stream>>>(n, rp_t, col_t, val_t);
  p->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_start_guide(mlmc_plan* p, const int64_t* cdf, unsigned long long W, int32_t* guide) {
  k_start_guide<<<grid_of(p, p->n), kBlock, 0, p->stream>>>(p->n, cdf, W, guide);
  p->launches++;
  return cudaGetLastError();
}

cudaError_t launch_start_table(mlmc_plan* p, const double* v, int64_t* w, int64_t* cdf,
                               int64_t* tmp, unsigned long long* vmax_bits) {
  cudaError_t err = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned long long), p->stream);
  if (err != cudaSuccess) return err;
  k_absmax<<<grid_of(p, p->n), kBlock, 0, p->stream>>>(p->n, v, vmax_bits);
  k_start_weights<<<grid_of(p, p->n), kBlock, 0, p->stream>>>(p->n, v, vmax_bits, w);
  p->launches += 2;
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return scan_int64(p, p->n, w, cdf, tmp);
}

}  // namespace mlmc
