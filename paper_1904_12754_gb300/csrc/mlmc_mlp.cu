// The learned proposal's network: a 16 -> 64 -> 64 -> 1 MLP with BF16
// weights and FP32 accumulation, trained on the GPU.
//
//   H1 = relu(X W1 + b1)      tcgen05 (BF16 x BF16 -> FP32 in TMEM), K = 16
//   H2 = relu(H1 W2 + b2)     tcgen05, K = 64
//   z  = H2 w3 + b3           CUDA cores (one output)
// Loss: mean (z - y)^2.  Backward:
//   dz = 2 (z - y) / B; dw3 = sum dz H2; db3 = sum dz
//   dA2 = dz w3 * [A2 > 0]
//   dH1 = dA2 W2^T            tcgen05 (dA2 rounded to BF16), K = 64
//   dA1 = dH1 * [A1 > 0]
//   dW2 = H1^T dA2, dW1 = X^T dA1, db = column sums   CUDA cores, FP32
// Adam updates FP32 master weights; BF16 copies feed the tensor cores.
// Rounding points (for an independent re-computation): X, W1, W2 and H1 are
// BF16 (round to nearest even); dA2 is rounded to BF16 for the dH1 GEMM;
// everything else is FP32.
//
// Training runs two kernels per step: k_mlp_train_tile does the whole
// forward and backward pass of 128 batch rows in one CTA (three tcgen05
// GEMMs, activations in shared memory and TMEM, weight gradients on the CUDA
// cores), and k_mlp_adam_tiles sums the tiles' gradients and takes the Adam
// step.  Inference (h for every node) uses the layer kernels below.
//
// tcgen05 tile kernel: one CTA of 128 threads computes a 128 x 64 output
// tile.  Operands are staged in shared memory in the canonical no-swizzle
// K-major layout (8-row x 16-byte core matrices; core matrices adjacent in K
// are 128 bytes apart, 8-row groups K/8*128 bytes apart); thread 0 issues
// K/16 tcgen05.mma into a TMEM accumulator and commits to an mbarrier;
// every warp then reads its 32 TMEM lanes with tcgen05.ld.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "mlmc_internal.h"

namespace mlmc {
namespace {

constexpr int kIn = 16;
constexpr int kHid = 64;
// Packed FP32 parameter vector: W1 [16][64] (row = input), b1 [64],
// W2 [64][64] (row = input), b2 [64], w3 [64], b3 [1].
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kParams = kOffB3 + 1;

constexpr int kTileM = 128;
constexpr int kTmemCols = 128;          // accumulator needs 64; the rest is slack
constexpr int kTileSmem = 64 * 1024;    // dynamic shared memory per tile CTA
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading (K) byte offset, stride
// (M/N) byte offset, version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t umma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major operand with K columns in the
// no-swizzle canonical layout.
__device__ __forceinline__ uint32_t core_offset(int row, int k, int K) {
  return static_cast<uint32_t>((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 +
                               (k & 7) * 2);
}

// Out[m][n] = epilogue( sum_k A[m][k] B[n][k] ) for one 128-row tile.
//   A: rows of K bf16 (row-major, lda = K); B: N=64 rows of K bf16 (the
//   K-major form of the right operand).  Epilogue: + bias[n] if bias,
//   relu if relu, stored as bf16 (out_bf16) and/or fp32 (out_f32); the
//   pre-activation sign mask is kept in pre_f32 if given.
template <int K>
__global__ void __launch_bounds__(128)
    k_mlp_tile(int64_t M, const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
               const float* __restrict__ bias, bool relu, __nv_bfloat16* __restrict__ out_bf16,
               float* __restrict__ out_f32, float* __restrict__ pre_f32, uint32_t* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                       // 128 x K bf16
  unsigned char* sB = smem + kTileM * K * 2;      // 64 x K bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kTileM * K * 2 + kHid * K * 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTileM;

  // Stage A (zero rows past M) and B, 16 bytes per copy.
  constexpr int kChunks = K / 8;  // 16-byte chunks per row
  for (int c = tid; c < kTileM * kChunks; c += 128) {
    const int r = c / kChunks, kc = c % kChunks;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (row0 + r < M) val = *reinterpret_cast<const uint4*>(A + (row0 + r) * K + kc * 8);
    *reinterpret_cast<uint4*>(sA + core_offset(r, kc * 8, K)) = val;
  }
  for (int c = tid; c < kHid * kChunks; c += 128) {
    const int r = c / kChunks, kc = c % kChunks;
    *reinterpret_cast<uint4*>(sB + core_offset(r, kc * 8, K)) =
        *reinterpret_cast<const uint4*>(B + r * K + kc * 8);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    constexpr uint32_t idesc = umma_idesc(kTileM, kHid);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    constexpr uint32_t lbo = 128, sbo = (K / 8) * 128;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = umma_desc(a0 + ks * 256, lbo, sbo);
      const uint64_t bd = umma_desc(b0 + ks * 256, lbo, sbo);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
  }
  // Bounded wait for the MMAs (phase 0).
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(0u)
        : "memory");
  }
  // Every thread of the block must agree before the warp-collective loads.
  done = __syncthreads_and(done);
  if (!done && tid == 0) atomicOr(err, 1u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (done) {
    // Warp w reads TMEM lanes 32w..32w+31 (its rows), 16 columns at a time.
    const int r = warp * 32 + (tid & 31);
    const int64_t grow = row0 + r;
#pragma unroll
    for (int cb = 0; cb < kHid / 16; ++cb) {
      uint32_t v[16];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb * 16;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (grow < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = cb * 16 + j;
          float a = __uint_as_float(v[j]);
          if (bias) a += bias[col];
          if (pre_f32) pre_f32[grow * kHid + col] = a;
          const float o = relu ? fmaxf(a, 0.0f) : a;
          if (out_bf16) out_bf16[grow * kHid + col] = __float2bfloat16_rn(o);
          if (out_f32) out_f32[grow * kHid + col] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Fused training step: the forward and backward passes of one 128-row tile
// of a batch in one CTA of 256 threads (row r = TMEM lane r, two threads a
// row).
//
//   weights  one bulk copy (cp.async.bulk, completion on an mbarrier) of the
//            operand image the Adam kernel writes after every update: W1^T,
//            W2^T and W2 as BF16 in the canonical K-major layout, then the
//            FP32 vectors b1, b2, w3, b3
//   GEMM 1   A1 = X W1 (+ b1)       tcgen05, K = 16, TMEM columns 0-63
//   GEMM 2   A2 = H1 W2 (+ b2)      tcgen05, K = 64, columns 64-127
//   head     z, dz, dA2 = dz w3 [A2 > 0] per row (CUDA cores, registers)
//   GEMM 3   dH1 = dA2 W2^T         tcgen05, K = 64, columns 128-191, issued
//            before the CUDA cores sum dW2 = H1^T dA2, db2, dw3, db3 from
//            shared memory, so the two overlap
//   then     dA1 = dH1 [A1 > 0]; dW1 = X^T dA1, db1 (CUDA cores)
//
// The tile's gradient (and loss) go to its own row of `part`; the Adam or
// reduction kernel sums the rows, so nothing is accumulated atomically.
// Rounding points are those of the unfused kernels (see the file header).
// ---------------------------------------------------------------------------
constexpr int kImgW1 = 0;                             // W1^T: 64 x 16 BF16, K = 16
constexpr int kImgW2t = kImgW1 + kHid * kIn * 2;      // W2^T: 64 x 64 BF16 (rows = outputs)
constexpr int kImgW2 = kImgW2t + kHid * kHid * 2;     // W2: 64 x 64 BF16 (rows = inputs)
constexpr int kImgVec = kImgW2 + kHid * kHid * 2;     // FP32 b1[64] b2[64] w3[64] b3
constexpr int kImgBytes = kImgVec + 256 * 4;          // 19456: a multiple of 16
constexpr int kVecB1 = 0, kVecB2 = 64, kVecW3 = 128, kVecB3 = 192;
constexpr int kPart = kParams + 1;                    // a tile's gradient, then its loss
constexpr int kPartStride = (kPart + 3) & ~3;        // row stride: 16-byte aligned rows
// Shared memory of the fused kernel (byte offsets; every part 128-byte aligned).
constexpr int kTsImg = 0;
constexpr int kTsX = kTsImg + kImgBytes;              // X tile, 128 x 16 BF16 (A of GEMM 1)
constexpr int kTsH1 = kTsX + kTileM * kIn * 2;        // H1, 128 x 64 BF16 (A of GEMM 2)
constexpr int kTsDA2b = kTsH1 + kTileM * kHid * 2;    // dA2, 128 x 64 BF16 (A of GEMM 3)
// FP32 row-major tiles with a row stride of 68 floats: a thread's 16-byte
// stores into its own row then fall in 8 distinct bank groups per warp.
constexpr int kLd = 68;
constexpr int kTsDA2 = kTsDA2b + kTileM * kHid * 2;   // dA2, 128 x 64 FP32
constexpr int kTsF2 = kTsDA2 + kTileM * kLd * 4;      // H2, then dA1: 128 x 64 FP32
constexpr int kTsDZ = kTsF2 + kTileM * kLd * 4;       // dz per row
constexpr int kTsLoss = kTsDZ + kTileM * 4;           // loss term per row
constexpr int kTsZ = kTsLoss + kTileM * 4;            // z's two partial sums per row
constexpr int kTsBar = kTsZ + 2 * kTileM * 4;         // 4 mbarriers
constexpr int kTsSlot = kTsBar + 4 * 8;               // TMEM address
constexpr int kTrainSmem = kTsSlot + 16;
constexpr int kTrainTmemCols = 256;                   // three 64-column accumulators
static_assert(kImgBytes % 16 == 0 && kTsX % 128 == 0 && kTsH1 % 128 == 0 && kTsDA2b % 128 == 0,
              "operand alignment");
static_assert(kTsDA2 % 16 == 0 && kTsF2 % 16 == 0 && kTsBar % 8 == 0, "alignment");

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// K/16 tcgen05.mma of a 128 x 64 tile into TMEM column `col`, committed to
// the mbarrier `bar` (issued by one thread).
template <int K>
__device__ __forceinline__ void issue_gemm(uint32_t tmem_d, uint32_t a0, uint32_t b0,
                                           uint32_t bar) {
  constexpr uint32_t idesc = umma_idesc(kTileM, kHid);
  constexpr uint32_t lbo = 128, sbo = (K / 8) * 128;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t ad = umma_desc(a0 + ks * 256, lbo, sbo);
    const uint64_t bd = umma_desc(b0 + ks * 256, lbo, sbo);
    const uint32_t acc = ks > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// 16 FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(u[j]);
}

// Eight values as BF16 into one 16-byte row of a core matrix.
__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v) {
  __nv_bfloat162 q[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(q);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Rows: batch row b of the tile is x[b] (sample == 0) or x[mix64(seed + b)
// mod n_src] (a uniform minibatch drawn on the device).  256 threads: warp w
// reads TMEM lanes 32 (w mod 4) .. + 31 (rows r = 32 (w mod 4) + lane) and
// the accumulator columns of half w / 4 (32 of the 64), so two threads share
// a row; the CUDA-core sums split the weight-gradient entries over all 256.
constexpr int kTrainThreads = 256;
__global__ void __launch_bounds__(kTrainThreads)
    k_mlp_train_tile(int64_t M, const __nv_bfloat16* __restrict__ x, const float* __restrict__ y,
                     int64_t n_src, uint64_t sample_seed, int sample,
                     const unsigned char* __restrict__ img, float* __restrict__ part,
                     uint32_t* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int r = (warp & 3) * 32 + (tid & 31);  // this thread's row (TMEM lane)
  const int half = warp >> 2;                  // its 32 accumulator columns
  const int c0 = half * 32;
  const int64_t b = static_cast<int64_t>(blockIdx.x) * kTileM + r;
  const bool valid = b < M;
  const uint32_t s0 = smem_u32(smem);
  const uint32_t bar = s0 + kTsBar;  // mbarriers: weights, GEMM 1, GEMM 2, GEMM 3
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTsSlot);
  const float* vec = reinterpret_cast<const float*>(smem + kTsImg + kImgVec);
  float* da2f = reinterpret_cast<float*>(smem + kTsDA2);
  float* f2 = reinterpret_cast<float*>(smem + kTsF2);
  float* dzs = reinterpret_cast<float*>(smem + kTsDZ);
  float* lss = reinterpret_cast<float*>(smem + kTsLoss);
  float* zpart = reinterpret_cast<float*>(smem + kTsZ);
  float* out = part + static_cast<int64_t>(blockIdx.x) * kPartStride;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar + 8 * i), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(kImgBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            s0 + kTsImg),
        "l"(img), "r"(kImgBytes), "r"(bar)
        : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTrainTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // Row r of X (zeros past M): inputs 0-7 from one thread of the pair,
  // 8-15 from the other; both keep the target.
  float yv = 0.f;
  {
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (valid) {
      int64_t src = b;
      if (sample) src = static_cast<int64_t>(mix64(sample_seed + static_cast<uint64_t>(b)) %
                                             static_cast<uint64_t>(n_src));
      q = reinterpret_cast<const uint4*>(x + src * kIn)[half];
      yv = y[src];
    }
    *reinterpret_cast<uint4*>(smem + kTsX + core_offset(r, 8 * half, kIn)) = q;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
  bool ok = __syncthreads_and(mbar_wait(bar, 0));

  // GEMM 1 and its epilogue: H1 = relu(A1) on this thread's 32 columns, the
  // sign mask of A1 kept in a register.
  uint32_t mask1 = 0u;
  if (ok) {
    if (tid == 0) issue_gemm<kIn>(tmem, s0 + kTsX, s0 + kTsImg + kImgW1, bar + 8);
    ok = __syncthreads_and(mbar_wait(bar + 8, 0));
  }
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      float v[16];
      const int col0 = c0 + cb * 16;
      tmem_ld16(tmem + lane_base + col0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float a = v[j] + vec[kVecB1 + col0 + j];
        if (a > 0.f) mask1 |= 1u << (cb * 16 + j);
        v[j] = fmaxf(a, 0.f);
      }
      store_bf16x8(smem + kTsH1 + core_offset(r, col0, kHid), v);
      store_bf16x8(smem + kTsH1 + core_offset(r, col0 + 8, kHid), v + 8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) issue_gemm<kHid>(tmem + 64, s0 + kTsH1, s0 + kTsImg + kImgW2t, bar + 16);
    ok = __syncthreads_and(mbar_wait(bar + 16, 0));
  }
  // GEMM 2's epilogue and the head: H2, z (the two halves' partial sums
  // meet in shared memory), dz, dA2 (FP32 and BF16).
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t mask2 = 0u;
    float zh = 0.f;
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      float v[16];
      const int col0 = c0 + cb * 16;
      tmem_ld16(tmem + lane_base + 64 + col0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float a = v[j] + vec[kVecB2 + col0 + j];
        if (a > 0.f) mask2 |= 1u << (cb * 16 + j);
        v[j] = fmaxf(a, 0.f);
        zh += v[j] * vec[kVecW3 + col0 + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(f2 + r * kLd + col0 + 4 * i) =
            make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    zpart[half * kTileM + r] = zh;
    __syncthreads();
    const float z = (zpart[r] + zpart[kTileM + r]) + vec[kVecB3];
    const float inv_b = 1.0f / static_cast<float>(M);
    const float res = z - yv;
    const float dz = valid ? 2.0f * res * inv_b : 0.f;
    if (half == 0) {
      dzs[r] = dz;
      lss[r] = valid ? res * res * inv_b : 0.f;
    }
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      float d[16];
      const int col0 = c0 + cb * 16;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        d[j] = (mask2 >> (cb * 16 + j)) & 1u ? dz * vec[kVecW3 + col0 + j] : 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(da2f + r * kLd + col0 + 4 * i) =
            make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]);
      store_bf16x8(smem + kTsDA2b + core_offset(r, col0, kHid), d);
      store_bf16x8(smem + kTsDA2b + core_offset(r, col0 + 8, kHid), d + 8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // GEMM 3 runs while the CUDA cores sum dW2 = H1^T dA2 (a 4 x 4 block of
    // it per thread), db2, dw3 and db3.
    if (tid == 0) issue_gemm<kHid>(tmem + 128, s0 + kTsDA2b, s0 + kTsImg + kImgW2, bar + 24);
    {
      const int k0 = 4 * (tid >> 4), j0 = 4 * (tid & 15);
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      for (int rr = 0; rr < kTileM; ++rr) {
        const uint2 hb = *reinterpret_cast<const uint2*>(smem + kTsH1 + core_offset(rr, k0, kHid));
        const float2 h01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hb.x));
        const float2 h23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hb.y));
        const float hv[4] = {h01.x, h01.y, h23.x, h23.y};
        const float4 d4 = *reinterpret_cast<const float4*>(da2f + rr * kLd + j0);
        const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(hv[i], dv[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(out + kOffW2 + (k0 + i) * kHid + j0) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
    if (tid < kHid) {
      float s = 0.f;
      for (int rr = 0; rr < kTileM; ++rr) s += da2f[rr * kLd + tid];
      out[kOffB2 + tid] = s;
    } else if (tid < 2 * kHid) {
      const int j = tid - kHid;
      float s = 0.f;
      for (int rr = 0; rr < kTileM; ++rr) s = fmaf(dzs[rr], f2[rr * kLd + j], s);
      out[kOffW3 + j] = s;
    } else if (warp == 4) {
      float sd = 0.f, sl = 0.f;
      for (int rr = tid & 31; rr < kTileM; rr += 32) {
        sd += dzs[rr];
        sl += lss[rr];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xFFFFFFFFu, sd, o);
        sl += __shfl_xor_sync(0xFFFFFFFFu, sl, o);
      }
      if ((tid & 31) == 0) {
        out[kOffB3] = sd;
        out[kParams] = sl;
      }
    }
    // every thread is done with H2 (f2) before dA1 overwrites it
    ok = __syncthreads_and(mbar_wait(bar + 24, 0));
  }
  // GEMM 3's epilogue: dA1 = dH1 [A1 > 0] into f2; then dW1 = X^T dA1 (four
  // entries per thread) and db1.
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      float v[16];
      const int col0 = c0 + cb * 16;
      tmem_ld16(tmem + lane_base + 128 + col0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (!((mask1 >> (cb * 16 + j)) & 1u)) v[j] = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(f2 + r * kLd + col0 + 4 * i) =
            make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    __syncthreads();
    const int k = tid >> 4, j0 = 4 * (tid & 15);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int rr = 0; rr < kTileM; ++rr) {
      const float xv = __bfloat162float(
          *reinterpret_cast<const __nv_bfloat16*>(smem + kTsX + core_offset(rr, k, kIn)));
      const float4 d4 = *reinterpret_cast<const float4*>(f2 + rr * kLd + j0);
      acc[0] = fmaf(xv, d4.x, acc[0]);
      acc[1] = fmaf(xv, d4.y, acc[1]);
      acc[2] = fmaf(xv, d4.z, acc[2]);
      acc[3] = fmaf(xv, d4.w, acc[3]);
    }
    *reinterpret_cast<float4*>(out + kOffW1 + k * kHid + j0) =
        make_float4(acc[0], acc[1], acc[2], acc[3]);
    if (tid < kHid) {
      float s = 0.f;
      for (int rr = 0; rr < kTileM; ++rr) s += f2[rr * kLd + tid];
      out[kOffB1 + tid] = s;
    }
  }
  if (!ok) {
    // a completion wait gave up: the tile contributes nothing
    if (tid == 0) atomicOr(err, 1u);
    for (int e = tid; e < kPart; e += kTrainThreads) out[e] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTrainTmemCols));
}

// The operand image of parameter e (value w) in `img` (see the fused kernel).
__device__ __forceinline__ void image_store(unsigned char* img, int e, float w) {
  float* vec = reinterpret_cast<float*>(img + kImgVec);
  if (e < kOffB1) {
    const int k = (e - kOffW1) / kHid, j = (e - kOffW1) % kHid;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW1 + core_offset(j, k, kIn)) = __float2bfloat16_rn(w);
  } else if (e < kOffW2) {
    vec[kVecB1 + e - kOffB1] = w;
  } else if (e < kOffB2) {
    const int i = (e - kOffW2) / kHid, j = (e - kOffW2) % kHid;
    const __nv_bfloat16 q = __float2bfloat16_rn(w);
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW2t + core_offset(j, i, kHid)) = q;
    *reinterpret_cast<__nv_bfloat16*>(img + kImgW2 + core_offset(i, j, kHid)) = q;
  } else if (e < kOffW3) {
    vec[kVecB2 + e - kOffB2] = w;
  } else if (e < kOffB3) {
    vec[kVecW3 + e - kOffW3] = w;
  } else {
    vec[kVecB3] = w;
  }
}

__global__ void k_mlp_image(const float* __restrict__ p, unsigned char* __restrict__ img) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kParams; e += gridDim.x * blockDim.x)
    image_store(img, e, p[e]);
}

// Sum the tiles' rows of `part`: the gradient (into grad, if given) and the
// loss (into *loss).  With m1 != nullptr also one Adam step on the FP32
// master parameters, whose new values go to the operand image.  A block of
// 32 x 8 threads takes 32 consecutive entries: thread (x, y) sums tiles
// y, y + 8, ..., and the column sums meet in shared memory.
constexpr int kAdamCols = 32, kAdamRows = 8;
__global__ void __launch_bounds__(kAdamCols * kAdamRows)
    k_mlp_adam_tiles(float* __restrict__ p, const float* __restrict__ part, int tiles,
                     float* __restrict__ grad, float* __restrict__ loss, float* __restrict__ m1,
                     float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1,
                     float c2, unsigned char* __restrict__ img) {
  __shared__ float red[kAdamRows][kAdamCols];
  const int tx = threadIdx.x % kAdamCols, ty = threadIdx.x / kAdamCols;
  const int e = blockIdx.x * kAdamCols + tx;
  float g = 0.f;
  if (e < kPart)
    for (int t = ty; t < tiles; t += kAdamRows) g += part[static_cast<int64_t>(t) * kPartStride + e];
  red[ty][tx] = g;
  __syncthreads();
  if (ty != 0 || e >= kPart) return;
#pragma unroll
  for (int r = 1; r < kAdamRows; ++r) g += red[r][tx];
  if (e == kParams) {
    if (loss) *loss = g;
    return;
  }
  if (grad) grad[e] = g;
  if (m1) {
    m1[e] = b1 * m1[e] + (1.f - b1) * g;
    m2[e] = b2 * m2[e] + (1.f - b2) * g * g;
    p[e] -= lr * (m1[e] / c1) / (sqrtf(m2[e] / c2) + eps);
    image_store(img, e, p[e]);
  }
}

// z = H2 w3 + b3 (inference).  One warp per row at a time: lane l holds
// hidden units l and l + 32 (coalesced row reads), z is a warp sum.
__global__ void k_mlp_head(int64_t M, const float* __restrict__ h2, const float* __restrict__ p,
                           float* __restrict__ z) {
  static_assert(kHid == 64, "two hidden units per lane");
  const int lane = threadIdx.x & 31;
  const float w3a = p[kOffW3 + lane];
  const float w3b = p[kOffW3 + lane + 32];
  const float b3 = p[kOffB3];
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < M;
       i += warps) {
    float zi = h2[i * kHid + lane] * w3a + h2[i * kHid + lane + 32] * w3b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zi += __shfl_xor_sync(0xFFFFFFFFu, zi, o);
    if (lane == 0) z[i] = zi + b3;
  }
}

// BF16 operand copies of the weights: W1t [64][16] = W1^T, W2t [64][64] =
// W2^T (forward: rows = outputs, K = inputs) and W2 [64][64] itself (the
// dH1 GEMM: rows = layer-1 units, K = layer-2 units).
__global__ void k_mlp_pack(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1t,
                           __nv_bfloat16* __restrict__ w2t, __nv_bfloat16* __restrict__ w2) {
  for (int e = threadIdx.x; e < kIn * kHid; e += blockDim.x) {
    const int k = e / kHid, j = e % kHid;
    w1t[j * kIn + k] = __float2bfloat16_rn(p[kOffW1 + e]);
  }
  for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
    const int k = e / kHid, j = e % kHid;
    w2t[j * kHid + k] = __float2bfloat16_rn(p[kOffW2 + e]);
    w2[e] = __float2bfloat16_rn(p[kOffW2 + e]);
  }
}

// out_i = sum_{j != i} (|a_ij| / L_ii) in_j: one step of the paper's jump
// law k (Eq. 12); rows without jumps keep in_i.
// One warp per row: the lanes take the row's entries in turn and their sums
// meet in a warp reduction (a hub row is not left to one thread).
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void k_jump_mean(int64_t n, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            const double* __restrict__ lii, const float* __restrict__ in,
                            float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    const double L = lii[i];
    if (!(L > 0.0)) {
      if (lane == 0) out[i] = in[i];
      continue;
    }
    double acc = 0.0;
    for (int64_t q = row_ptr[i] + lane; q < row_ptr[i + 1]; q += 32)
      if (col[q] != i) acc += fabs(val[q]) * static_cast<double>(in[col[q]]);
    acc = warp_sum_d(acc);
    if (lane == 0) out[i] = static_cast<float>(acc / L);
  }
}

// out = |v| + sum_{m=1..3} (t |A|)^m |v| / m!  (the first Taylor terms of
// exp(t |A|) |v|: the value of the walks' unsigned weights to order 3),
// with `term` as scratch (n floats).
__global__ void k_abs_taylor_step(int64_t n, const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  double scale, const float* __restrict__ in,
                                  float* __restrict__ term_out, float* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    double s = 0.0;
    for (int64_t q = row_ptr[i] + lane; q < row_ptr[i + 1]; q += 32)
      if (col[q] != i) s += fabs(val[q]) * static_cast<double>(in[col[q]]);
    s = warp_sum_d(s);
    if (lane == 0) {
      const float tv = static_cast<float>(scale * s);
      term_out[i] = tv;
      acc[i] += tv;
    }
  }
}

__global__ void k_abs_float32(int64_t n, const double* __restrict__ in, float* __restrict__ out,
                              float* __restrict__ acc) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    out[i] = fabsf(static_cast<float>(in[i]));
    acc[i] = out[i];
  }
}

// Time-piece warm starts (reading R19): row p of h (K x n) is the
// third-order Taylor value of exp(tau t|N|)|v| at tau = 1 - (p + 1/2)/K, the
// time left at the middle of piece p,
//   h_p,i = |v_i| + tau c1_i + tau^2 c2_i + tau^3 c3_i + f,  c_m = (t|N|)^m |v| / m!.
__global__ void k_piece_h(int64_t n, int k_pieces, const float* __restrict__ absv,
                          const float* __restrict__ c1, const float* __restrict__ c2,
                          const float* __restrict__ c3, float f, float* __restrict__ h) {
  const int64_t total = n * k_pieces;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = q / n, i = q - p * n;
    const float tau = 1.0f - (static_cast<float>(p) + 0.5f) / static_cast<float>(k_pieces);
    h[q] = fmaf(tau, fmaf(tau, fmaf(tau, c3[i], c2[i]), c1[i]), absv[i]) + f;
  }
}

// h_i = (a_i + fa)^alpha (|b_i| + fb)^(1 - alpha) in FP32.
__global__ void k_power_product(int64_t n, const float* __restrict__ a, const double* __restrict__ b,
                                float fa, float fb, float alpha, float* __restrict__ h) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    h[i] = expf(alpha * logf(a[i] + fa) +
                (1.0f - alpha) * logf(fabsf(static_cast<float>(b[i])) + fb));
}

__global__ void k_to_float32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = static_cast<float>(in[i]);
}

// Per-node features of the proposal network (16, BF16).  The pilot
// estimates are the targets, never inputs, so the network smooths their
// noise.  With k = the jump law and p_m = k^m v (the mean of v after m
// jumps): 1, log1p(deg), t L_ii, t d_i, v_i, p_1..p_4, neighbour mean and max
// of log1p(deg), neighbour mean of t d, log(|v|+eps), log(|p_2|+eps),
// log(|p_4|+eps), log(T_3 + eps) with T_3 = sum_{m<=3} (t|A|)^m |v| / m!;
// eps = 1e-6.
__global__ void k_mlp_features(int64_t n, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const Meta64* __restrict__ meta,
                               const double* __restrict__ lii, double t, const float* __restrict__ v,
                               const float* __restrict__ p1, const float* __restrict__ p2,
                               const float* __restrict__ p3, const float* __restrict__ p4,
                               const float* __restrict__ taylor3, __nv_bfloat16* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    float f[kIn];
    const Meta64 m = meta[i];
    f[0] = 1.f;
    f[1] = log1pf(static_cast<float>(m.deg));
    f[2] = static_cast<float>(t * lii[i]);
    f[3] = static_cast<float>(m.dl);
    f[4] = v[i];
    f[5] = p1[i];
    f[6] = p2[i];
    f[7] = p3[i];
    f[8] = p4[i];
    float sd = 0.f, mx = 0.f, sdl = 0.f;
    int c = 0;
    for (int64_t q = row_ptr[i] + lane; q < row_ptr[i + 1]; q += 32) {
      const int64_t j = col[q];
      if (j == i) continue;
      const Meta64 mj = meta[j];
      const float ld = log1pf(static_cast<float>(mj.deg));
      sd += ld;
      mx = fmaxf(mx, ld);
      sdl += static_cast<float>(mj.dl);
      ++c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sd += __shfl_xor_sync(0xFFFFFFFFu, sd, o);
      mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
      sdl += __shfl_xor_sync(0xFFFFFFFFu, sdl, o);
      c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    }
    if (lane != 0) continue;
    const float ic = c > 0 ? 1.f / static_cast<float>(c) : 0.f;
    f[9] = sd * ic;
    f[10] = mx;
    f[11] = sdl * ic;
    f[12] = logf(fabsf(v[i]) + 1e-6f);
    f[13] = logf(fabsf(p2[i]) + 1e-6f);
    f[14] = logf(fabsf(p4[i]) + 1e-6f);
    f[15] = logf(taylor3[i] + 1e-6f);
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[i * kIn + k] = __float2bfloat16_rn(f[k]);
  }
}

// A pilot's row sums S_i (M walks each) to x-hat_i = S_i / M in place, with
// per-block partials of sum_i S_i^2 / M (part[b]) and max_i |x-hat_i|
// (part[gridDim.x + b]); fixed grid and reduction order, so the pilot's
// variance is the same number on every run.
constexpr int kStatBlocks = 256;
// The largest time-piece warm start the learning tries (reading R19).
constexpr int32_t kLearnMaxPieces = 8;
__global__ void __launch_bounds__(256) k_pilot_stats(int64_t n, double scale, double* __restrict__ sums,
                                                     double* __restrict__ part) {
  __shared__ double s_sq[8], s_mx[8];
  double sq = 0.0, mx = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double sv = sums[i];
    sq += sv * sv * scale;
    const double x = sv * scale;
    sums[i] = x;
    mx = fmax(mx, fabs(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
    mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_sq[warp] = sq;
    s_mx[warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      a += s_sq[w];
      b = fmax(b, s_mx[w]);
    }
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
  }
}

// Per-block partials of max_i |v_i| into part[b] (fixed grid of kStatBlocks).
__global__ void __launch_bounds__(256) k_absmax_partials(int64_t n, const double* __restrict__ v,
                                                         double* __restrict__ part) {
  __shared__ double s_mx[8];
  double mx = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    mx = fmax(mx, fabs(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) b = fmax(b, s_mx[w]);
    part[blockIdx.x] = b;
  }
}

// log targets and, for the proposal, h = exp(z) clamped.
// y_i = alpha log(|x-hat_i| + floor_x) + (1 - alpha) log(|v_i| + floor_v)
// (v may be null when alpha = 1).
__global__ void k_log_target(int64_t n, const double* __restrict__ xhat, float floor_abs,
                             const double* __restrict__ v, float floor_v, float alpha,
                             float* __restrict__ y) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float lx = logf(fabsf(static_cast<float>(xhat[i])) + floor_abs);
    y[i] = v && alpha < 1.0f
               ? alpha * lx + (1.0f - alpha) * logf(fabsf(static_cast<float>(v[i])) + floor_v)
               : lx;
  }
}

__global__ void k_exp_h(int64_t n, const float* __restrict__ z, float* __restrict__ h) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    h[i] = expf(fminf(fmaxf(z[i], -60.f), 60.f));
}

// Gather rows idx[0..B) of X (bf16, 16 wide) and y.
__global__ void k_gather(int64_t B, const int64_t* __restrict__ idx, const __nv_bfloat16* __restrict__ x,
                         const float* __restrict__ y, __nv_bfloat16* __restrict__ xb,
                         float* __restrict__ yb) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < B * kIn;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / kIn, k = e % kIn;
    xb[e] = x[idx[r] * kIn + k];
    if (k == 0) yb[r] = y[idx[r]];
  }
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

struct mlmc_mlp {
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  float* d_p = nullptr;      // FP32 master parameters
  float* d_g = nullptr;      // gradients (mlmc_mlp_loss_grad)
  float* d_m1 = nullptr;     // Adam moments
  float* d_m2 = nullptr;
  float* d_loss = nullptr;
  uint32_t* d_err = nullptr;
  __nv_bfloat16* d_w1t = nullptr;  // inference operands (k_mlp_pack)
  __nv_bfloat16* d_w2t = nullptr;
  __nv_bfloat16* d_w2 = nullptr;
  unsigned char* d_img = nullptr;  // the fused training kernel's operand image
  float* d_part = nullptr;         // per-tile gradients and losses
  int64_t part_tiles = 0;
  // inference activations for up to cap rows
  int64_t cap = 0;
  __nv_bfloat16* d_h1 = nullptr;
  float* d_h2 = nullptr;
  int64_t adam_t = 0;
  int64_t launches = 0;
};

namespace {

mlmc_status mfail(mlmc_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

#define MLP_CUDA(call, what)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return mfail(e_ == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA,             \
                   std::string("mlp ") + (what) + ": " + cudaGetErrorString(e_));              \
  } while (0)

mlmc_status ensure_cap(mlmc_mlp* m, int64_t rows) {
  if (rows <= m->cap) return MLMC_OK;
  cudaFree(m->d_h1);
  cudaFree(m->d_h2);
  m->d_h1 = nullptr;
  m->d_h2 = nullptr;
  m->cap = 0;
  const size_t r = static_cast<size_t>(rows) * kHid;
  MLP_CUDA(cudaMalloc(&m->d_h1, r * 2), "alloc");
  MLP_CUDA(cudaMalloc(&m->d_h2, r * 4), "alloc");
  m->cap = rows;
  return MLMC_OK;
}

mlmc_status ensure_tiles(mlmc_mlp* m, int64_t tiles) {
  if (tiles <= m->part_tiles) return MLMC_OK;
  cudaFree(m->d_part);
  m->d_part = nullptr;
  m->part_tiles = 0;
  MLP_CUDA(cudaMalloc(&m->d_part, sizeof(float) * static_cast<size_t>(tiles) * kPartStride), "alloc");
  m->part_tiles = tiles;
  return MLMC_OK;
}

template <int K>
cudaError_t tile(mlmc_mlp* m, int64_t M, const __nv_bfloat16* A, const __nv_bfloat16* B,
                 const float* bias, bool relu, __nv_bfloat16* ob, float* of, float* pre) {
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = ensure_dynamic_smem(k_mlp_tile<K>, kTileSmem, attr_done);
  if (e != cudaSuccess) return e;
  const unsigned grid = static_cast<unsigned>((M + kTileM - 1) / kTileM);
  if (grid == 0) return cudaSuccess;
  k_mlp_tile<K><<<grid, 128, kTileSmem, m->stream>>>(M, A, B, bias, relu, ob, of, pre, m->d_err);
  m->launches++;
  return cudaGetLastError();
}

// Inference: z = MLP(x) for rows x[0..M) (bf16, 16 wide).
mlmc_status forward(mlmc_mlp* m, const __nv_bfloat16* x, int64_t M, float* z) {
  mlmc_status st = ensure_cap(m, M);
  if (st != MLMC_OK) return st;
  MLP_CUDA((k_mlp_pack<<<1, 256, 0, m->stream>>>(m->d_p, m->d_w1t, m->d_w2t, m->d_w2),
            cudaGetLastError()), "pack");
  MLP_CUDA(tile<kIn>(m, M, x, m->d_w1t, m->d_p + kOffB1, true, m->d_h1, nullptr, nullptr),
           "layer 1");
  MLP_CUDA(tile<kHid>(m, M, m->d_h1, m->d_w2t, m->d_p + kOffB2, true, nullptr, m->d_h2, nullptr),
           "layer 2");
  // one warp per row: 8 rows per block of 256 at a time
  const unsigned g = static_cast<unsigned>(std::min<int64_t>((M + 7) / 8, m->num_sms * 8));
  k_mlp_head<<<std::max(1u, g), 256, 0, m->stream>>>(M, m->d_h2, m->d_p, z);
  MLP_CUDA(cudaGetLastError(), "head");
  m->launches += 2;
  return MLMC_OK;
}

// The fused forward and backward of M batch rows (x[b], or a device-drawn
// minibatch of the n_src rows when sample), one CTA per 128 rows; the
// tiles' gradients and losses land in d_part.
mlmc_status train_tiles(mlmc_mlp* m, const __nv_bfloat16* x, const float* y, int64_t n_src,
                        int64_t M, bool sample, uint64_t sample_seed, int64_t* tiles_out) {
  static std::atomic<uint64_t> attr_done{0};
  MLP_CUDA(ensure_dynamic_smem(k_mlp_train_tile, kTrainSmem, attr_done), "smem attribute");
  const int64_t tiles = (M + kTileM - 1) / kTileM;
  mlmc_status st = ensure_tiles(m, tiles);
  if (st != MLMC_OK) return st;
  k_mlp_train_tile<<<static_cast<unsigned>(tiles), kTrainThreads, kTrainSmem, m->stream>>>(
      M, x, y, n_src, sample_seed, sample ? 1 : 0, m->d_img, m->d_part, m->d_err);
  MLP_CUDA(cudaGetLastError(), "train tile");
  m->launches++;
  *tiles_out = tiles;
  return MLMC_OK;
}

// The operand image from the current parameters.
mlmc_status make_image(mlmc_mlp* m) {
  k_mlp_image<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->d_p, m->d_img);
  MLP_CUDA(cudaGetLastError(), "image");
  m->launches++;
  return MLMC_OK;
}

mlmc_status check_err(mlmc_mlp* m) {
  uint32_t e = 0;
  MLP_CUDA(cudaMemcpyAsync(&e, m->d_err, sizeof(e), cudaMemcpyDeviceToHost, m->stream), "read err");
  MLP_CUDA(cudaStreamSynchronize(m->stream), "sync");
  if (e) return mfail(MLMC_ERR_CUDA, "mlp: tensor-core completion wait timed out");
  return MLMC_OK;
}

}  // namespace

extern "C" {

mlmc_status mlmc_mlp_create(mlmc_mlp** out, uint64_t seed, void* cuda_stream) {
  if (!out) return mfail(MLMC_ERR_INVALID_ARG, "NULL out");
  mlmc_mlp* m = new mlmc_mlp();
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](cudaError_t e) {
    mlmc_mlp_destroy(m);
    return mfail(MLMC_ERR_CUDA, std::string("mlp create: ") + cudaGetErrorString(e));
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&m->d_p, kParams * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_g, kParams * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_m1, kParams * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_m2, kParams * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_loss, 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_err, 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_w1t, kIn * kHid * 2)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_w2t, kHid * kHid * 2)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_w2, kHid * kHid * 2)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&m->d_img, kImgBytes)) != cudaSuccess) return bail(e);
  if ((e = cudaMemset(m->d_img, 0, kImgBytes)) != cudaSuccess) return bail(e);
  // He-style initialisation from a seeded host generator (splitmix64).
  std::vector<float> p(kParams, 0.f);
  uint64_t s = seed ^ 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (static_cast<double>(z >> 11) + 0.5) * 0x1p-53;
  };
  for (int e2 = 0; e2 < kIn * kHid; ++e2) p[kOffW1 + e2] = static_cast<float>((next() - 0.5) * 2.0 * std::sqrt(6.0 / kIn));
  for (int e2 = 0; e2 < kHid * kHid; ++e2) p[kOffW2 + e2] = static_cast<float>((next() - 0.5) * 2.0 * std::sqrt(6.0 / kHid));
  for (int e2 = 0; e2 < kHid; ++e2) p[kOffW3 + e2] = static_cast<float>((next() - 0.5) * 2.0 * std::sqrt(3.0 / kHid));
  if ((e = cudaMemcpy(m->d_p, p.data(), kParams * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
  cudaMemset(m->d_m1, 0, kParams * 4);
  cudaMemset(m->d_m2, 0, kParams * 4);
  cudaMemset(m->d_err, 0, 4);
  *out = m;
  return MLMC_OK;
}

void mlmc_mlp_destroy(mlmc_mlp* m) {
  if (!m) return;
  cudaFree(m->d_p);
  cudaFree(m->d_g);
  cudaFree(m->d_m1);
  cudaFree(m->d_m2);
  cudaFree(m->d_loss);
  cudaFree(m->d_err);
  cudaFree(m->d_w1t);
  cudaFree(m->d_w2t);
  cudaFree(m->d_w2);
  cudaFree(m->d_img);
  cudaFree(m->d_part);
  cudaFree(m->d_h1);
  cudaFree(m->d_h2);
  delete m;
}

int32_t mlmc_mlp_param_count(void) { return kParams; }

int64_t mlmc_mlp_launch_count(const mlmc_mlp* m) { return m ? m->launches : 0; }

mlmc_status mlmc_mlp_params(mlmc_mlp* m, const float* set, float* get) {
  if (!m) return mfail(MLMC_ERR_INVALID_ARG, "NULL mlp");
  if (set) MLP_CUDA(cudaMemcpyAsync(m->d_p, set, kParams * 4, cudaMemcpyDefault, m->stream), "set");
  if (get) MLP_CUDA(cudaMemcpyAsync(get, m->d_p, kParams * 4, cudaMemcpyDefault, m->stream), "get");
  MLP_CUDA(cudaStreamSynchronize(m->stream), "sync");
  return MLMC_OK;
}

mlmc_status mlmc_mlp_forward(mlmc_mlp* m, const uint16_t* x, int64_t n, float* z) {
  if (!m || !x || !z || n < 1) return mfail(MLMC_ERR_INVALID_ARG, "mlmc_mlp_forward: bad argument");
  mlmc_status st = forward(m, reinterpret_cast<const __nv_bfloat16*>(x), n, z);
  if (st != MLMC_OK) return st;
  return check_err(m);
}

mlmc_status mlmc_mlp_loss_grad(mlmc_mlp* m, const uint16_t* x, const float* y, int64_t n,
                               float* loss, float* grad) {
  if (!m || !x || !y || n < 1) return mfail(MLMC_ERR_INVALID_ARG, "mlmc_mlp_loss_grad: bad argument");
  mlmc_status st = make_image(m);
  int64_t tiles = 0;
  if (st == MLMC_OK)
    st = train_tiles(m, reinterpret_cast<const __nv_bfloat16*>(x), y, n, n, false, 0, &tiles);
  if (st != MLMC_OK) return st;
  k_mlp_adam_tiles<<<(kPart + kAdamCols - 1) / kAdamCols, kAdamCols * kAdamRows, 0, m->stream>>>(
      m->d_p, m->d_part, static_cast<int>(tiles), m->d_g, m->d_loss, nullptr, nullptr, 0.f, 0.f,
      0.f, 0.f, 1.f, 1.f, nullptr);
  MLP_CUDA(cudaGetLastError(), "reduce");
  m->launches++;
  if (loss) MLP_CUDA(cudaMemcpyAsync(loss, m->d_loss, 4, cudaMemcpyDefault, m->stream), "loss");
  if (grad) MLP_CUDA(cudaMemcpyAsync(grad, m->d_g, kParams * 4, cudaMemcpyDefault, m->stream), "grad");
  return check_err(m);
}

mlmc_status mlmc_mlp_train(mlmc_mlp* m, const uint16_t* x, const float* y, int64_t n, int32_t steps,
                           int32_t batch, float lr, uint64_t seed, float* final_loss) {
  if (!m || !x || !y || n < 1 || steps < 1 || batch < 1)
    return mfail(MLMC_ERR_INVALID_ARG, "mlmc_mlp_train: bad argument");
  const int64_t B = std::min<int64_t>(batch, n);
  // Two launches per step: the fused forward and backward of the batch's
  // tiles (rows drawn on the device), then the tiles' sum and the Adam
  // step, which also rewrites the operand image for the next step.
  mlmc_status st = make_image(m);
  for (int it = 0; it < steps && st == MLMC_OK; ++it) {
    int64_t tiles = 0;
    const uint64_t sample_seed = (seed * 0x9E3779B97F4A7C15ull) ^ (static_cast<uint64_t>(it) << 40);
    st = train_tiles(m, reinterpret_cast<const __nv_bfloat16*>(x), y, n, B, true, sample_seed,
                     &tiles);
    if (st != MLMC_OK) break;
    ++m->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, static_cast<float>(m->adam_t));
    const float c2 = 1.f - std::pow(b2, static_cast<float>(m->adam_t));
    k_mlp_adam_tiles<<<(kPart + kAdamCols - 1) / kAdamCols, kAdamCols * kAdamRows, 0, m->stream>>>(
        m->d_p, m->d_part, static_cast<int>(tiles), nullptr, m->d_loss, m->d_m1, m->d_m2, lr, b1,
        b2, 1e-8f, c1, c2, m->d_img);
    m->launches++;
    if (cudaGetLastError() != cudaSuccess) st = mfail(MLMC_ERR_CUDA, "mlp train: launch");
  }
  if (st != MLMC_OK) return st;
  if (final_loss) MLP_CUDA(cudaMemcpyAsync(final_loss, m->d_loss, 4, cudaMemcpyDefault, m->stream), "loss");
  return check_err(m);
}

// Learn a proposal for `plan`: a pilot of `pilot_walks` walks per row at
// l0 gives per-row estimates x-hat (the method's own statistics); the MLP
// is trained on features -> a log-value target; h = exp(z) becomes the
// plan's importance-sampling proposal (mlmc_plan_set_tilt with alpha).
// Jumps only: target log|x-hat|.  Jumps and clocks (the h-transform): the
// zero-variance h of a walk at time s is exp((1-s)tA)v, which runs from x at
// the start to v at the end; its geometric mean over the walk,
// sqrt(|x-hat| |v|), is the target (0.5 (log|x-hat| + log|v|)).  Each round
// after the first draws its pilot with the previous round's proposal, whose
// estimates are less noisy.
mlmc_status mlmc_learn_proposal(mlmc_plan* p, mlmc_mlp* m, const double* v, uint64_t seed,
                                int64_t pilot_walks, int32_t steps, int32_t batch, float lr,
                                double alpha, float* final_loss) {
  return mlmc_learn_tilt(p, m, v, seed, pilot_walks, steps, batch, lr, alpha, MLMC_TILT_JUMPS, 1,
                         final_loss);
}

mlmc_status mlmc_learn_tilt(mlmc_plan* p, mlmc_mlp* m, const double* v, uint64_t seed,
                            int64_t pilot_walks, int32_t steps, int32_t batch, float lr,
                            double alpha, int32_t tilt, int32_t rounds, float* final_loss) {
  if (!p || !m || !v || pilot_walks < 1 || rounds < 1 || rounds > 8)
    return mfail(MLMC_ERR_INVALID_ARG, "mlmc_learn_tilt: bad argument");
  if (tilt != MLMC_TILT_JUMPS && tilt != (MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS) &&
      tilt != (MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS | MLMC_TILT_TIME))
    return mfail(MLMC_ERR_INVALID_ARG, "mlmc_learn_tilt: tilt must be MLMC_TILT_JUMPS, "
                                       "MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS or "
                                       "MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS | MLMC_TILT_TIME");
  // The targets are backward value estimates (x-hat per start row); a
  // forward walk's value would be the adjoint problem's.
  if (p->sched.mode != MLMC_BACKWARD)
    return mfail(MLMC_ERR_INVALID_ARG, "mlmc_learn_tilt: backward-mode plans only");
  const bool clocks = (tilt & MLMC_TILT_CLOCKS) != 0;
  const bool timed = (tilt & MLMC_TILT_TIME) != 0;
  const int32_t tilt_law = tilt & (MLMC_TILT_JUMPS | MLMC_TILT_CLOCKS);  // one law: set_tilt's
  // The pilots draw from their own stream (a hash of seed), never from the
  // one mlmc_expmv draws with the same seed: the tilt must not depend on the
  // walks that later estimate x.
  uint64_t learn_seed = seed ^ 0x6C6561726E74696Cull;
  learn_seed = (learn_seed ^ (learn_seed >> 30)) * 0xBF58476D1CE4E5B9ull;
  learn_seed = (learn_seed ^ (learn_seed >> 27)) * 0x94D049BB133111EBull;
  learn_seed ^= learn_seed >> 31;
  const bool was = p->proposal_active;
  const bool was_clocks = p->clock_tilt;
  const int32_t was_pieces = p->pieces;
  const double was_alpha = p->alpha;
  // The plan's proposal before the call (h of every time piece), put back if
  // the call fails.
  float* saved_h = nullptr;
  if (was && p->d_h) {
    const size_t nh = sizeof(float) * static_cast<size_t>(p->n) * static_cast<size_t>(was_pieces);
    if (cudaMalloc(&saved_h, nh) != cudaSuccess ||
        cudaMemcpyAsync(saved_h, p->d_h, nh, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
      cudaFree(saved_h);
      return mfail(MLMC_ERR_CUDA, "mlmc_learn_tilt: saving the plan's proposal failed");
    }
  }
  auto restore = [&]() {
    if (was && saved_h) {
      const mlmc_status rs =
          was_clocks ? mlmc_plan_set_tilt_pieces(p, saved_h, was_pieces, was_alpha)
                     : mlmc_plan_set_tilt(p, saved_h, was_alpha, MLMC_TILT_JUMPS);
      if (rs != MLMC_OK) {
        p->proposal_active = p->clock_tilt = false;  // the paper's walk: always consistent
        p->pieces = 1;
      }
    } else {
      p->proposal_active = was;
      p->clock_tilt = was_clocks;
      p->pieces = was_pieces;
    }
  };
  // The first pilot uses the paper's walk (jumps only) or, with tilted
  // clocks, the tilt of h0 = sqrt(T_3 |v|) (below).
  p->proposal_active = false;
  double* sums = nullptr;
  double* dv = nullptr;
  __nv_bfloat16* feat = nullptr;
  float* y = nullptr;
  float* z = nullptr;
  float* h = nullptr;
  float* pv = nullptr;  // v, k^m v (m = 1..4), T_3, |v|, -, the Taylor terms c_1..c_3 (11 x n)
  float* hp = nullptr;            // a time-piece warm start (K x n)
  float* best_h = nullptr;        // the tilt with the smallest pilot variance so far (K x n)
  int32_t best_pieces = 1;
  double* xwarm = nullptr;        // x-hat of the best warm start's pilot
  double* stats = nullptr;        // a pilot's per-block partial sums (k_pilot_stats)
  __nv_bfloat16* wfeat = nullptr;
  float* wy = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;  // a pilot's walk launch, timed
  auto cleanup = [&]() {
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
    cudaFree(best_h);
    cudaFree(hp);
    cudaFree(xwarm);
    cudaFree(stats);
    cudaFree(wfeat);
    cudaFree(wy);
    cudaFree(pv);
    cudaFree(sums);
    cudaFree(dv);
    cudaFree(feat);
    cudaFree(y);
    cudaFree(z);
    cudaFree(h);
    cudaFree(saved_h);
  };
#define LP_CUDA(call, what)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      const std::string msg_ = std::string("learn proposal ") + (what) + ": " +                \
                               cudaGetErrorString(e_);                                         \
      restore();                                                                               \
      cleanup();                                                                               \
      return mfail(MLMC_ERR_CUDA, msg_);                                                       \
    }                                                                                          \
  } while (0)
  LP_CUDA(cudaEventCreate(&ev_a), "event");
  LP_CUDA(cudaEventCreate(&ev_b), "event");
  LP_CUDA(cudaMalloc(&sums, sizeof(double) * (p->n + kTotSlots)), "alloc");
  LP_CUDA(cudaMalloc(&dv, sizeof(double) * p->n), "alloc");
  LP_CUDA(cudaMalloc(&feat, sizeof(__nv_bfloat16) * p->n * kIn), "alloc");
  LP_CUDA(cudaMalloc(&y, sizeof(float) * p->n), "alloc");
  LP_CUDA(cudaMalloc(&z, sizeof(float) * p->n), "alloc");
  LP_CUDA(cudaMalloc(&h, sizeof(float) * p->n), "alloc");
  LP_CUDA(cudaMalloc(&pv, sizeof(float) * p->n * 11), "alloc");
  const int32_t max_warm_pieces = timed ? std::min(kLearnMaxPieces, 1 << std::min(p->l0, 8)) : 1;
  LP_CUDA(cudaMalloc(&best_h, sizeof(float) * p->n * max_warm_pieces), "alloc");
  if (max_warm_pieces > 1) LP_CUDA(cudaMalloc(&hp, sizeof(float) * p->n * max_warm_pieces), "alloc");
  LP_CUDA(cudaMalloc(&xwarm, sizeof(double) * p->n), "alloc");
  LP_CUDA(cudaMalloc(&stats, sizeof(double) * 2 * kStatBlocks), "alloc");
  LP_CUDA(cudaMemcpyAsync(dv, v, sizeof(double) * p->n, cudaMemcpyDefault, p->stream), "copy v");
  const unsigned g = static_cast<unsigned>(std::min<int64_t>((p->n + 255) / 256, p->num_sms * 8));
  // warp-per-row kernels: 8 rows per block of 256
  const unsigned gw = static_cast<unsigned>(std::min<int64_t>((p->n + 7) / 8, p->num_sms * 16));
  // Features (fixed over the rounds: they use the paper's jump law).
  k_to_float32<<<g, 256, 0, p->stream>>>(p->n, dv, pv);
  p->launches++;
  for (int mstep = 1; mstep <= 4; ++mstep) {
    k_jump_mean<<<gw, 256, 0, p->stream>>>(p->n, p->d_row_ptr, p->d_col, p->d_val, p->d_lii,
                                           pv + (mstep - 1) * p->n, pv + mstep * p->n);
    p->launches++;
  }
  {
    // T_3 in slot 5, |v| in slot 6 and the terms c_m = (t|N|)^m |v| / m! in
    // slots 7 + m
    float* t3 = pv + 5 * p->n;
    k_abs_float32<<<g, 256, 0, p->stream>>>(p->n, dv, pv + 6 * p->n, t3);
    p->launches++;
    for (int mstep = 1; mstep <= 3; ++mstep) {
      k_abs_taylor_step<<<gw, 256, 0, p->stream>>>(p->n, p->d_row_ptr, p->d_col, p->d_val,
                                                  p->t / mstep, pv + (mstep == 1 ? 6 : 6 + mstep) * p->n,
                                                  pv + (7 + mstep) * p->n, t3);
      p->launches++;
    }
  }
  k_mlp_features<<<gw, 256, 0, p->stream>>>(p->n, p->d_row_ptr, p->d_col, p->d_meta64, p->d_lii, p->t,
                                            pv, pv + p->n, pv + 2 * p->n, pv + 3 * p->n,
                                            pv + 4 * p->n, pv + 5 * p->n, feat);
  p->launches++;
  LP_CUDA(cudaGetLastError(), "features");
  double vmax = 0.0;
  {
    k_absmax_partials<<<kStatBlocks, 256, 0, p->stream>>>(p->n, dv, stats);
    p->launches++;
    std::vector<double> hv(kStatBlocks);
    LP_CUDA(cudaMemcpyAsync(hv.data(), stats, sizeof(double) * kStatBlocks, cudaMemcpyDeviceToHost,
                            p->stream), "read max |v|");
    LP_CUDA(cudaStreamSynchronize(p->stream), "sync");
    for (double q : hv) vmax = std::max(vmax, q);
  }
  mlmc_status st = MLMC_OK;
  // Training rows weighted by degree: row i appears 1 + floor(deg_i / mean
  // deg) times (at most 4n rows in all).  Rows with many off-diagonals are
  // few, but their h sets the clocks and jump laws of every row around them,
  // and an MLP fitted to rows drawn uniformly would fit them worst.
  // (The list depends on the matrix alone: the plan keeps it.)
  if (!p->d_train_rows) {
    std::vector<int64_t> rp(p->n + 1);
    LP_CUDA(cudaMemcpyAsync(rp.data(), p->d_row_ptr, sizeof(int64_t) * (p->n + 1),
                            cudaMemcpyDeviceToHost, p->stream), "read row_ptr");
    LP_CUDA(cudaStreamSynchronize(p->stream), "sync");
    const double mean_deg = std::max(1.0, static_cast<double>(rp[p->n]) / static_cast<double>(p->n));
    std::vector<int64_t> idx;
    idx.reserve(static_cast<size_t>(2 * p->n));
    for (int64_t i = 0; i < p->n; ++i) {
      const int64_t c = 1 + static_cast<int64_t>(static_cast<double>(rp[i + 1] - rp[i]) / mean_deg);
      for (int64_t k = 0; k < c && static_cast<int64_t>(idx.size()) < 4 * p->n; ++k) idx.push_back(i);
    }
    int64_t* rows = nullptr;
    LP_CUDA(cudaMalloc(&rows, sizeof(int64_t) * idx.size()), "alloc");
    cudaError_t e = cudaMemcpyAsync(rows, idx.data(), sizeof(int64_t) * idx.size(),
                                    cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) cudaFree(rows);
    LP_CUDA(e, "write rows");
    p->d_train_rows = rows;
    p->n_train_rows = static_cast<int64_t>(idx.size());
  }
  const int64_t n_train = p->n_train_rows;
  const int64_t* widx = p->d_train_rows;
  LP_CUDA(cudaMalloc(&wfeat, sizeof(__nv_bfloat16) * n_train * kIn), "alloc");
  LP_CUDA(cudaMalloc(&wy, sizeof(float) * n_train), "alloc");
  // One pilot at l0 with the plan's current walk law: walks [rep_begin,
  // rep_begin + reps) of every row.  Leaves x-hat (the per-row means) in
  // sums, its largest magnitude in *xmax, and the per-walk variance of the
  // law (the rows' sample variances, averaged over the rows) in *var.
  // The pilot's walk time per walk (ms), from CUDA events on the plan's
  // stream around its launch.
  double pilot_cost = 0.0;
  auto pilot = [&](int64_t rep_begin, int64_t reps, double* xmax, double* var) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * (p->n + kTotSlots), p->stream);
    if (e != cudaSuccess) return e;
    WalkLaunch w;
    w.level = p->l0;
    w.coarse = false;
    w.rep_begin = rep_begin;
    w.reps = reps;
    w.seed = learn_seed;
    w.v = dv;
    w.sum_y = sums;
    w.totals = sums + p->n;
    if ((e = cudaEventRecord(ev_a, p->stream)) != cudaSuccess) return e;
    if ((e = launch_walk(p, w)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_b, p->stream)) != cudaSuccess) return e;
    // x-hat in place and the variance's sums on the device; only the
    // partials and the sum of squares come back
    k_pilot_stats<<<kStatBlocks, 256, 0, p->stream>>>(p->n, 1.0 / static_cast<double>(reps), sums,
                                                      stats);
    p->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<double> hs(2 * kStatBlocks + 1);
    e = cudaMemcpyAsync(hs.data(), stats, sizeof(double) * 2 * kStatBlocks, cudaMemcpyDeviceToHost,
                        p->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hs.data() + 2 * kStatBlocks, sums + p->n + kTotY2, sizeof(double),
                          cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return e;
    double sq = 0.0;
    *xmax = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) {
      sq += hs[b];
      *xmax = std::max(*xmax, hs[kStatBlocks + b]);
    }
    *var = reps > 1 ? (hs[2 * kStatBlocks] - sq) / static_cast<double>(reps - 1) /
                          static_cast<double>(p->n)
                    : std::numeric_limits<double>::infinity();
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, ev_a, ev_b)) != cudaSuccess) return e;
    pilot_cost = static_cast<double>(ms) / (static_cast<double>(reps) * static_cast<double>(p->n));
    return cudaSuccess;
  };
  // Every pilot measures the law it walks with; the law with the smallest
  // measured variance is the one installed at the end (for jumps only the
  // paper's walk, h = 1, is a candidate too).  A law with time pieces costs
  // more per walk (its carry-overs, K sets of tables): it has to win on
  // variance x the pilot's walk time per walk, the work to a given error.
  double best_var = std::numeric_limits<double>::infinity();
  double best_cost = 0.0;
  p->learn_var.clear();
  p->learn_choice = -1;
  int64_t next_rep = 0;
  // src: the h (pieces x n) of the law the pilot walked with, kept if its
  // variance is the smallest so far (nullptr: the law installed last, which
  // stays installed when it wins).
  auto consider = [&](double var, const float* src, int32_t pieces) -> cudaError_t {
    p->learn_var.push_back(var);
    const bool better = pieces > 1 ? var * pilot_cost < best_var * best_cost : var < best_var;
    if (!better) return cudaSuccess;
    best_var = var;
    best_cost = pilot_cost;
    p->learn_choice = static_cast<int32_t>(p->learn_var.size()) - 1;
    best_pieces = pieces;
    return src ? cudaMemcpyAsync(best_h, src, sizeof(float) * p->n * static_cast<size_t>(pieces),
                                 cudaMemcpyDeviceToDevice, p->stream)
               : cudaSuccess;
  };
  // The exponent of x-hat in the training targets (jumps only: 1).
  float target_alpha = 1.0f;
  double xmax_warm = 0.0;
  if (clocks) {
    // Warm starts: the first pilots walk with the tilts of
    //   h0 = (T_3 + f)^a (|v| + f_v)^(1 - a),  a = 1/2, 3/4, 1,
    // T_3 the third-order Taylor value of exp(t|N|)|v| (a feature above) in
    // place of x: the paper's walk gives pilot estimates with the heavy
    // tails the tilt exists to remove (long stays at rows of large t d_ii),
    // and a network fitted to them would misjudge exactly those rows.  The
    // exponent sets how far the clocks follow x: on the scale-free graphs
    // a = 3/4 measured 7-14x below a = 1/2.  The best form's pilot gives the
    // first round's targets, with its exponent.
    const float forms[3] = {0.5f, 0.75f, 1.0f};
    for (int k = 0; k < 3; ++k) {
      k_power_product<<<g, 256, 0, p->stream>>>(p->n, pv + 5 * p->n, dv, static_cast<float>(1e-6),
                                                static_cast<float>(1e-3 * vmax + 1e-30), forms[k], h);
      p->launches++;
      LP_CUDA(cudaGetLastError(), "warm start");
      st = mlmc_plan_set_tilt(p, h, alpha, tilt_law);
      if (st != MLMC_OK) break;
      double xmax = 0.0, var = 0.0;
      LP_CUDA(pilot(next_rep, pilot_walks, &xmax, &var), "warm pilot");
      next_rep += pilot_walks;
      const bool better = var < best_var;
      LP_CUDA(consider(var, h, 1), "keep tilt");
      if (better) {
        target_alpha = forms[k];
        xmax_warm = xmax;
        LP_CUDA(cudaMemcpyAsync(xwarm, sums, sizeof(double) * p->n, cudaMemcpyDeviceToDevice,
                                p->stream), "keep x-hat");
      }
    }
  }
  for (int32_t round = 0; round < rounds && st == MLMC_OK; ++round) {
    double xmax = 0.0;
    if (round == 0 && clocks) {
      // the best warm start's pilot
      LP_CUDA(cudaMemcpyAsync(sums, xwarm, sizeof(double) * p->n, cudaMemcpyDeviceToDevice,
                              p->stream), "x-hat");
      xmax = xmax_warm;
    } else {
      // Later rounds walk with the previous tilt, whose samples are cheap
      // and much less noisy: four times the first round's walks per row.
      const int64_t round_walks = round == 0 ? pilot_walks : 4 * pilot_walks;
      double var = 0.0;
      LP_CUDA(pilot(next_rep, round_walks, &xmax, &var), "pilot walks");
      next_rep += round_walks;
      // (round 0 without clocks walks the paper's law: nothing to keep)
      LP_CUDA(consider(var, round > 0 ? h : nullptr, 1), "keep tilt");
    }
    // Targets a log(|x-hat| + 1e-3 max|x-hat|) + (1 - a) log(|v| + 1e-3
    // max|v|) (rows the pilot never reached do not get arbitrarily small h).
    k_log_target<<<g, 256, 0, p->stream>>>(p->n, sums, static_cast<float>(1e-3 * xmax + 1e-30),
                                           clocks ? dv : nullptr,
                                           static_cast<float>(1e-3 * vmax + 1e-30), target_alpha, y);
    p->launches++;
    LP_CUDA(cudaGetLastError(), "targets");
    LP_CUDA(cudaStreamSynchronize(p->stream), "sync");
    m->stream = p->stream;
    k_gather<<<p->num_sms * 2, 256, 0, p->stream>>>(n_train, widx, feat, y, wfeat, wy);
    p->launches++;
    LP_CUDA(cudaGetLastError(), "training rows");
    LP_CUDA(cudaStreamSynchronize(p->stream), "sync");
    st = mlmc_mlp_train(m, reinterpret_cast<const uint16_t*>(wfeat), wy, n_train, steps, batch, lr,
                        seed ^ (0xABCDEFull + static_cast<uint64_t>(round)), final_loss);
    if (st == MLMC_OK) st = forward(m, feat, p->n, z);
    if (st == MLMC_OK) st = check_err(m);
    if (st != MLMC_OK) break;
    k_exp_h<<<g, 256, 0, p->stream>>>(p->n, z, h);
    p->launches++;
    LP_CUDA(cudaGetLastError(), "h");
    st = mlmc_plan_set_tilt(p, h, alpha, tilt_law);
  }
  if (st == MLMC_OK) {
    // The last round's tilt is measured like the others; if an earlier law
    // had the smaller variance, that one is installed instead.
    double xmax = 0.0, var = 0.0;
    LP_CUDA(pilot(next_rep, 4 * pilot_walks, &xmax, &var), "final pilot");
    next_rep += 4 * pilot_walks;
    int32_t last = static_cast<int32_t>(p->learn_var.size());
    // (kept: a time-piece law may be installed after it)
    LP_CUDA(consider(var, timed && max_warm_pieces > 1 ? h : nullptr, 1), "final");
    if (timed && max_warm_pieces > 1) {
      // The time-piece warm start (reading R19), walked last so that, when
      // it wins, its tables are the ones already built: K = min(8, 2^l0)
      // pieces, h_p the Taylor value of exp((1 - s_p) t|N|)|v| at the middle
      // s_p of piece p, the zero-variance h(s) = exp((1-s)tA)v that one law
      // can only average over time.  More pieces never measured a larger
      // variance, so only the largest is tried; it is installed when its
      // variance x walk time per walk is below the best single law's.
      const int32_t k_p = max_warm_pieces;
      k_piece_h<<<g, 256, 0, p->stream>>>(p->n, k_p, pv + 6 * p->n, pv + 8 * p->n, pv + 9 * p->n,
                                          pv + 10 * p->n, static_cast<float>(1e-3 * vmax + 1e-30), hp);
      p->launches++;
      LP_CUDA(cudaGetLastError(), "time-piece warm start");
      st = mlmc_plan_set_tilt_pieces(p, hp, k_p, alpha);
      if (st == MLMC_OK) {
        double xk = 0.0, vk = 0.0;
        LP_CUDA(pilot(next_rep, pilot_walks, &xk, &vk), "time-piece pilot");
        last = static_cast<int32_t>(p->learn_var.size());
        LP_CUDA(consider(vk, nullptr, k_p), "time-piece law");
      }
    }
    if (st != MLMC_OK) {
      // reported below
    } else if (p->learn_choice < 0)
      st = mfail(MLMC_ERR_NUMERIC, "mlmc_learn_tilt: no pilot measured a finite variance");
    else if (p->learn_choice != last && best_pieces > 1)
      st = mlmc_plan_set_tilt_pieces(p, best_h, best_pieces, alpha);
    else if (p->learn_choice != last)
      st = mlmc_plan_set_tilt(p, p->learn_choice == 0 && !clocks ? nullptr : best_h, alpha, tilt_law);
  }
  if (st != MLMC_OK) {
    const std::string msg = mlmc_last_error();
    restore();
    set_error(msg);  // the first failure's message, not the restore's
  }
  cleanup();
  return st;
#undef LP_CUDA
}

mlmc_status mlmc_plan_learn_report(const mlmc_plan* p, int32_t* chosen, double* var, int32_t cap,
                                   int32_t* count) {
  if (!p || (cap > 0 && !var) || cap < 0) return mfail(MLMC_ERR_INVALID_ARG, "mlmc_plan_learn_report: bad argument");
  const int32_t k = static_cast<int32_t>(p->learn_var.size());
  if (count) *count = k;
  if (chosen) *chosen = p->learn_choice;
  for (int32_t i = 0; i < k && i < cap; ++i) var[i] = p->learn_var[static_cast<size_t>(i)];
  return MLMC_OK;
}

}  // extern "C"
