// Device primitives of the MLMC walk: Philox4x32-10, uniforms, -ln(u), and
// the packed table layouts.  Every floating-point step uses an explicit
// round-to-nearest intrinsic (no FMA contraction), so a walk's decisions are
// a fixed function of its counter and can be replayed exactly on a CPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

// ---------------------------------------------------------------------------
// Table layouts (device)
// ---------------------------------------------------------------------------
// Per-row record for the FP32 walk: alias row start (= CSR row start),
// off-diagonal count, 1/(t L_ii) and t d_i (Eq. 1, scaled time).  16 bytes:
// one LDG.128 per visited state.
struct __align__(16) Meta32 {
  int32_t start;
  int32_t deg;
  float inv_rate;
  float dl;
};

// Per-row record for the FP64 walk (32 bytes, one sector).
struct __align__(16) Meta64 {
  int32_t start;
  int32_t deg;
  int32_t pad0;
  int32_t pad1;
  double inv_rate;
  double dl;
};

// Alias entry (16 bytes, one LDG.128 per jump): threshold, kept column and
// alias column, each column with the sign of a_ij in bit 31.
// While a row's table is being built the same 16 bytes hold the bucket's
// working probability (double) and the next-bucket link of the Vose queue.
struct __align__(16) AliasEntry {
  uint32_t thr;
  uint32_t keep;
  uint32_t alias;
  uint32_t pad;
};

// Alias entry of an importance-sampling proposal (32 bytes, one sector):
// the plain entry plus log(k/q) of the kept and of the alias column, where
// k is the paper's jump law and q the proposal.
struct __align__(16) AliasEntryIS {
  uint32_t thr;
  uint32_t keep;
  uint32_t alias;
  uint32_t pad;
  float lr_keep;
  float lr_alias;
  uint32_t pad1;
  uint32_t pad2;
};

// Fused alias entry of the walk: the plain entry followed by the row records
// of its kept and its alias column, so that a jump reads the next state's
// record together with the entry (independent loads from one entry, one
// round trip to L2) instead of after it.  48 bytes (FP32), 80 bytes (FP64).
struct __align__(16) FusedEntry32 {
  uint32_t thr;
  uint32_t keep;
  uint32_t alias;
  uint32_t pad;
  Meta32 mk;
  Meta32 ma;
};
struct __align__(16) FusedEntry64 {
  uint32_t thr;
  uint32_t keep;
  uint32_t alias;
  uint32_t pad;
  Meta64 mk;
  Meta64 ma;
};

constexpr uint32_t kSignBit = 0x80000000u;
constexpr uint32_t kColMask = 0x7FFFFFFFu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    // one 32 x 32 -> 64-bit product per multiplier (high and low words)
    const unsigned long long p0 = static_cast<unsigned long long>(kPhiloxM0) * c.x;
    const unsigned long long p1 = static_cast<unsigned long long>(kPhiloxM1) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
  }
  return c;
}

// The ten round keys of one Philox key: (k0 + r W0, k1 + r W1), r = 0..9.  A
// launch passes them as a constant kernel parameter so that each round xors
// its key straight from the parameter bank instead of forming it.
struct PhiloxRoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
    rk.k1[r] = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = static_cast<unsigned long long>(kPhiloxM0) * c.x;
    const unsigned long long p1 = static_cast<unsigned long long>(kPhiloxM1) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ rk.k0[r], static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ rk.k1[r], static_cast<uint32_t>(p0));
  }
  return c;
}

// ---------------------------------------------------------------------------
// Uniforms in (0,1): odd multiples of 2^-53 (FP64) or 2^-24 (FP32), exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double uniform64(uint32_t x0, uint32_t x1) {
  const unsigned long long w = (static_cast<unsigned long long>(x0) << 32) | x1;
  return __dmul_rn(__ull2double_rn((w >> 11) | 1ull), 0x1p-53);
}

__device__ __forceinline__ float uniform32(uint32_t x0) {
  return __fmul_rn(__uint2float_rn((x0 >> 8) | 1u), 0x1p-24f);
}

// ---------------------------------------------------------------------------
// -ln(u) for normal u in (0,1).
// u = m 2^e, m in [sqrt(1/2), sqrt(2)); ln u = e ln2_hi + (e ln2_lo + ln m),
// ln2_hi with trailing zero bits so the product is exact.
// FP64: ln m = 2 atanh(z) = 2 z sum_k z^{2k}/(2k+1) with z = (m-1)/(m+1),
// |z| <= 0.1716, 12 terms; the coefficients are 1/(2k+1) correctly rounded
// and the host checks these literals against its own IEEE division at
// library load.
// FP32: ln m = f + f^2 Q(f), f = m - 1 (exact), Q of degree 8 by Horner's
// rule with fused multiply-adds.  Q's coefficients are the FP64
// least-squares fit of the relative error of f + f^2 Q(f) against ln(1+f) on
// 1000 Chebyshev (Gauss) points of [sqrt(1/2) - 1, sqrt(2) - 1], each rounded
// to FP32; the result is within 0.87 ulp of -ln(u) and strictly decreasing
// over all 2^23 FP32 uniforms (2i+1) 2^-24.
// ---------------------------------------------------------------------------
constexpr double kLn2Hi64 = 0x1.62e42fefa3800p-1;
constexpr double kLn2Lo64 = 0x1.ef35793c76730p-45;
constexpr float kLn2Hi32 = 0x1.62e400p-1f;
constexpr float kLn2Lo32 = 0x1.7f7d1cp-20f;
constexpr double kSqrtHalf64 = 0x1.6a09e667f3bcdp-1;
constexpr float kSqrtHalf32 = 0x1.6a09e6p-1f;

constexpr int kNeglogTerms64 = 12;
constexpr int kNeglogDeg32 = 8;

__host__ __device__ constexpr double neglog_c64(int k) {
  constexpr double c[kNeglogTerms64] = {
      0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
      0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4,
      0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5};
  return c[k];
}

__host__ __device__ constexpr float neglog_q32(int k) {
  constexpr float c[kNeglogDeg32 + 1] = {-0x1.fffff8p-2f, 0x1.555558p-2f, -0x1.000422p-2f,
                                         0x1.999fc2p-3f,  -0x1.5424e0p-3f, 0x1.22bf86p-3f,
                                         -0x1.0f9b0cp-3f, 0x1.068b2ap-3f,  -0x1.321a4cp-4f};
  return c[k];
}

__device__ __forceinline__ double neglog64(double u) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(u));
  int e = static_cast<int>((b >> 52) & 0x7ffull) - 1022;
  double m = __longlong_as_double(
      static_cast<long long>((b & 0x000fffffffffffffull) | (0x3feull << 52)));
  if (m < kSqrtHalf64) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z2 = __dmul_rn(z, z);
  double p = neglog_c64(kNeglogTerms64 - 1);
#pragma unroll
  for (int k = kNeglogTerms64 - 2; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, z2), neglog_c64(k));
  const double lnm = __dmul_rn(__dmul_rn(2.0, z), p);
  const double ed = static_cast<double>(e);
  const double lnu = __dadd_rn(__dmul_rn(ed, kLn2Hi64), __dadd_rn(__dmul_rn(ed, kLn2Lo64), lnm));
  return -lnu;
}

__device__ __forceinline__ float neglog32(float u) {
  const uint32_t b = __float_as_uint(u);
  int e = static_cast<int>((b >> 23) & 0xffu) - 126;
  float m = __uint_as_float((b & 0x007fffffu) | (0x7eu << 23));
  if (m < kSqrtHalf32) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  float q = neglog_q32(kNeglogDeg32);
#pragma unroll
  for (int k = kNeglogDeg32 - 1; k >= 0; --k) q = __fmaf_rn(q, f, neglog_q32(k));
  const float lnm = __fmaf_rn(__fmul_rn(f, f), q, f);
  const float ef = static_cast<float>(e);
  const float lnu = __fmaf_rn(ef, kLn2Hi32, __fmaf_rn(ef, kLn2Lo32, lnm));
  return -lnu;
}

// FP32 walks: the largest uniform index i (u = (2i+1) 2^-24, i < 2^23) whose
// first holding time fl(-ln(u)) / (t L_row) reaches s = 1, or -1 if none.  The
// holding time is non-increasing in i (the FP32 -ln(u) is strictly
// decreasing over all 2^23 uniforms, an exhaustive host check of the same
// arithmetic, and rounding a product with a positive factor is monotone), so
// a walk never jumps exactly when its index is <= the returned one.  The 32
// lanes test 32 points of the open interval per round: the passing points
// form a prefix, and an interval of at most 33 points is settled in one
// round (5 rounds from 2^23).
__device__ __forceinline__ int32_t still_index32(float inv_rate, int lane) {
  int32_t lo = -1, hi = 1 << 23;  // the test holds at lo (or lo = -1), fails at hi (or hi = 2^23)
  while (hi - lo > 1) {
    const int64_t width = hi - lo;
    const int32_t c = lo + static_cast<int32_t>((static_cast<int64_t>(lane + 1) * width) / 33);
    bool pass;
    if (c <= lo) {
      pass = true;
    } else if (c >= hi) {
      pass = false;
    } else {
      const float u = __fmul_rn(__uint2float_rn(2u * static_cast<uint32_t>(c) + 1u), 0x1p-24f);
      pass = !(__fmul_rn(neglog32(u), inv_rate) < 1.0f);
    }
    const int t = __popc(__ballot_sync(0xFFFFFFFFu, pass));
    const int32_t c_last = __shfl_sync(0xFFFFFFFFu, c, t > 0 ? t - 1 : 0);
    const int32_t c_first_fail = __shfl_sync(0xFFFFFFFFu, c, t < 32 ? t : 31);
    if (t > 0 && c_last > lo) lo = c_last;
    if (t < 32 && c_first_fail < hi) hi = c_first_fail;
  }
  return lo;
}

// still_index32 for a law with K time pieces (reading R19): the first
// holding time E / rate_0, carried over each piece boundary b = (p+1)/K it
// reaches as b + (s - b) * ir[p+1] / ir[p] (infinite when either inverse
// rate is), must reach s = 1.  The carried time does not decrease with E,
// so the passing indices still form a prefix.
__device__ __forceinline__ bool still_pieces32(float u, const float* ir, int k_pieces, float inv_k) {
  float s = __fmul_rn(neglog32(u), ir[0]);
  for (int p = 0; p + 1 < k_pieces; ++p) {
    const float b = __fmul_rn(static_cast<float>(p + 1), inv_k);
    if (!(s >= b)) break;
    s = (isinf(ir[p]) || isinf(ir[p + 1])) ? __int_as_float(0x7f800000)
                                           : __fmaf_rn(__fsub_rn(s, b), __fdiv_rn(ir[p + 1], ir[p]), b);
  }
  return !(s < 1.0f);
}

__device__ __forceinline__ int32_t still_index32_pieces(const float* ir, int k_pieces, float inv_k,
                                                        int lane) {
  int32_t lo = -1, hi = 1 << 23;
  while (hi - lo > 1) {
    const int64_t width = hi - lo;
    const int32_t c = lo + static_cast<int32_t>((static_cast<int64_t>(lane + 1) * width) / 33);
    bool pass;
    if (c <= lo) {
      pass = true;
    } else if (c >= hi) {
      pass = false;
    } else {
      const float u = __fmul_rn(__uint2float_rn(2u * static_cast<uint32_t>(c) + 1u), 0x1p-24f);
      pass = still_pieces32(u, ir, k_pieces, inv_k);
    }
    const int t = __popc(__ballot_sync(0xFFFFFFFFu, pass));
    const int32_t c_last = __shfl_sync(0xFFFFFFFFu, c, t > 0 ? t - 1 : 0);
    const int32_t c_first_fail = __shfl_sync(0xFFFFFFFFu, c, t < 32 ? t : 31);
    if (t > 0 && c_last > lo) lo = c_last;
    if (t < 32 && c_first_fail < hi) hi = c_first_fail;
  }
  return lo;
}

}  // namespace mlmc
