// fxarith.cuh -- the integer arithmetic of the fixed-point passes (the
// single-problem pass in fxpass.cu and the batched pass in batched.cu).
//
// A value is held as a 55-bit integer relative to a binade bound `top`:
// v ~= F 2^(top - 1077), |F| < 2^55, with F = hi 2^28 + lo, 0 <= lo < 2^28,
// stored as int2 {lo, hi}.  Products of two such values are formed exactly
// from three 32 x 32 -> 64-bit multiply-adds (Karatsuba: hi*Xh,
// (hi + lo)*(Xh + Xl), lo*Xl), and sums are exact in 64- and 128-bit
// integers; the results are rounded to FP64 once, to nearest with ties to
// even.
#pragma once
#include <climits>
#include <cstdint>

namespace lsk {
namespace fx {

constexpr int kNoExp = INT_MIN;                 // "no nonzero value yet"

// |v| = M 2^(be - 1075), M < 2^53, be >= 1 (subnormals: be = 1, no implicit bit).
__device__ __forceinline__ void fx_decode(uint64_t bits, uint64_t& M, int& be) {
  const int e = (int)((bits >> 52) & 0x7FF);
  M = bits & 0xFFFFFFFFFFFFFull;
  if (e) M |= 1ull << 52;
  be = e ? e : 1;
}

// round(M 2^s) for s <= 2, ties to even.
__device__ __forceinline__ int64_t fx_round_shift(uint64_t M, int s) {
  if (s >= 0) return (int64_t)(M << s);
  const int r = -s;
  if (r > 53) return 0;                          // M / 2^r < 1/2
  const uint64_t q = M >> r;
  const uint64_t rem = M & ((1ull << r) - 1);
  const uint64_t half = 1ull << (r - 1);
  return (int64_t)(q + ((rem > half) || (rem == half && (q & 1ull))));
}

// Fixed point of the FP64 `bits` relative to the binade bound `top`
// (>= the value's be): v ~= F 2^(top - 1077), |F| < 2^55.
__device__ __forceinline__ int64_t fx_of(uint64_t bits, int top) {
  uint64_t M;
  int be;
  fx_decode(bits, M, be);
  const int64_t F = fx_round_shift(M, be - top + 2);
  return (bits >> 63) ? -F : F;
}

__device__ __forceinline__ int2 fx_limbs(int64_t F) {
  return make_int2((int)(F & 0x0FFFFFFF), (int)(F >> 28));
}

// c + a b, 32 x 32 -> 64-bit signed (one IMAD.WIDE).
__device__ __forceinline__ int64_t mad_wide(int a, int b, int64_t c) {
  int64_t d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// v 2^k for a finite double, exact unless the result leaves the normal range.
__device__ __forceinline__ double scale2(double v, int k) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  if (v == 0.0) return v;
  if (e != 0 && e + k >= 1 && e + k <= 2046)
    return __longlong_as_double((long long)(bits + ((uint64_t)(int64_t)k << 52)));
  return ldexp(v, k);
}

// Nearest FP64 to a 128-bit integer (two conversions and one FMA: within
// 1.5 units in the last place).
__device__ __forceinline__ double i128_to_double(__int128 s) {
  const long long hi = (long long)(s >> 64);
  const unsigned long long lo = (unsigned long long)s;
  return fma((double)hi, 0x1p64, (double)lo);
}

// Bit length of a nonzero 128-bit magnitude.
__device__ __forceinline__ int bitlen_u128(unsigned __int128 mag) {
  const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
  return hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
}

// The rounding of a normalised magnitude: |v| = N 2^(e - 127) with N the
// 128-bit value whose top 64 bits are Nh (bit 63 set) and whose lower bits
// are nonzero iff Ns.  fx_round53 gives the FP64 nearest to +-|v| when
// |v| is in [2^e, 2^(e+1)) (ties to even; outside the normal range ldexp);
// fx_round_norm gives round(|v| 2^(w - e - 1)) for the integer whose bit
// length is w <= 63 (the value N 2^(w - 128)), ties to even.
__device__ __forceinline__ double fx_round53(uint64_t Nh, bool Ns, bool neg, int e) {
  uint64_t q = Nh >> 11;
  const uint64_t rem = Nh & 0x7FFull;
  q += (rem > 0x400ull) || (rem == 0x400ull && (Ns || (q & 1ull)));
  if (q >> 53) { q >>= 1; e += 1; }
  const int be = e + 1023;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (q & 0xFFFFFFFFFFFFFull)));
  const double d = ldexp((double)q, e - 52);   // q is exact in FP64
  return neg ? -d : d;
}

__device__ __forceinline__ int64_t fx_round_norm(uint64_t Nh, bool Ns, int w) {
  if (w < 0) return 0;                           // below 1/2
  if (w == 0) return (Nh == (1ull << 63) && !Ns) ? 0 : 1;   // in [1/2, 1): a tie only at 1/2
  const int sh = 64 - w;
  const uint64_t q = Nh >> sh;
  const uint64_t rem = Nh & ((1ull << sh) - 1);
  const uint64_t half = 1ull << (sh - 1);
  return (int64_t)(q + ((rem > half) || (rem == half && (Ns || (q & 1ull)))));
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
  const unsigned long long lo = (unsigned long long)v;
  const long long hi = (long long)(v >> 64);
  const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
  const long long hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
  return ((__int128)hi2 << 64) | (__int128)lo2;
}

__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace fx
}  // namespace lsk
