// fixedpoint.cuh -- exact accumulation of FP64 products on the integer pipe.
//
// GB300 executes about 2 FP64 FMAs per clock per SM but ~128 integer ops, so
// the c = A^T r half of the fused pass is done with integers: each product
// a * r of two doubles is formed from the 53-bit significands (64x64-bit high
// multiply), aligned to a per-column anchor and added to a 128-bit two's
// complement accumulator.  Partial accumulators of all CTAs are summed
// exactly (192-bit) and rounded once to the nearest double, so the result is
// the correctly rounded value of the sum of the (truncated) products, in any
// order.  Truncation: each product keeps its top 64 of 106 significand bits
// (relative error < 2^-62) and bits below the accumulator's unit 2^(E-100)
// are dropped, E being an upper bound of log2 |a r| for the column.
#pragma once
#include <stdint.h>

namespace lsk {

// Unit exponent of the accumulator window below the anchor E (products are
// at most 2^E = 2^100 units; 2^24 of them stay below 2^124).
static constexpr int kFxWindow = 100;

struct Fx128 {
  uint64_t lo, hi;
};

__device__ inline void fx_add(Fx128& a, uint64_t vlo, uint64_t vhi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(vlo), "l"(vhi));
}

// Decompose a double into (biased exponent, 53-bit significand); exponent 0
// means zero or subnormal (treated as zero), 0x7FF means inf/nan.
__device__ inline void fx_split(double v, int& ebiased, uint64_t& mant, uint32_t& sign) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  sign = (uint32_t)(bits >> 63);
  ebiased = (int)((bits >> 52) & 0x7FF);
  mant = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
}

// acc += sign(a r) * (top 64 bits of |ma mr|) aligned so that the value of
// one accumulator unit is 2^(W0); ea, er are unbiased exponents.
// Precondition: ea + er - 62 - W0 <= 36 (the caller's anchor guarantees it).
__device__ inline void fx_mac(Fx128& acc, uint64_t ma, int ea, uint32_t sa, uint64_t mr_shifted, int er,
                              uint32_t sr, int W0) {
  const uint64_t t = __umul64hi(ma << 11, mr_shifted);   // (ma * mr) >> 42, in [2^62, 2^64)
  const int L = ea + er - 62 - W0;
  uint64_t vlo, vhi;
  if (L >= 0) {
    vlo = t << L;
    vhi = (L == 0) ? 0ull : (t >> (64 - L));
  } else {
    vlo = (L > -64) ? (t >> (-L)) : 0ull;
    vhi = 0ull;
  }
  const uint64_t neg = (uint64_t)0 - (uint64_t)(sa ^ sr);   // all ones if negative
  vlo ^= neg;
  vhi ^= neg;
  fx_add(acc, vlo, vhi);
  fx_add(acc, neg & 1ull, 0ull);                             // two's complement: + 1
}

// 192-bit signed sum of 128-bit accumulators.
struct Fx192 {
  uint64_t w0, w1, w2;
};
__device__ inline void fx192_add128(Fx192& s, uint64_t lo, uint64_t hi) {
  const uint64_t ext = (uint64_t)((int64_t)hi >> 63);       // sign extension
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(s.w0), "+l"(s.w1), "+l"(s.w2)
      : "l"(lo), "l"(hi), "l"(ext));
}

// Round s * 2^W0 to the nearest double (ties to even).
__device__ inline double fx192_to_double(Fx192 s, int W0) {
  const bool negv = ((int64_t)s.w2) < 0;
  if (negv) {   // magnitude
    s.w0 = ~s.w0; s.w1 = ~s.w1; s.w2 = ~s.w2;
    asm("add.cc.u64 %0, %0, 1;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
        : "+l"(s.w0), "+l"(s.w1), "+l"(s.w2));
  }
  int p;   // position of the leading one
  uint64_t top, rest_nz;
  if (s.w2) {
    const int z = __clzll(s.w2);
    p = 191 - z;
  } else if (s.w1) {
    p = 127 - __clzll(s.w1);
  } else if (s.w0) {
    p = 63 - __clzll(s.w0);
  } else {
    return 0.0;
  }
  // window of 64 bits ending at p: bits [p-63, p]
  auto bitword = [&](int lo) -> uint64_t {    // 64 bits starting at bit `lo` (lo may be negative)
    uint64_t w[3] = {s.w0, s.w1, s.w2};
    if (lo <= -64) return 0ull;
    if (lo < 0) return w[0] << (-lo);
    const int q = lo >> 6, r = lo & 63;
    const uint64_t a = (q < 3) ? w[q] : 0ull;
    const uint64_t b = (q + 1 < 3) ? w[q + 1] : 0ull;
    return r ? ((a >> r) | (b << (64 - r))) : a;
  };
  top = bitword(p - 63);                      // leading one at bit 63
  // sticky: any set bit below p-63
  rest_nz = 0ull;
  if (p - 63 > 0) {
    const int lo = p - 63;
    const int q = lo >> 6, r = lo & 63;
    uint64_t w[3] = {s.w0, s.w1, s.w2};
    for (int i = 0; i < q && i < 3; ++i) rest_nz |= w[i];
    if (q < 3 && r) rest_nz |= (w[q] & ((1ull << r) - 1ull));
  }
  uint64_t mant = top >> 11;                   // 53 bits
  const uint64_t round_bit = (top >> 10) & 1ull;
  const uint64_t sticky = ((top & 0x3FFull) != 0ull) || rest_nz;
  if (round_bit && (sticky || (mant & 1ull))) mant += 1ull;
  int e = p - 52 + W0;                          // value = mant * 2^e
  const double v = scalbn((double)mant, e);
  return negv ? -v : v;
}

}  // namespace lsk
