// Host build of the fixed-point passes' integer arithmetic
// (paper_2311_04362_gb300/csrc/fxarith.cuh, included as it is) for the CPU
// tests: the few CUDA names it uses are given host meanings here, and a C
// interface exposes the rounding steps to ctypes.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>

#define __device__
#define __forceinline__ inline
struct int2 { int x, y; };
static inline int2 make_int2(int a, int b) { return int2{a, b}; }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
static inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
static inline int __clzll(long long v) { return v ? __builtin_clzll((unsigned long long)v) : 64; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
using std::max;

#include "../paper_2311_04362_gb300/csrc/fxarith.cuh"

using namespace lsk::fx;

extern "C" {
int64_t fxh_of(uint64_t bits, int top) { return fx_of(bits, top); }
int64_t fxh_round_shift(uint64_t M, int s) { return fx_round_shift(M, s); }
void fxh_limbs(int64_t F, int* lo, int* hi) { const int2 l = fx_limbs(F); *lo = l.x; *hi = l.y; }
int fxh_bitlen(uint64_t hi, uint64_t lo) { return bitlen_u128(((unsigned __int128)hi << 64) | lo); }
uint64_t fxh_round53(uint64_t Nh, int Ns, int neg, int e) {
  return (uint64_t)__double_as_longlong(fx_round53(Nh, Ns != 0, neg != 0, e));
}
int64_t fxh_round_norm(uint64_t Nh, int Ns, int w) { return fx_round_norm(Nh, Ns != 0, w); }
}
