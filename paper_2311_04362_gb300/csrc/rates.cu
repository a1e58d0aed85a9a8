// rates.cu -- instruction-throughput probe for the roofline of the fused pass
// (built as librates.so, separate from libls.so; bench.py --rates runs it).
//
// Each probe kernel runs one CTA of 1024 threads per SM; every thread keeps
// eight independent dependency chains of one instruction form and repeats
// them `iters` times.  The CTA reads %clock64 around its loop, so the result
// is the SM's sustained rate of that form in thread-operations per SM clock
// (an FP64 FMA counts as one operation).  The printed forms are the ones the
// pass can be built from: FP64 FMA, FP32 FMA, the 32-bit integer multiply
// forms (low, high, 32x32->64 wide), the carry chain of a multi-word add,
// LOP3, funnel shift, byte permute, and the conversions between widths.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

namespace {

enum Op {
  kDfma, kFfma, kImadLo, kImadHi, kImadWide, kImadWideU, kMadCc96, kLop3, kShf, kPrmt, kIadd64, kF2fF32F64,
  kI2fF64S64, kI2fF32S32, kNumOps
};
const char* kNames[kNumOps] = {"dfma",       "ffma",         "imad_lo",     "imad_hi",      "imad_wide_s32",
                               "imad_wide_u32", "mad_cc_96bit_x3", "lop3",     "shf",          "prmt",
                               "add_u64_x2",    "cvt_f32_f64",  "cvt_f64_s64", "cvt_f32_s32"};
// operations per chain step (a step may be several instructions)
const int kOpsPerStep[kNumOps] = {1, 1, 1, 1, 1, 1, 3, 1, 1, 1, 2, 1, 1, 1};

template <int OP>
__global__ void __launch_bounds__(1024, 1) k_rate(int iters, uint32_t seed, unsigned long long* cycles, uint32_t* sink) {
  uint32_t a = seed ^ threadIdx.x, b = seed * 2654435761u + 1u;
  uint32_t v[8], w[8], z[8];
  uint64_t q[8];
  double dv[8];
  float fv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = a + i; w[i] = b ^ i; z[i] = 0; q[i] = ((uint64_t)v[i] << 20) | w[i];
    dv[i] = 1.0 + 1e-9 * i; fv[i] = 1.0f + 1e-6f * i;
  }
  const double dm = 0.999999999, da = 1e-12;
  const float fm = 0.9999f, fa = 1e-7f;
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (OP == kDfma) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(dv[i]) : "d"(dm), "d"(da));
      if (OP == kFfma) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(fv[i]) : "f"(fm), "f"(fa));
      if (OP == kImadLo) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v[i]) : "r"(b), "r"(a));
      if (OP == kImadHi) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(v[i]) : "r"(b), "r"(a));
      if (OP == kImadWide) {
        asm volatile("mad.wide.s32 %0, %1, %2, %0;" : "+l"(q[i]) : "r"(v[i]), "r"(b));
      }
      if (OP == kImadWideU) {
        asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(q[i]) : "r"(v[i]), "r"(b));
      }
      if (OP == kMadCc96)
        asm volatile("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
                     : "+r"(w[i]), "+r"(z[i]), "+r"(v[i])
                     : "r"(a), "r"(b));
      if (OP == kLop3) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[i]) : "r"(a), "r"(b));
      if (OP == kShf) asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;" : "+r"(v[i]) : "r"(w[i]), "r"(a));
      if (OP == kPrmt) asm volatile("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(v[i]) : "r"(b));
      if (OP == kIadd64) asm volatile("add.u64 %0, %0, %1;" : "+l"(q[i]) : "l"((uint64_t)b << 7));
      if (OP == kF2fF32F64) {
        float f;
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(dv[i]));
        v[i] ^= __float_as_uint(f);
        dv[i] = __longlong_as_double(__double_as_longlong(dv[i]) ^ (long long)(v[i] & 1u));
      }
      if (OP == kI2fF64S64) {
        double d;
        asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(d) : "l"(q[i]));
        q[i] += (uint64_t)__double_as_longlong(d);
      }
      if (OP == kI2fF32S32) {
        float f;
        asm volatile("cvt.rn.f32.s32 %0, %1;" : "=f"(f) : "r"(v[i]));
        v[i] += __float_as_uint(f);
      }
    }
  }
  const unsigned long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    acc ^= v[i] ^ w[i] ^ z[i] ^ (uint32_t)q[i] ^ (uint32_t)(q[i] >> 32) ^ __float_as_uint(fv[i]) ^
           (uint32_t)__double_as_longlong(dv[i]);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
int run_one(int sms, int iters, unsigned long long* d_cyc, uint32_t* d_sink, double* rate_clk, double* rate_ns,
            int threads = 1024) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_rate<OP><<<sms, threads>>>(8, 1u, d_cyc, d_sink);   // warm-up
  cudaEventRecord(e0);
  k_rate<OP><<<sms, threads>>>(iters, 1u, d_cyc, d_sink);
  cudaEventRecord(e1);
  if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long* h = new unsigned long long[sms];
  cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
  double cyc = 0;
  for (int i = 0; i < sms; ++i) cyc += (double)h[i];
  cyc /= sms;
  delete[] h;
  const double ops_per_cta = (double)threads * 8.0 * iters * kOpsPerStep[OP];
  *rate_clk = ops_per_cta / cyc;
  *rate_ns = ops_per_cta * sms / (ms * 1e6);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() != cudaSuccess;
}

template <int OP>
int run_upto(int sms, int iters, unsigned long long* c, uint32_t* s, double* rc, double* rn) {
  int err = 0;
  if constexpr (OP > 0) err |= run_upto<OP - 1>(sms, iters, c, s, rc, rn);
  err |= run_one<OP>(sms, iters, c, s, rc + OP, rn + OP);
  return err;
}

}  // namespace

// Writes one JSON object into out: {"sms": N, "rates": {"<form>": [per SM
// clock, per ns on the GPU], ...}}.  Returns 0 on success.
extern "C" __attribute__((visibility("default"))) int ls_probe_rates(char* out, int out_len, int iters) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  unsigned long long* d_cyc = nullptr;
  uint32_t* d_sink = nullptr;
  if (cudaMalloc(&d_cyc, sizeof(unsigned long long) * sms) != cudaSuccess) return 1;
  if (cudaMalloc(&d_sink, sizeof(uint32_t) * 1024 * sms) != cudaSuccess) return 1;
  double rc[kNumOps] = {0}, rn[kNumOps] = {0};
  int err = run_upto<kNumOps - 1>(sms, iters, d_cyc, d_sink, rc, rn);
  // the same forms with fewer warps per SM (one CTA of 128, 256, 512 threads):
  // what a kernel with 1, 2 or 4 warps per sub-partition issuing them gets
  const int occ[3] = {128, 256, 512};
  double wide[3], ffma[3], dfma[3];
  for (int i = 0; i < 3; ++i) {
    double dummy;
    err |= run_one<kImadWide>(sms, iters, d_cyc, d_sink, &wide[i], &dummy, occ[i]);
    err |= run_one<kFfma>(sms, iters, d_cyc, d_sink, &ffma[i], &dummy, occ[i]);
    err |= run_one<kDfma>(sms, iters, d_cyc, d_sink, &dfma[i], &dummy, occ[i]);
  }
  cudaFree(d_cyc);
  cudaFree(d_sink);
  int pos = snprintf(out, out_len, "{\"sms\": %d, \"iters\": %d, \"rates\": {", sms, iters);
  for (int i = 0; i < kNumOps && pos < out_len; ++i)
    pos += snprintf(out + pos, out_len - pos, "%s\"%s\": [%.3f, %.2f]", i ? ", " : "", kNames[i], rc[i], rn[i]);
  if (pos < out_len)
    pos += snprintf(out + pos, out_len - pos,
                    "}, \"by_threads_per_sm\": {\"threads\": [128, 256, 512, 1024], "
                    "\"imad_wide_s32\": [%.3f, %.3f, %.3f, %.3f], \"ffma\": [%.3f, %.3f, %.3f, %.3f], "
                    "\"dfma\": [%.3f, %.3f, %.3f, %.3f]}",
                    wide[0], wide[1], wide[2], rc[kImadWide], ffma[0], ffma[1], ffma[2], rc[kFfma], dfma[0], dfma[1],
                    dfma[2], rc[kDfma]);
  if (pos < out_len) snprintf(out + pos, out_len - pos, "}");
  return err;
}
