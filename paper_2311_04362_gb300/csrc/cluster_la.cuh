// cluster_la.cuh -- small dense FP64 linear algebra on one thread-block
// cluster (8 or 16 CTAs x 256 threads, one CTA per SM).
//
// The n x n triangular factor R of the sketch is worked on by a cluster
// rather than one CTA: the FP64 rate of one SM (about 2 FMA per clock) makes
// an n = 1000 substitution take ~0.25 ms on one SM.  Vectors live in global
// memory (L2); every cross-CTA read uses ld.global.cg after a cluster barrier
// (release/acquire), so no L1 line can be stale.  Sums are taken in a fixed
// order (per-CTA trees, then CTA 0..P-1), so every result is bit-identical run
// to run and identical in all CTAs that compute it.
//
// Row blocks of 32 are owned block-cyclically: block b (rows 32b..32b+31)
// belongs to CTA b mod P.  A substitution solves the diagonal block on its
// owner (one warp, lanes = rows), publishes the 32 solved entries, and after
// one cluster barrier every CTA updates the right-hand side of the blocks it
// owns (right-looking), so there is one barrier per block.
#pragma once
#include "ls_internal.cuh"

namespace lsk {

struct CL {
  uint32_t rank, ncta;
};

__device__ inline CL cl_this() { return CL{cluster_rank(), cluster_nctas()}; }

__device__ inline void cl_sync() {
  __threadfence();
  cluster_sync();
}

// Deterministic CTA-wide sum of one value per thread (tree: warps, then warp 0).
__device__ inline double cta_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    s = warp_sum(s);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__device__ inline float cta_sum(float v) {
  __shared__ float red32[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red32[w] = v;
  __syncthreads();
  float s = 0.0f;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? red32[l] : 0.0f;
    s = warp_sum(s);
    if (l == 0) red32[0] = s;
  }
  __syncthreads();
  s = red32[0];
  __syncthreads();
  return s;
}

__device__ inline double cta_max(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// Cluster sum of one per-CTA value (all threads get the same result).
// `slots` holds ncta doubles of global scratch.
__device__ inline double cl_sum(const CL& cl, double cta_value, double* slots) {
  if (threadIdx.x == 0) __stcg(slots + cl.rank, cta_value);
  cl_sync();
  double s = 0.0;
  for (uint32_t r = 0; r < cl.ncta; ++r) s += __ldcg(slots + r);
  cl_sync();
  return s;
}

__device__ inline double cl_max(const CL& cl, double cta_value, double* slots) {
  if (threadIdx.x == 0) __stcg(slots + cl.rank, cta_value);
  cl_sync();
  double s = 0.0;
  for (uint32_t r = 0; r < cl.ncta; ++r) s = fmax(s, __ldcg(slots + r));
  cl_sync();
  return s;
}

// Index of the first entry of largest magnitude of x[0..n) (global, all
// entries valid); ties go to the smaller index.
__device__ inline int cl_argmax_abs(const CL& cl, int n, const double* x, double* slots) {
  __shared__ double sv[256];
  __shared__ int si[256];
  double bv = -1.0;
  int bi = 0x7fffffff;
  const int nb = (n + 31) / 32;
  for (int b = cl.rank; b < nb; b += cl.ncta) {
    for (int i = 32 * b + (int)threadIdx.x; i < min(n, 32 * b + 32); i += blockDim.x) {
      const double v = fabs(__ldcg(x + i));
      if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double v2 = sv[threadIdx.x + o];
      const int i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __stcg(slots + 2 * cl.rank, sv[0]);
    __stcg(slots + 2 * cl.rank + 1, (double)si[0]);
  }
  cl_sync();
  double best = -1.0;
  int besti = 0x7fffffff;
  for (uint32_t r = 0; r < cl.ncta; ++r) {
    const double v = __ldcg(slots + 2 * r);
    const int i = (int)__ldcg(slots + 2 * r + 1);
    if (v > best || (v == best && i < besti)) { best = v; besti = i; }
  }
  cl_sync();
  return besti;
}

// Iterate over the rows of the blocks this CTA owns: f(i).
template <class F>
__device__ inline void for_owned_rows(const CL& cl, int n, F f) {
  const int nb = (n + 31) / 32;
  const int mine = (nb - (int)cl.rank + (int)cl.ncta - 1) / (int)cl.ncta;  // blocks owned
  for (int idx = threadIdx.x; idx < mine * 32; idx += blockDim.x) {
    const int b = (int)cl.rank + (idx >> 5) * (int)cl.ncta;
    const int i = 32 * b + (idx & 31);
    if (i < n) f(i);
  }
}

// Solve R^T y = rhs (R upper, so R^T lower) by blocked forward substitution.
// Rt[a + b*n] = R[b, a].  On entry work[i] = rhs_i for the rows this CTA
// owns; on exit y[0..n) holds the solution (every entry written by its
// owner, visible cluster-wide).  Ends with a cluster barrier.
__device__ inline void cl_solve_RT(const CL& cl, const double* __restrict__ Rt, int n,
                                   const double* __restrict__ inv_diag, double* work, double* y) {
  __shared__ double yb[32];
  const int nb = (n + 31) / 32;
  for (int b = 0; b < nb; ++b) {
    const int r0 = 32 * b, bs = min(32, n - r0);
    if ((uint32_t)(b % (int)cl.ncta) == cl.rank && threadIdx.x < 32) {
      // lane l holds row l of the diagonal block of R^T (one wave of loads)
      const int l = threadIdx.x;
      double rowv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        rowv[i] = (l < bs && i < l) ? __ldg(Rt + (size_t)(r0 + l) + (size_t)(r0 + i) * n) : 0.0;
      const double inv = (l < bs) ? __ldg(inv_diag + r0 + l) : 0.0;
      double wl = (l < bs) ? __ldcg(work + r0 + l) : 0.0;
      double yl = 0.0;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const double yi = __shfl_sync(0xffffffffu, wl * inv, i);
        if (l == i) yl = yi;
        if (l > i) wl = wl - rowv[i] * yi;
      }
      if (l < bs) __stcg(y + r0 + l, yl);
    }
    cl_sync();
    if ((int)threadIdx.x < bs) yb[threadIdx.x] = __ldcg(y + r0 + threadIdx.x);
    __syncthreads();
    for_owned_rows(cl, n, [&](int i) {
      if (i >= r0 + 32) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k < bs) s += __ldg(Rt + (size_t)i + (size_t)(r0 + k) * n) * yb[k];
        __stcg(work + i, __ldcg(work + i) - s);
      }
    });
    __syncthreads();
  }
  cl_sync();
}

// Solve R x = rhs by blocked back substitution; R column-major (ldr).
// Same contract as cl_solve_RT (work holds the owned rhs entries).
__device__ inline void cl_solve_R(const CL& cl, const double* __restrict__ R, int64_t ldr, int n,
                                  const double* __restrict__ inv_diag, double* work, double* x) {
  __shared__ double xb[32];
  const int nb = (n + 31) / 32;
  for (int b = nb - 1; b >= 0; --b) {
    const int r0 = 32 * b, bs = min(32, n - r0);
    if ((uint32_t)(b % (int)cl.ncta) == cl.rank && threadIdx.x < 32) {
      // lane l holds row l of the diagonal block of R (one wave of loads)
      const int l = threadIdx.x;
      double rowv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        rowv[i] = (l < bs && i > l && i < bs) ? __ldg(R + (size_t)(r0 + l) + (size_t)(r0 + i) * ldr) : 0.0;
      const double inv = (l < bs) ? __ldg(inv_diag + r0 + l) : 0.0;
      double wl = (l < bs) ? __ldcg(work + r0 + l) : 0.0;
      double xl = 0.0;
#pragma unroll
      for (int i = 31; i >= 0; --i) {
        const double xi = __shfl_sync(0xffffffffu, wl * inv, i);
        if (l == i) xl = xi;
        if (l < i) wl = wl - rowv[i] * xi;
      }
      if (l < bs) __stcg(x + r0 + l, xl);
    }
    cl_sync();
    if ((int)threadIdx.x < bs) xb[threadIdx.x] = __ldcg(x + r0 + threadIdx.x);
    __syncthreads();
    for_owned_rows(cl, n, [&](int i) {
      if (i < r0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k < bs) s += __ldg(R + (size_t)i + (size_t)(r0 + k) * ldr) * xb[k];
        __stcg(work + i, __ldcg(work + i) - s);
      }
    });
    __syncthreads();
  }
  cl_sync();
}

// Copy src (all entries valid cluster-wide) into work for the owned rows.
__device__ inline void cl_load_owned(const CL& cl, int n, const double* src, double* work) {
  for_owned_rows(cl, n, [&](int i) { __stcg(work + i, __ldcg(src + i)); });
  __syncthreads();
}

// Euclidean norm of v[0..n) (all entries valid).
__device__ inline double cl_norm2(const CL& cl, int n, const double* v, double* slots) {
  double s = 0.0;
  for_owned_rows(cl, n, [&](int i) { const double t = __ldcg(v + i); s += t * t; });
  return sqrt(cl_sum(cl, cta_sum(s), slots));
}

__device__ inline double cl_norm1(const CL& cl, int n, const double* v, double* slots) {
  double s = 0.0;
  for_owned_rows(cl, n, [&](int i) { s += fabs(__ldcg(v + i)); });
  return cl_sum(cl, cta_sum(s), slots);
}

// Power-method and 1-norm estimator helpers shared by the single-problem and
// batched post-factor kernels.
__device__ inline double sgn1(double v) { return v >= 0.0 ? 1.0 : -1.0; }

__device__ inline double power_start(uint64_t seed, uint32_t domain, int i) {
  WordStream s(seed, (uint64_t)i, domain);
  const uint32_t w0 = s.next(), w1 = s.next();
  const uint64_t bits = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
  return 2.0 * ((double)bits * 0x1.0p-53) - 1.0;
}

// w = R v (rows i of R, from Rt) for owned rows.
__device__ inline void cl_matvec_R(const CL& cl, const double* Rt, int n, const double* v, double* w) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nb = (n + 31) / 32;
  for (int b = cl.rank; b < nb; b += cl.ncta)
    for (int i = 32 * b + warp; i < min(n, 32 * b + 32); i += nw) {
      double s = 0.0;
      for (int k = i + lane; k < n; k += 32) s += __ldg(Rt + (size_t)k + (size_t)i * n) * __ldcg(v + k);
      s = warp_sum(s);
      if (lane == 0) __stcg(w + i, s);
    }
}

// v = R^T w (column i of R) for owned rows.
__device__ inline void cl_matvec_RT(const CL& cl, const double* R, int64_t ldr, int n, const double* w, double* v) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nb = (n + 31) / 32;
  for (int b = cl.rank; b < nb; b += cl.ncta)
    for (int i = 32 * b + warp; i < min(n, 32 * b + 32); i += nw) {
      double s = 0.0;
      for (int k = lane; k <= i; k += 32) s += __ldg(R + (size_t)k + (size_t)i * ldr) * __ldcg(w + k);
      s = warp_sum(s);
      if (lane == 0) __stcg(v + i, s);
    }
}

__device__ inline int power_steps(int n) {
  int k = 0;
  while (k < 64 && exp((double)k) < (double)n) ++k;
  return k < 1 ? 1 : k;
}

}  // namespace lsk
