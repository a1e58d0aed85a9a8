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


// ------------------------------------------------- broadcast substitutions
// The per-iteration pair of solves R^T y = c, R d = y (Algorithm 2's
// preconditioned step) without a cluster-wide barrier inside a solve.
//
// Blocks of 32 rows are owned as above (block b by CTA b mod P) and, inside
// the CTA, by warp pair q = (b / P) mod 4: warp 2q holds the row's sum over
// columns 0..15 of every off-diagonal block, warp 2q+1 over columns 16..31
// (a lane per row).  When block k's 32 solved entries land in a CTA's shared
// memory (one mbarrier per block, completed by the bytes themselves), every
// pair folds them into the rows it still has to solve.  The pair owning the
// next block does so as soon as they land, adds its two halves, solves its
// diagonal block in one warp and pushes the 32 results into every CTA with
// st.async.  The operand slices of R for the next block are loaded while
// the current one is waited for.
//
// Every row's inner product is summed in a fixed order (block by block, two
// interleaved chains per half, then half 0 + half 1), so results are
// reproducible; any fixed order keeps the substitution backward stable.
//
// A diagonal block D is solved as the unit-triangular system with D's
// off-diagonal entries divided by their pivots (D = U diag(D) for R^T, the
// columns of R for R itself), then each entry is multiplied by 1 / D_ii.
// Each of the 32 sequential steps is then one FP64 FMA and a shuffle instead
// of a multiply, a shuffle and an FMA: an FP64 warp instruction occupies a
// GB300 sub-partition for 64 cycles however many lanes it uses, so the
// chain is bound by its FP64 instruction count.  The scaled entries carry
// one extra rounding each, a componentwise relative perturbation of u, so
// the substitution stays backward stable.
constexpr int kTsMaxN = 2048;
constexpr int kTsMaxBlocks = kTsMaxN / 32;
constexpr int kTsMaxOwn = 8;         // diagonal blocks per CTA: n <= 256 P

struct TsSmem {
  double v[2][kTsMaxN];              // solved entries of each solve, every block pushed to every CTA
  double dg[2][kTsMaxOwn][32 * 33];  // owned diagonal blocks, scaled by the pivots:
                                     //   dg[0][o][i*33 + l] = R[32b+i, 32b+l] / R[32b+i, 32b+i], i < l
                                     //   dg[1][o][l*33 + i] = R[32b+l, 32b+i] / R[32b+i, 32b+i], l < i
  double hs[2][kTsMaxOwn][32];       // half-1 sums handed to the half-0 warp
  uint64_t bar[2][kTsMaxBlocks];     // bar[s][k]: block k of solve s has landed
};

__device__ inline int ts_owned(const CL& cl, int nb) {
  return (nb - (int)cl.rank + (int)cl.ncta - 1) / (int)cl.ncta;
}

// Barriers for both solves and the owned diagonal blocks; call before the
// cluster barrier that precedes the first solve.
__device__ inline void ts_setup(const CL& cl, TsSmem& sm, const double* __restrict__ R, int64_t ldr,
                                const double* __restrict__ inv_diag, int n) {
  const int nb = (n + 31) / 32;
  if ((int)threadIdx.x < 2 * nb) {
    const int sidx = threadIdx.x / nb, k = threadIdx.x % nb;
    mbar_init(&sm.bar[sidx][k], 1);
    mbar_arrive_expect_tx(&sm.bar[sidx][k], 8u * (uint32_t)min(32, n - 32 * k));
  }
  const int mine = ts_owned(cl, nb);
  for (int idx = threadIdx.x; idx < mine * 1024; idx += blockDim.x) {
    const int o = idx >> 10, l = (idx >> 5) & 31, i = idx & 31;
    const int r0 = 32 * ((int)cl.rank + o * (int)cl.ncta);
    // R[r0+i, r0+l] (i < l) scaled by its row's pivot (forward) and by its column's (backward)
    const bool in = i < l && r0 + l < n;
    const double v = in ? __ldg(R + (size_t)(r0 + i) + (size_t)(r0 + l) * ldr) : 0.0;
    sm.dg[0][o][i * 33 + l] = in ? v * __ldg(inv_diag + r0 + i) : 0.0;
    sm.dg[1][o][i * 33 + l] = in ? v * __ldg(inv_diag + r0 + l) : 0.0;
  }
  fence_mbar_init();
}

// Wait until every block of both solves has landed in this CTA (no st.async
// may still be in flight towards it when it leaves).
__device__ inline void ts_drain(TsSmem& sm, int n, uint64_t deadline, int& timed_out) {
  const int nb = (n + 31) / 32;
  if ((int)threadIdx.x < 2 * nb)
    if (!mbar_wait_bounded(&sm.bar[threadIdx.x / nb][threadIdx.x % nb], 0, deadline)) timed_out = 1;
}

// For a kernel that solves more than once with buffer set sidx: wait until
// every block of the solve that used phase `par` has landed here, then arm
// the set's barriers for the next phase.  The caller then meets the other
// CTAs at a cluster barrier before the next solve with this set, so no CTA
// is still reading its entries when the next ones are pushed.  (A push for
// the next phase may reach a barrier before it is armed: the transaction
// count goes below zero and the phase cannot complete before the local
// arrival, so nothing is lost.)
__device__ inline void ts_finish(TsSmem& sm, int n, int sidx, uint32_t par, uint64_t deadline, int& timed_out) {
  const int nb = (n + 31) / 32;
  if ((int)threadIdx.x < nb) {
    const int k = threadIdx.x;
    if (!mbar_wait_bounded(&sm.bar[sidx][k], par, deadline)) timed_out = 1;
    mbar_arrive_expect_tx(&sm.bar[sidx][k], 8u * (uint32_t)min(32, n - 32 * k));
  }
}

// One substitution.  kBack = false: R^T y = rhs with M = R^T column-major
// (M[i + j*ldm] = R[j, i]); kBack = true: R x = rhs with M = R.  rhs[s] is
// read by the half-0 lane of slot s (row 32 b_s + lane); out[s] receives the
// solution there.  sidx selects the buffers (0 first solve, 1 second); par
// is the barrier phase of this use of the set (ts_finish).
template <int PP, bool kBack>
__device__ inline void ts_solve(const CL& cl, TsSmem& sm, int sidx, const double* __restrict__ M, int64_t ldm,
                                const double* __restrict__ inv_diag, int n, const double (&rhs)[PP],
                                double (&out)[PP], uint64_t deadline, int& timed_out, uint32_t par = 0) {
  const int nb = (n + 31) / 32, P = (int)cl.ncta;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, q = w >> 1, h = w & 1;
  const int mine = ts_owned(cl, nb);
  int bk[PP], row[PP];
  bool has[PP], rowok[PP];
  int klo = nb, khi = -1;
#pragma unroll
  for (int s = 0; s < PP; ++s) {
    const int o = q + 4 * s;
    has[s] = o < mine;
    bk[s] = has[s] ? (int)cl.rank + o * P : -1;
    row[s] = 32 * bk[s] + l;
    rowok[s] = has[s] && row[s] < n;
    out[s] = 0.0;
    if (has[s]) { klo = min(klo, bk[s]); khi = max(khi, bk[s]); }
  }
  if (khi < 0) return;                          // this pair owns no block
  // forward: blocks 0 .. khi; backward: nb-1 .. klo
  const int kfirst = kBack ? nb - 1 : 0, kend = kBack ? klo - 1 : khi + 1, step = kBack ? -1 : 1;
  double acc[PP], cur[PP][16], nxt[PP][16], inv[PP];
  auto needs = [&](int s, int k) { return has[s] && (kBack ? k > bk[s] : k < bk[s]); };
  auto load = [&](double (&dst)[PP][16], int k) {
#pragma unroll
    for (int s = 0; s < PP; ++s) {
      const bool nd = needs(s, k) && rowok[s];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 32 * k + 16 * h + j;
        dst[s][j] = (nd && c < n) ? __ldg(M + (size_t)row[s] + (size_t)c * ldm) : 0.0;
      }
    }
  };
#pragma unroll
  for (int s = 0; s < PP; ++s) {
    acc[s] = 0.0;
    inv[s] = (h == 0 && rowok[s]) ? __ldg(inv_diag + row[s]) : 0.0;
  }
  load(cur, kfirst);
  for (int k = kfirst; k != kend; k += step) {
    if (k + step != kend) load(nxt, k + step);
    bool any = false;
#pragma unroll
    for (int s = 0; s < PP; ++s) any = any || needs(s, k);
    if (any) {
      if (!mbar_wait_bounded(&sm.bar[sidx][k], par, deadline)) timed_out = 1;
      double vk[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 32 * k + 16 * h + j;
        vk[j] = c < n ? sm.v[sidx][c] : 0.0;
      }
#pragma unroll
      for (int s = 0; s < PP; ++s)
        if (needs(s, k)) {
          double p0 = 0.0, p1 = 0.0;
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            p0 += cur[s][j] * vk[j];
            p1 += cur[s][j + 1] * vk[j + 1];
          }
          acc[s] += p0 + p1;
        }
    }
#pragma unroll
    for (int s = 0; s < PP; ++s)
      if (has[s] && k == bk[s]) {
        const int o = q + 4 * s;
        if (h == 1) sm.hs[sidx][o][l] = acc[s];
        asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
        if (h == 0) {
          // lane l: row l of the unit-triangular block (column l of the scaled R)
          double rv[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) rv[i] = kBack ? sm.dg[1][o][l * 33 + i] : sm.dg[0][o][i * 33 + l];
          double wl = rowok[s] ? rhs[s] - (acc[s] + sm.hs[sidx][o][l]) : 0.0;
          if (!kBack) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const double wi = __shfl_sync(0xffffffffu, wl, i);
              if (l > i) wl = wl - rv[i] * wi;
            }
          } else {
#pragma unroll
            for (int i = 31; i >= 0; --i) {
              const double wi = __shfl_sync(0xffffffffu, wl, i);
              if (l < i) wl = wl - rv[i] * wi;
            }
          }
          const double yl = wl * inv[s];
          out[s] = yl;
          if (rowok[s]) {
            const uint32_t va = smem_u32(&sm.v[sidx][row[s]]), ba = smem_u32(&sm.bar[sidx][k]);
            for (int d = 0; d < P; ++d) {
              uint32_t ra, rb;
              asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(va), "r"(d));
              asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(ba), "r"(d));
              st_async_f64(ra, yl, rb);
            }
          }
        }
      }
    if (k + step != kend) {
#pragma unroll
      for (int s = 0; s < PP; ++s)
#pragma unroll
        for (int j = 0; j < 16; ++j) cur[s][j] = nxt[s][j];
    }
  }
}

// Pairs-per-slot needed for n on a cluster of P CTAs (0: too large).
__host__ __device__ inline int ts_slots(int n, int P) {
  const int nb = (n + 31) / 32, mine = (nb + P - 1) / P;
  return mine <= 4 ? 1 : mine <= 8 ? 2 : 0;
}

}  // namespace lsk
