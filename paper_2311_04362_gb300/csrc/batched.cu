// batched.cu -- many independent least-squares problems of different shapes
// solved together (Algorithm 2 with the Sec. 3.3 stopping rule per problem),
// one launch per phase for the whole batch.
//
//  * sketch: k_b_sparse_sign writes every column's zeta rows as global bucket
//    ids (problem offset + row); k_b_csr (one CTA per problem) counts, scans
//    and scatters the problem's entries with shared-memory atomics and sorts
//    every bucket (a warp-wide bitonic sort in shared memory; the CTA sorts
//    buckets above 1024 entries in global scratch), so the CSR is the unique
//    stable one; k_b_gather forms B_p with 32, 16, 8 or 4 lanes per bucket
//    (one column per lane, the narrowest width that holds n + 1 columns) with
//    the same left-to-right sums as the single-problem path, so every B_p is
//    bit-identical to ls_sketch of that problem.
//  * factor: one CTA per problem (k_b_householder: unblocked LAPACK-convention
//    Householder on B_p in L2), then k_prepare_R-like and post-factor work
//    per problem on 1-CTA clusters with the cluster_la.cuh routines.
//  * iterate: k_b_compact lists the active problems and the prefix of their
//    row tiles; k_b_pass, persistent (two CTAs per SM), walks those tiles with
//    a two-buffer cp.async.bulk pipeline (rows of A land in shared memory at
//    a stride = 2 mod 4 doubles, so column-wise reads are at most 2-way bank
//    conflicted).  Each tile is used twice: row dots A_j x by (row, column
//    chunk) threads -- no shuffle trees, the FP64 pipe does one FMA per
//    element -- then c += A^T r by (column, row group) threads.  One partial
//    (c, ||r||^2, ||r - r_prev||^2) per tile; k_b_step (one CTA per problem)
//    sums a problem's partials in tile order, applies the stopping rule and
//    does the two substitutions and the update.
#include <algorithm>

#include "cluster_la.cuh"

namespace lsk {



size_t bprob_bytes() { return sizeof(BProb); }
int64_t batch_boff(const BProb* P, int p) { return P[p].boff; }
int64_t batch_roff(const BProb* P, int p) { return P[p].roff; }

void batch_offsets(const BProb* P, int np, int64_t* moffs, int64_t* doffs, int64_t* toffs) {
  for (int p = 0; p < np; ++p) { moffs[p] = P[p].moff; doffs[p] = P[p].doff; toffs[p] = P[p].toff; }
}

__device__ inline int find_problem(const int64_t* offs, int np, int64_t g) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

enum { V_INVD = 0, V_XPREV, V_Y, V_D, V_WORK, V_V, V_W, V_XI, V_COUNT };
__device__ inline double* bvec(const BPools& pl, const BProb& pr, int k) {
  return pl.V + pr.voff + (int64_t)k * pr.n;
}
__device__ inline double* bR(const BPools& pl, const BProb& pr) { return pl.R + pr.roff; }
__device__ inline double* bRt(const BPools& pl, const BProb& pr) { return pl.R + pr.roff + pr.n * pr.n; }

// Completion record (server mode): the finished slot and its outcome.
__device__ inline void b_record_done(const BPools& pl, int p, const IterState& s) {
  if (!pl.done_count) return;
  const unsigned int pos = atomicAdd(pl.done_count, 1u);
  BDone r;
  r.slot = p; r.iters = s.iter; r.stop_reason = s.stop_reason; r.pad = 0;
  r.res_norm = s.rnorm; r.step_norm = s.dnorm; r.normest = s.normest; r.condest = s.condest;
  pl.done_rec[pos] = r;
}

// ---------------------------------------------------------------- sketch
__global__ void __launch_bounds__(256) k_b_sparse_sign(const BProb* __restrict__ P, const int64_t* __restrict__ moffs,
                                                       int np, int64_t mtotal, int zeta, int32_t* __restrict__ rows,
                                                       uint32_t* __restrict__ signs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= mtotal) return;
  const int p = find_problem(moffs, np, g);
  const int64_t j = g - P[p].moff;
  const int64_t d = P[p].d;
  WordStream s(P[p].seed, (uint64_t)j, 0u);
  const uint32_t mask = s.next();
  int32_t r[32];
  int cnt = 0;
  for (int64_t t = d - zeta; t < d; ++t) {
    const int32_t v = (int32_t)s.below((uint32_t)(t + 1));
    bool seen = false;
    for (int i = 0; i < cnt; ++i) seen |= (r[i] == v);
    r[cnt++] = seen ? (int32_t)t : v;
  }
  for (int i = 1; i < cnt; ++i) {
    const int32_t key = r[i];
    int k = i - 1;
    while (k >= 0 && r[k] > key) { r[k + 1] = r[k]; --k; }
    r[k + 1] = key;
  }
  int32_t* out = rows + g * zeta;
  for (int i = 0; i < cnt; ++i) out[i] = (int32_t)(P[p].doff + r[i]);
  signs[g] = mask;
}

// Largest bucket count handled by k_b_csr (shared-memory counters).
static constexpr int kCsrMaxD = 12288;
static constexpr int kCsrThreads = 512;
static constexpr int kCsrWarpKeys = 1024;   // per-warp sort scratch (keys)

// Warp-wide bitonic sort of s[0..P) ascending (P a power of two <= 1024).
__device__ inline void warp_bitonic(uint32_t* s, int P, int lane) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = s[i], b = s[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { s[i] = b; s[ixj] = a; }
        }
      }
      __syncwarp();
    }
  }
}

// One CTA per problem: CSR of the problem's part of S (row_ptr over its d
// buckets, entries (global column << 1 | negative) sorted within each bucket).
// The entries of problem p occupy [moff * zeta, (moff + m) * zeta).
__global__ void __launch_bounds__(kCsrThreads) k_b_csr(const BProb* __restrict__ P, int zeta,
                                                       const int32_t* __restrict__ rows,
                                                       const uint32_t* __restrict__ signs,
                                                       int64_t* __restrict__ row_ptr, uint32_t* __restrict__ ent,
                                                       uint32_t* __restrict__ scratch,
                                                       unsigned int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char csr_smem[];
  int* cnt = reinterpret_cast<int*>(csr_smem);                               // kCsrMaxD
  uint32_t* wscr = reinterpret_cast<uint32_t*>(cnt + kCsrMaxD);              // 16 x 1024
  __shared__ int wtot[32];
  __shared__ int s_big;
  const BProb pr = P[blockIdx.x];
  const int d = (int)pr.d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t e0 = pr.moff * zeta;                 // first entry of this problem
  const int64_t ne = pr.m * zeta;
  const int32_t* rw = rows + e0;
  for (int t = tid; t < d; t += kCsrThreads) cnt[t] = 0;
  if (tid == 0) s_big = 0;
  __syncthreads();
  for (int64_t e = tid; e < ne; e += kCsrThreads) atomicAdd(&cnt[rw[e] - (int)pr.doff], 1);
  __syncthreads();
  // exclusive scan of cnt[0..d) in chunks of the block
  int carry = 0;
  for (int base = 0; base < d; base += kCsrThreads) {
    const int t = base + tid;
    const int v = (t < d) ? cnt[t] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int w = (lane < kCsrThreads / 32) ? wtot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wtot[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (warp ? wtot[warp - 1] : 0) + incl - v;
    if (t < d) {
      cnt[t] = excl;
      row_ptr[pr.doff + t] = e0 + excl;
      if (v > kCsrWarpKeys) s_big = 1;
    }
    carry += wtot[kCsrThreads / 32 - 1];
    __syncthreads();
  }
  if (tid == 0) row_ptr[pr.doff + d] = e0 + ne;      // equals the next problem's first row_ptr
  // scatter (bucket order of equal keys is fixed by the sort below)
  for (int64_t e = tid; e < ne; e += kCsrThreads) {
    const int64_t j = e / zeta;
    const int k = (int)(e - j * zeta);
    const uint32_t neg = (signs[pr.moff + j] >> k) & 1u;
    const int pos = atomicAdd(&cnt[rw[e] - (int)pr.doff], 1);
    ent[e0 + pos] = ((uint32_t)(pr.moff + j) << 1) | neg;
  }
  __syncthreads();
  // cnt[t] is now the end of bucket t (= start of bucket t + 1)
  uint32_t* mys = wscr + warp * kCsrWarpKeys;
  for (int t = warp; t < d; t += kCsrThreads / 32) {
    const int b0 = t ? cnt[t - 1] : 0, sz = cnt[t] - b0;
    if (sz <= 1 || sz > kCsrWarpKeys) continue;
    int Pw = 1;
    while (Pw < sz) Pw <<= 1;
    for (int i = lane; i < Pw; i += 32) mys[i] = (i < sz) ? ent[e0 + b0 + i] : 0xFFFFFFFFu;
    __syncwarp();
    warp_bitonic(mys, Pw, lane);
    for (int i = lane; i < sz; i += 32) ent[e0 + b0 + i] = mys[i];
    __syncwarp();
  }
  if (!s_big) return;                                  // uniform
  if (!scratch) {
    if (tid == 0) atomicOr(status, LS_DEV_BADSIZE);
    return;
  }
  for (int t = 0; t < d; ++t) {                        // rare: buckets above 1024 entries
    const int b0 = t ? cnt[t - 1] : 0, sz = cnt[t] - b0;
    if (sz <= kCsrWarpKeys) continue;
    int Pb = 1;
    while (Pb < sz) Pb <<= 1;
    uint32_t* buf = scratch + 2 * (e0 + b0);
    for (int i = tid; i < Pb; i += kCsrThreads) buf[i] = (i < sz) ? ent[e0 + b0 + i] : 0xFFFFFFFFu;
    __syncthreads();
    bitonic(buf, Pb);
    for (int i = tid; i < sz; i += kCsrThreads) ent[e0 + b0 + i] = buf[i];
    __syncthreads();
  }
}

// B_p[t, c] = s * (left-to-right sum over the bucket of +-[A_p b_p][j, c]).
// A warp serves 32 / gw buckets of one problem, gw lanes each (one column per
// lane, column chunks of gw).  Warps are numbered per problem from woffs.
// F = double: the oracle's sums; F = float: the same order in FP32 (each
// A entry rounded to FP32, FP32 accumulation, the scale applied in FP64 and
// the product rounded once to FP32).
template <typename F>
__global__ void __launch_bounds__(256) k_b_gather(const BProb* __restrict__ P, const int64_t* __restrict__ woffs,
                                                  int np, int64_t nwarps, const int64_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ ent, double scale,
                                                  F* __restrict__ Bpool) {
  const int64_t wg = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (wg >= nwarps) return;
  const int p = find_problem(woffs, np, wg);
  const BProb pr = P[p];
  const int gw = pr.gw;
  const int64_t t = (wg - pr.toff) * (32 / gw) + lane / gw;   // bucket within the problem
  if (t >= pr.d) return;
  const int cl = lane % gw;
  const int64_t tg = pr.doff + t;
  const int64_t e0 = row_ptr[tg], e1 = row_ptr[tg + 1];
  F* B = Bpool + pr.boff;
  const uint32_t mo = (uint32_t)pr.moff;              // entries hold global column ids
  for (int64_t c = cl; c <= pr.n; c += gw) {
    const bool isb = (c == pr.n);
    const double* base = isb ? pr.b : (pr.A + c);
    const int64_t stride = isb ? 1 : pr.lda;
    F acc = F(0);
    int64_t e = e0;
    for (; e + 4 <= e1; e += 4) {
      const uint32_t n0 = __ldg(ent + e), n1 = __ldg(ent + e + 1), n2 = __ldg(ent + e + 2), n3 = __ldg(ent + e + 3);
      const F v0 = (F)__ldg(base + (int64_t)((n0 >> 1) - mo) * stride);
      const F v1 = (F)__ldg(base + (int64_t)((n1 >> 1) - mo) * stride);
      const F v2 = (F)__ldg(base + (int64_t)((n2 >> 1) - mo) * stride);
      const F v3 = (F)__ldg(base + (int64_t)((n3 >> 1) - mo) * stride);
      acc = acc + signed_by(v0, n0);
      acc = acc + signed_by(v1, n1);
      acc = acc + signed_by(v2, n2);
      acc = acc + signed_by(v3, n3);
    }
    for (; e < e1; ++e) {
      const uint32_t n0 = __ldg(ent + e);
      const F v0 = (F)__ldg(base + (int64_t)((n0 >> 1) - mo) * stride);
      acc = acc + signed_by(v0, n0);
    }
    B[t + c * pr.d] = (F)(scale * (double)acc);
  }
}

// ---------------------------------------------------------------- factor
// One CTA per problem, problems in order of decreasing work (d n^2), blocked
// Householder QR (LAPACK convention) of B_p = [S A_p, S b_p], d x (n + 1):
// panels of kHB columns are factored column by column; the panel's
// reflectors are then applied to the trailing columns at once in compact-WY
// form, C <- C - V T^T (V^T C), reading C twice per panel instead of twice
// per column.  The trailing update runs on (row group, column) threads that
// keep W = V^T C and Y = T^T W for their column in registers while V is
// staged in shared memory by row chunks.
static constexpr int kHB = 16;        // panel width
static constexpr int kHChunk = 64;    // rows of V per shared-memory chunk

template <typename F>
__global__ void __launch_bounds__(256, 3) k_b_householder(const BProb* __restrict__ P, const int* __restrict__ order,
                                                       F* __restrict__ Bpool,
                                                       unsigned int* __restrict__ pstatus) {
  __shared__ F Vs[kHChunk * kHB];
  __shared__ F Wp[256 * kHB];
  __shared__ F T[kHB * kHB];
  __shared__ F Gs[kHB * kHB];
  __shared__ F taus[kHB];
  __shared__ F tmp[kHB];
  __shared__ F s_par[3];
  __shared__ int s_bad;
  const int p = order[blockIdx.x];
  const BProb pr = P[p];
  const int64_t d = pr.d;
  const int n = (int)pr.n;
  F* B = Bpool + pr.boff;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k0 = 0; k0 < n; k0 += kHB) {
    const int w = min(kHB, n - k0);
    // ---- panel: columns k0 .. k0 + w - 1, unblocked
    for (int kk = 0; kk < w; ++kk) {
      const int k = k0 + kk;
      F* col = B + k + (int64_t)k * d;
      const int64_t len = d - k;
      F ss = F(0);
      for (int64_t i = 1 + tid; i < len; i += 256) ss += col[i] * col[i];
      ss = cta_sum(ss);
      if (tid == 0) {
        const F alpha = col[0];
        const F xnorm = sqrt(ss);
        F beta, tau, scal;
        if (xnorm == F(0)) { beta = alpha; tau = F(0); scal = F(1); }
        else {
          const F h = hypot(alpha, xnorm);
          beta = (alpha >= F(0)) ? -h : h;
          tau = (beta - alpha) / beta;
          scal = F(1) / (alpha - beta);
        }
        s_par[0] = beta; s_par[1] = tau; s_par[2] = scal;
        s_bad = (beta == F(0) || !isfinite(beta)) ? 1 : 0;
        taus[kk] = tau;
      }
      __syncthreads();
      if (s_bad) {
        if (tid == 0) pstatus[p] |= LS_DEV_RANK;
        return;
      }
      const F tau = s_par[1], scal = s_par[2];
      if (tau != F(0))
        for (int64_t i = 1 + tid; i < len; i += 256) col[i] *= scal;
      __syncthreads();
      if (tid == 0) col[0] = s_par[0];
      if (tau != F(0)) {
        for (int j = k + 1 + warp; j < k0 + w; j += 8) {
          F* cj = B + k + (int64_t)j * d;
          F acc = F(0);
          for (int64_t i = lane; i < len; i += 32) acc += ((i == 0) ? F(1) : col[i]) * cj[i];
          acc = warp_sum(acc);
          const F tw = tau * acc;
          for (int64_t i = lane; i < len; i += 32) cj[i] = cj[i] - tw * ((i == 0) ? F(1) : col[i]);
        }
      }
      __syncthreads();
    }
    const int j0 = k0 + w;                  // first trailing column
    const int ncols = n + 1 - j0;           // >= 1 (column n is S b)
    // ---- Gram G[a][b] = v_a^T v_b (a < b) of the panel's reflectors
    const int npairs = w * (w - 1) / 2;
    for (int pi = warp; pi < npairs; pi += 8) {
      int a = 0, rem = pi;
      while (rem >= w - 1 - a) { rem -= w - 1 - a; ++a; }
      const int b = a + 1 + rem;
      const F* va = B + (int64_t)(k0 + a) * d;
      const F* vb = B + (int64_t)(k0 + b) * d;
      F acc = F(0);
      for (int64_t i = k0 + b + lane; i < d; i += 32) acc += va[i] * ((i == k0 + b) ? F(1) : vb[i]);
      acc = warp_sum(acc);
      if (lane == 0) Gs[a * kHB + b] = acc;
    }
    if (tid < kHB * kHB) T[tid] = F(0);
    __syncthreads();
    // ---- T (upper): T[kk][kk] = tau_kk, T[0:kk, kk] = -tau_kk T[0:kk, 0:kk] G[0:kk, kk]
    for (int kk = 0; kk < w; ++kk) {
      if (tid < kk) {
        F t = F(0);
        for (int c = tid; c < kk; ++c) t += T[tid * kHB + c] * Gs[c * kHB + kk];
        tmp[tid] = -taus[kk] * t;
      }
      __syncthreads();
      if (tid < kk) T[tid * kHB + kk] = tmp[tid];
      if (tid == 0) T[kk * kHB + kk] = taus[kk];
      __syncthreads();
    }
    // ---- trailing update of columns j0 .. n, rows k0 .. d - 1
    for (int cb = 0; cb < ncols; cb += 256) {
      const int nc = min(256, ncols - cb);
      const int Gr = max(1, 256 / nc);
      const int g = tid / nc, jl = tid - g * nc;
      const bool active = g < Gr;
      F* cj = B + (int64_t)(j0 + cb + jl) * d;
      F acc[kHB];
#pragma unroll
      for (int q = 0; q < kHB; ++q) acc[q] = F(0);
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t r0 = k0; r0 < d; r0 += kHChunk) {
          const int h = (int)min((int64_t)kHChunk, d - r0);
          for (int e = tid; e < h * kHB; e += 256) {
            const int i = e / kHB, q = e - i * kHB;
            const int64_t R = r0 + i, dq = k0 + q;
            F v = F(0);
            if (q < w) v = (R < dq) ? F(0) : (R == dq ? F(1) : B[R + dq * d]);
            Vs[e] = v;
          }
          __syncthreads();
          if (active) {
            const int rpg = (h + Gr - 1) / Gr;
            const int i0 = g * rpg, i1 = min(h, i0 + rpg);
            if (pass == 0) {
              for (int i = i0; i < i1; ++i) {
                const F c = cj[r0 + i];
                const F* vr = Vs + i * kHB;
#pragma unroll
                for (int q = 0; q < kHB; ++q) acc[q] = fma(vr[q], c, acc[q]);
              }
            } else {
              for (int i = i0; i < i1; ++i) {
                F c = cj[r0 + i];
                const F* vr = Vs + i * kHB;
#pragma unroll
                for (int q = 0; q < kHB; ++q) c = fma(-vr[q], acc[q], c);
                cj[r0 + i] = c;
              }
            }
          }
          __syncthreads();
        }
        if (pass == 0) {
          // W of column jl = sum of the row groups' partials (group order);
          // then Y = T^T W, handed to every row group through Wp
          if (active)
#pragma unroll
            for (int q = 0; q < kHB; ++q) Wp[(g * nc + jl) * kHB + q] = acc[q];
          __syncthreads();
          if (active && g == 0) {
            F wv[kHB];
#pragma unroll
            for (int q = 0; q < kHB; ++q) {
              F t = F(0);
              for (int gg = 0; gg < Gr; ++gg) t += Wp[(gg * nc + jl) * kHB + q];
              wv[q] = t;
            }
#pragma unroll
            for (int q = 0; q < kHB; ++q) {
              F y = F(0);
#pragma unroll
              for (int a = 0; a <= q; ++a) y = fma(T[a * kHB + q], wv[a], y);
              acc[q] = y;
            }
          }
          __syncthreads();
          if (active && g == 0)
#pragma unroll
            for (int q = 0; q < kHB; ++q) Wp[jl * kHB + q] = acc[q];
          __syncthreads();
          if (active)
#pragma unroll
            for (int q = 0; q < kHB; ++q) acc[q] = Wp[jl * kHB + q];
          __syncthreads();
        }
      }
    }
  }
}

// One thread-block cluster per problem (large n): the same blocked
// compact-WY Householder QR as k_b_householder with the rows of B_p split
// into contiguous slices, one per CTA of the cluster.  Each reduction over
// rows (a column norm, the panel's dot products, the Gram matrix of the
// panel's reflectors, W = V^T C) is a per-CTA partial in shared memory,
// summed by every CTA over the cluster in CTA order through distributed
// shared memory after a cluster barrier; every CTA then takes the same
// reflector and T, and updates its own rows.  Two cluster barriers per
// column, two per panel.
static constexpr int kCQMaxN = 512;                    // widest problem (ncols <= kCQMaxN + 1)
static constexpr int kCQMinN = 256;                    // narrower problems factor on one CTA
static constexpr int kCQW = kHB * (kCQMaxN + 8);       // doubles of one W / Y table

__global__ void __launch_bounds__(256, 1) k_b_qr_cluster(const BProb* __restrict__ P, const int* __restrict__ list,
                                                         double* __restrict__ Bpool,
                                                         unsigned int* __restrict__ pstatus) {
  extern __shared__ __align__(16) double cq[];
  double* Wc = cq;                         // this CTA's partial W (column-major by 16), read by the cluster
  double* Ys = Wc + kCQW;                  // Y = T^T W for all trailing columns
  double* Gq = Ys + kCQW;                  // row-group partials (256 x 16)
  double* Vs = Gq + 256 * kHB;             // V chunk (kHChunk x 16)
  __shared__ double red_ss[2], red_alpha[2], red_dot[2][kHB], Gp[kHB * kHB];
  __shared__ double T[kHB * kHB], Gs[kHB * kHB], taus[kHB], tmp[kHB], s_par[3];
  __shared__ int s_bad;
  const uint32_t rank = cluster_rank(), C = cluster_nctas();
  const int p = list[blockIdx.x / C];
  const BProb pr = P[p];
  const int64_t d = pr.d;
  const int n = (int)pr.n;
  double* B = Bpool + pr.boff;
  const int64_t h = (d + C - 1) / C;
  const int64_t rlo = min(d, (int64_t)rank * h), rhi = min(d, rlo + h);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k0 = 0; k0 < n; k0 += kHB) {
    const int w = min(kHB, n - k0);
    for (int kk = 0; kk < w; ++kk) {
      const int k = k0 + kk, par = kk & 1;
      double* col = B + (int64_t)k * d;
      // ---- column norm below the diagonal, reflector (identical in every CTA)
      double ss = 0.0;
      for (int64_t i = max(rlo, (int64_t)k + 1) + tid; i < rhi; i += 256) ss += col[i] * col[i];
      ss = cta_sum(ss);
      const uint32_t owner = (uint32_t)(k / h);
      if (tid == 0) {
        red_ss[par] = ss;
        if (owner == rank) red_alpha[par] = col[k];
      }
      cluster_sync();
      if (tid == 0) {
        double t = 0.0;
        for (uint32_t c = 0; c < C; ++c) t += ld_cluster_f64(map_shared(&red_ss[par], c));
        const double alpha = ld_cluster_f64(map_shared(&red_alpha[par], owner));
        const double xnorm = sqrt(t);
        double beta, tau, scal;
        if (xnorm == 0.0) { beta = alpha; tau = 0.0; scal = 1.0; }
        else {
          const double hh = hypot(alpha, xnorm);
          beta = (alpha >= 0.0) ? -hh : hh;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        s_par[0] = beta; s_par[1] = tau; s_par[2] = scal;
        s_bad = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        taus[kk] = tau;
      }
      __syncthreads();
      if (s_bad) {                               // the same decision in every CTA
        if (rank == 0 && tid == 0) pstatus[p] |= LS_DEV_RANK;
        cluster_sync();                          // no CTA leaves while others read its shared memory
        return;
      }
      const double tau = s_par[1], scal = s_par[2];
      if (tau != 0.0)
        for (int64_t i = max(rlo, (int64_t)k + 1) + tid; i < rhi; i += 256) col[i] *= scal;
      __syncthreads();
      if (tid == 0 && owner == rank) col[k] = s_par[0];
      // ---- the reflector applied to the rest of the panel
      for (int j = k + 1 + warp; j < k0 + w; j += 8) {
        const double* cj = B + (int64_t)j * d;
        double acc = 0.0;
        if (tau != 0.0)
          for (int64_t i = max(rlo, (int64_t)k) + lane; i < rhi; i += 32) acc += ((i == k) ? 1.0 : col[i]) * cj[i];
        acc = warp_sum(acc);
        if (lane == 0) red_dot[par][j - k0] = acc;
      }
      cluster_sync();
      if (tau != 0.0) {
        for (int j = k + 1 + warp; j < k0 + w; j += 8) {
          double dot = 0.0;
          if (lane == 0)
            for (uint32_t c = 0; c < C; ++c) dot += ld_cluster_f64(map_shared(&red_dot[par][j - k0], c));
          dot = __shfl_sync(0xffffffffu, dot, 0);
          const double tw = tau * dot;
          double* cj = B + (int64_t)j * d;
          for (int64_t i = max(rlo, (int64_t)k) + lane; i < rhi; i += 32) cj[i] = cj[i] - tw * ((i == k) ? 1.0 : col[i]);
        }
      }
      __syncthreads();
    }
    const int j0 = k0 + w;
    const int ncols = n + 1 - j0;
    // ---- Gram of the panel's reflectors over this CTA's rows, summed over the cluster
    const int npairs = w * (w - 1) / 2;
    for (int pi = warp; pi < npairs; pi += 8) {
      int a = 0, rem = pi;
      while (rem >= w - 1 - a) { rem -= w - 1 - a; ++a; }
      const int b = a + 1 + rem;
      const double* va = B + (int64_t)(k0 + a) * d;
      const double* vb = B + (int64_t)(k0 + b) * d;
      double acc = 0.0;
      for (int64_t i = max(rlo, (int64_t)(k0 + b)) + lane; i < rhi; i += 32)
        acc += va[i] * ((i == k0 + b) ? 1.0 : vb[i]);
      acc = warp_sum(acc);
      if (lane == 0) Gp[a * kHB + b] = acc;
    }
    cluster_sync();
    for (int e = tid; e < kHB * kHB; e += 256) {
      const int a = e / kHB, b = e - a * kHB;
      double g = 0.0;
      if (a < b && b < w)
        for (uint32_t c = 0; c < C; ++c) g += ld_cluster_f64(map_shared(&Gp[e], c));
      Gs[e] = g;
      T[e] = 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < w; ++kk) {
      if (tid < kk) {
        double t = 0.0;
        for (int c = tid; c < kk; ++c) t += T[tid * kHB + c] * Gs[c * kHB + kk];
        tmp[tid] = -taus[kk] * t;
      }
      __syncthreads();
      if (tid < kk) T[tid * kHB + kk] = tmp[tid];
      if (tid == 0) T[kk * kHB + kk] = taus[kk];
      __syncthreads();
    }
    // ---- W = V^T C over this CTA's rows (row groups x columns), all column blocks
    const int64_t lo = max(rlo, (int64_t)k0);
    for (int cb = 0; cb < ncols; cb += 256) {
      const int nc = min(256, ncols - cb);
      const int Gr = max(1, 256 / nc);
      const int g = tid / nc, jl = tid - g * nc;
      const bool active = g < Gr;
      const double* cj = B + (int64_t)(j0 + cb + jl) * d;
      double acc[kHB];
#pragma unroll
      for (int q = 0; q < kHB; ++q) acc[q] = 0.0;
      for (int64_t r0 = lo; r0 < rhi; r0 += kHChunk) {
        const int hgt = (int)min((int64_t)kHChunk, rhi - r0);
        for (int e = tid; e < hgt * kHB; e += 256) {
          const int i = e / kHB, q = e - i * kHB;
          const int64_t R = r0 + i, dq = k0 + q;
          Vs[e] = (q < w) ? ((R < dq) ? 0.0 : (R == dq ? 1.0 : B[R + dq * d])) : 0.0;
        }
        __syncthreads();
        if (active) {
          const int rpg = (hgt + Gr - 1) / Gr;
          const int i0 = g * rpg, i1 = min(hgt, i0 + rpg);
          for (int i = i0; i < i1; ++i) {
            const double c = cj[r0 + i];
            const double* vr = Vs + i * kHB;
#pragma unroll
            for (int q = 0; q < kHB; ++q) acc[q] = fma(vr[q], c, acc[q]);
          }
        }
        __syncthreads();
      }
      if (active)
#pragma unroll
        for (int q = 0; q < kHB; ++q) Gq[(g * nc + jl) * kHB + q] = acc[q];
      __syncthreads();
      if (active && g == 0)
#pragma unroll
        for (int q = 0; q < kHB; ++q) {
          double t = 0.0;
          for (int gg = 0; gg < Gr; ++gg) t += Gq[(gg * nc + jl) * kHB + q];
          Wc[(cb + jl) * kHB + q] = t;
        }
      __syncthreads();
    }
    cluster_sync();
    // ---- Y = T^T (sum over the cluster of W), for every trailing column
    for (int j = tid; j < ncols; j += 256) {
      double wv[kHB];
#pragma unroll
      for (int q = 0; q < kHB; ++q) wv[q] = 0.0;
      for (uint32_t c = 0; c < C; ++c) {
        const uint32_t base = map_shared(Wc + j * kHB, c);
#pragma unroll
        for (int q = 0; q < kHB; ++q) wv[q] += ld_cluster_f64(base + 8u * q);
      }
#pragma unroll
      for (int q = 0; q < kHB; ++q) {
        double y = 0.0;
#pragma unroll
        for (int a = 0; a <= q; ++a) y = fma(T[a * kHB + q], wv[a], y);
        Ys[j * kHB + q] = y;
      }
    }
    __syncthreads();
    // ---- C <- C - V Y on this CTA's rows
    for (int cb = 0; cb < ncols; cb += 256) {
      const int nc = min(256, ncols - cb);
      const int Gr = max(1, 256 / nc);
      const int g = tid / nc, jl = tid - g * nc;
      const bool active = g < Gr;
      double* cj = B + (int64_t)(j0 + cb + jl) * d;
      double y[kHB];
#pragma unroll
      for (int q = 0; q < kHB; ++q) y[q] = active ? Ys[(cb + jl) * kHB + q] : 0.0;
      for (int64_t r0 = lo; r0 < rhi; r0 += kHChunk) {
        const int hgt = (int)min((int64_t)kHChunk, rhi - r0);
        for (int e = tid; e < hgt * kHB; e += 256) {
          const int i = e / kHB, q = e - i * kHB;
          const int64_t R = r0 + i, dq = k0 + q;
          Vs[e] = (q < w) ? ((R < dq) ? 0.0 : (R == dq ? 1.0 : B[R + dq * d])) : 0.0;
        }
        __syncthreads();
        if (active) {
          const int rpg = (hgt + Gr - 1) / Gr;
          const int i0 = g * rpg, i1 = min(hgt, i0 + rpg);
          for (int i = i0; i < i1; ++i) {
            double c = cj[r0 + i];
            const double* vr = Vs + i * kHB;
#pragma unroll
            for (int q = 0; q < kHB; ++q) c = fma(-vr[q], y[q], c);
            cj[r0 + i] = c;
          }
        }
        __syncthreads();
      }
    }
  }
  cluster_sync();                                  // no CTA leaves while others read its shared memory
}

// Mixed precision: the top n rows of each problem's FP32-factored sketch (R
// on and above the diagonal, (Q^T S b)[0:n] in column n), widened to FP64
// into a compact n x (n+1) block at P64[p].boff (leading dimension n).
__global__ void k_b_widen_top(const BProb* __restrict__ P, const BProb* __restrict__ P64, int np,
                              const float* __restrict__ B32, double* __restrict__ Bc) {
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const int64_t n = P[p].n, d = P[p].d;
    const float* src = B32 + P[p].boff;
    double* dst = Bc + P64[p].boff;
    for (int64_t e = threadIdx.x; e < n * (n + 1); e += blockDim.x) {
      const int64_t c = e / n, i = e - c * n;
      dst[i + c * n] = (double)src[i + c * d];
    }
  }
}

__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// R_p, R_p^T and 1/diag(R_p) of the listed problems (all when list is null).
__global__ void k_b_prepare_R(const BProb* __restrict__ P, const int* __restrict__ list, int count, BPools pl) {
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int p = list ? list[idx] : idx;
    const BProb pr = P[p];
    const int n = (int)pr.n;
    const double* B = pl.B + pr.boff;
    double* R = bR(pl, pr);
    double* Rt = bRt(pl, pr);
    double* invd = bvec(pl, pr, V_INVD);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int j = e / n, i = e - j * n;
      const double r = (i <= j) ? B[i + (int64_t)j * pr.d] : 0.0;
      R[i + (int64_t)j * n] = r;
      Rt[j + (int64_t)i * n] = r;
      if (i == j) {
        invd[i] = 1.0 / r;
        if (r == 0.0 || !isfinite(r)) atomicOr(&pl.pstatus[p], LS_DEV_RANK);
      }
    }
  }
}

// One 1-CTA cluster per problem: x0 = R^{-1} z, normest, condest (the same
// steps as the single-problem post-factor kernel).
__global__ void __launch_bounds__(256) k_b_post_factor(const BProb* __restrict__ P, const int* __restrict__ list,
                                                       BPools pl) {
  const int p = list ? list[blockIdx.x] : blockIdx.x;
  if (pl.pstatus[p] & LS_DEV_RANK) return;
  const BProb pr = P[p];
  const CL cl{0u, 1u};
  const int n = (int)pr.n;
  const double* B = pl.B + pr.boff;
  const double* R = bR(pl, pr);
  const double* Rt = bRt(pl, pr);
  const double* invd = bvec(pl, pr, V_INVD);
  double* work = bvec(pl, pr, V_WORK);
  double* v = bvec(pl, pr, V_V);
  double* w = bvec(pl, pr, V_W);
  double* xi = bvec(pl, pr, V_XI);
  double* slots = pl.slots + (size_t)p * 64;
  cl_load_owned(cl, n, B + (int64_t)n * pr.d, work);
  cl_solve_R(cl, R, n, n, invd, work, pr.x);
  // normest
  for_owned_rows(cl, n, [&](int i) { __stcg(v + i, power_start(pr.seed, 1u, i)); });
  cl_sync();
  double nv = cl_norm2(cl, n, v, slots);
  for_owned_rows(cl, n, [&](int i) { __stcg(v + i, __ldcg(v + i) / nv); });
  cl_sync();
  const int steps = power_steps(n);
  for (int st = 0; st < steps; ++st) {
    cl_matvec_R(cl, Rt, n, v, w);
    cl_sync();
    cl_matvec_RT(cl, R, n, n, w, v);
    cl_sync();
    nv = cl_norm2(cl, n, v, slots);
    for_owned_rows(cl, n, [&](int i) { __stcg(v + i, __ldcg(v + i) / nv); });
    cl_sync();
  }
  cl_matvec_R(cl, Rt, n, v, w);
  cl_sync();
  const double normest = cl_norm2(cl, n, w, slots);
  // condest = ||R||_1 * Hager estimate of ||R^{-1}||_1
  double colmax = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s += fabs(__ldg(R + i + (size_t)j * n));
    colmax = fmax(colmax, s);
  }
  const double norm1 = cl_max(cl, cta_max(colmax), slots);
  double* x = v;
  double* y = w;
  for_owned_rows(cl, n, [&](int i) { __stcg(work + i, 1.0 / (double)n); });
  __syncthreads();
  cl_solve_R(cl, R, n, n, invd, work, y);
  double est;
  if (n == 1) {
    est = fabs(__ldcg(y));
  } else {
    est = cl_norm1(cl, n, y, slots);
    for_owned_rows(cl, n, [&](int i) { __stcg(xi + i, sgn1(__ldcg(y + i))); });
    cl_sync();
    cl_load_owned(cl, n, xi, work);
    cl_solve_RT(cl, Rt, n, invd, work, x);
    int j = cl_argmax_abs(cl, n, x, slots);
    int iter = 2;
    for (;;) {
      for_owned_rows(cl, n, [&](int i) { __stcg(work + i, i == j ? 1.0 : 0.0); });
      __syncthreads();
      cl_solve_R(cl, R, n, n, invd, work, y);
      const double est_old = est;
      est = cl_norm1(cl, n, y, slots);
      double diff = 0.0;
      for_owned_rows(cl, n, [&](int i) { if (sgn1(__ldcg(y + i)) != __ldcg(xi + i)) diff = 1.0; });
      const double any_diff = cl_max(cl, cta_max(diff), slots);
      if (any_diff == 0.0 || est <= est_old) break;
      for_owned_rows(cl, n, [&](int i) { __stcg(xi + i, sgn1(__ldcg(y + i))); });
      cl_sync();
      cl_load_owned(cl, n, xi, work);
      cl_solve_RT(cl, Rt, n, invd, work, x);
      const int jlast = j;
      j = cl_argmax_abs(cl, n, x, slots);
      if (__ldcg(x + jlast) != fabs(__ldcg(x + j)) && iter < 5) { iter += 1; continue; }
      break;
    }
    for_owned_rows(cl, n, [&](int i) {
      const double vv = 1.0 + (double)i / (double)(n - 1);
      __stcg(work + i, (i % 2 == 0) ? vv : -vv);
    });
    __syncthreads();
    cl_solve_R(cl, R, n, n, invd, work, y);
    double alt = cl_norm1(cl, n, y, slots);
    alt = 2.0 * alt / (3.0 * (double)n);
    if (alt > est) est = alt;
  }
  if (threadIdx.x == 0) {
    pl.est[2 * p] = normest;
    pl.est[2 * p + 1] = norm1 * est;
  }
}

// ---------------------------------------------------------------- iterate
// Per-problem iteration state set-up: x_prev = x0, state from the estimates.
// r_prev is not read before it is written (the first pass has no previous
// residual), so it needs no clearing.
__global__ void k_b_iter_init(const BProb* __restrict__ P, const int* __restrict__ list, int count, BPools pl,
                              double gamma, double rho, double alpha, double beta) {
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int p = list ? list[idx] : idx;
    const BProb pr = P[p];
    const bool rank = (pl.pstatus[p] & LS_DEV_RANK) != 0;
    double* xp = bvec(pl, pr, V_XPREV);
    if (!rank)
      for (int i = threadIdx.x; i < pr.n; i += blockDim.x) xp[i] = pr.x[i];
    if (threadIdx.x == 0) {
      IterState s{};
      s.gamma = gamma; s.rho = rho; s.alpha = alpha; s.beta = beta;
      s.normest = rank ? 0.0 : pl.est[2 * p];
      s.condest = rank ? 0.0 : pl.est[2 * p + 1];
      // a rank-deficient problem is reported by the next k_b_step (so that
      // every completion is recorded by the kernel on the iteration stream)
      if (rank) s.pad = 1;
      s.done = 1;
      pl.st[p] = s;
      __threadfence();
      *reinterpret_cast<volatile int*>(&pl.st[p].done) = 0;   // published last
    }
  }
}

static constexpr int kBThreads = 256;
// The tile size and rows per item come from the PassTune table (defaults:
// 3840 doubles, i.e. 30 KB per buffer and 3 CTAs per SM; 128 rows per item).

// Active problems in index order (alist) and the exclusive prefix of their
// pass items (aoff); cnt[0] = active problems, cnt[1] = their items, cnt[2] =
// the pass's work counter (items handed out beyond the first gridDim.x).
__global__ void __launch_bounds__(1024) k_b_compact(const BProb* __restrict__ P, int np,
                                                    const IterState* __restrict__ st, int* __restrict__ alist,
                                                    int64_t* __restrict__ aoff, int64_t* __restrict__ cnt) {
  __shared__ int64_t wa[32], wt[32];
  __shared__ int64_t carry_a, carry_t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry_a = 0; carry_t = 0; }
  __syncthreads();
  for (int base = 0; base < np; base += blockDim.x) {
    const int p = base + threadIdx.x;
    const int64_t fa = (p < np && !st[p].done) ? 1 : 0;
    const int64_t ft = fa ? (int64_t)P[p].items : 0;
    int64_t ia = fa, it = ft;                         // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t ya = __shfl_up_sync(0xffffffffu, ia, o), yt = __shfl_up_sync(0xffffffffu, it, o);
      if (lane >= o) { ia += ya; it += yt; }
    }
    if (lane == 31) { wa[warp] = ia; wt[warp] = it; }
    __syncthreads();
    if (warp == 0) {
      int64_t xa = (lane < (int)(blockDim.x >> 5)) ? wa[lane] : 0, xt = (lane < (int)(blockDim.x >> 5)) ? wt[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t ya = __shfl_up_sync(0xffffffffu, xa, o), yt = __shfl_up_sync(0xffffffffu, xt, o);
        if (lane >= o) { xa += ya; xt += yt; }
      }
      wa[lane] = xa; wt[lane] = xt;                   // inclusive over warps
    }
    __syncthreads();
    const int64_t pa = carry_a + (warp ? wa[warp - 1] : 0) + ia - fa;   // exclusive
    const int64_t pt = carry_t + (warp ? wt[warp - 1] : 0) + it - ft;
    if (fa) { alist[pa] = p; aoff[pa] = pt; }
    __syncthreads();
    if (threadIdx.x == 0) { carry_a += wa[(blockDim.x >> 5) - 1]; carry_t += wt[(blockDim.x >> 5) - 1]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { cnt[0] = carry_a; cnt[1] = carry_t; cnt[2] = 0; }
}

__device__ inline void bulk_load(void* smem_dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(smem_dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

struct BItem {
  int64_t v;        // item index in the active list (-1: none)
  int p, item;
};

// Issue the copies of one tile of problem pr into buf (warp 0; lane 0 sets
// the expected bytes first).
__device__ inline void b_issue_tile(const BProb& pr, int tile, double* buf, uint64_t* bar, int lane) {
  const int64_t row0 = (int64_t)tile * pr.tr;
  const int rows = (int)min((int64_t)pr.tr, pr.m - row0);
  const uint32_t row_bytes = (uint32_t)(pr.lda * sizeof(double));
  if (lane == 0) mbar_arrive_expect_tx(bar, row_bytes * (uint32_t)rows);
  __syncwarp();
  const double* src = pr.A + row0 * pr.lda;
  if (pr.rowcopy) {
    for (int r = lane; r < rows; r += 32) bulk_load(buf + (size_t)r * pr.ss, src + (size_t)r * pr.lda, row_bytes, bar);
  } else if (lane == 0) {
    bulk_load(buf, src, row_bytes * (uint32_t)rows, bar);
  }
}

__device__ inline BItem b_locate(const int* __restrict__ alist, const int64_t* __restrict__ aoff, int na, int64_t v,
                                 int64_t items) {
  BItem it{-1, 0, 0};
  if (v >= items) return it;
  const int i = find_problem(aoff, na, v);
  it.v = v;
  it.p = alist[i];
  it.item = (int)(v - aoff[i]);
  return it;
}

// Persistent pass over the items (runs of tpi consecutive row tiles) of the
// active problems.  Column sums of A^T r and the two squared norms are kept
// in registers across the tiles of an item; one partial per item.
__global__ void __launch_bounds__(kBThreads, 3) k_b_pass(const BProb* __restrict__ P, const int* __restrict__ alist,
                                                         const int64_t* __restrict__ aoff,
                                                         int64_t* __restrict__ cnt, BPools pl, int max_n,
                                                         int cap, unsigned int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* buf0 = reinterpret_cast<double*>(smem_raw);
  double* xs = buf0 + 2 * (size_t)cap;               // max_n (even)
  double* part1 = xs + ((max_n + 1) & ~1);           // 256
  double* rt = part1 + kBThreads;                    // 256
  double* q1 = rt + kBThreads;                       // 256: r_j
  double* q2 = q1 + kBThreads;                       // 256: r_j - r_prev_j
  double* gs = q2 + kBThreads;                       // 256: phase-2 group sums
  uint64_t* bar = reinterpret_cast<uint64_t*>(gs + kBThreads);
  __shared__ int64_t s_next;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int na = (int)cnt[0];
  const int64_t items = cnt[1];
  if ((int64_t)blockIdx.x >= items) return;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // items are handed out dynamically (CTAs that start late, e.g. behind other
  // kernels' CTAs, take fewer); which CTA computes an item does not change it
  BItem cur = b_locate(alist, aoff, na, blockIdx.x, items);
  int k = 0;                                          // tiles consumed by this CTA
  if (warp == 0) {
    const BProb& pr0 = P[cur.p];
    b_issue_tile(pr0, cur.item * pr0.tpi, buf0, &bar[0], lane);
  }
  while (cur.v >= 0) {
    if (tid == 0)
      s_next = (int64_t)gridDim.x + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cnt + 2), 1ull);
    __syncthreads();
    const BItem nxt = b_locate(alist, aoff, na, s_next, items);
    const BProb pr = P[cur.p];
    const int n = (int)pr.n, TR = pr.tr, ss = pr.ss, S = pr.S;
    const int t0 = cur.item * pr.tpi, t1 = min(pr.tiles, t0 + pr.tpi);
    for (int i = tid; i < n; i += kBThreads) xs[i] = pr.x[i];
    const int clen = (n + S - 1) / S;
    const int G = (n < kBThreads) ? kBThreads / n : 1;
    const int g = (n < kBThreads) ? tid / n : 0, cg = (n < kBThreads) ? tid - g * n : tid;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};            // column sums (n >= 256: columns tid + 256 u)
    double nv = 0.0;                                  // warps 0 / 1: squared norms
    for (int t = t0; t < t1; ++t, ++k) {
      // prefetch the next tile of this item, else the first tile of the next item
      if (warp == 0) {
        double* nb = buf0 + (size_t)((k + 1) & 1) * cap;
        if (t + 1 < t1) b_issue_tile(pr, t + 1, nb, &bar[(k + 1) & 1], lane);
        else if (nxt.v >= 0) {
          const BProb& pn = P[nxt.p];
          b_issue_tile(pn, nxt.item * pn.tpi, nb, &bar[(k + 1) & 1], lane);
        }
      }
      const bool more = (t + 1 < t1) || (nxt.v >= 0);
      const double* tl = buf0 + (size_t)(k & 1) * cap;
      const int64_t row0 = (int64_t)t * TR;
      const int rows = (int)min((int64_t)TR, pr.m - row0);
      const bool ok = mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1, gtimer() + LS_WAIT_NS);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(status, LS_DEV_TIMEOUT);
        if (tid == 0 && more) mbar_wait_bounded(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1, gtimer() + LS_WAIT_NS);
        return;
      }
      // phase 1: partial row dots, thread = (row r, column chunk s)
      if (tid < S * TR) {
        const int r = tid % TR, sidx = tid / TR;
        if (r < rows) {
          const int c0 = sidx * clen, c1 = min(n, c0 + clen);
          const double* a = tl + (size_t)r * ss;
          // four interleaved accumulators: a dot of rounding error ~ (len/4 + 2) u
          // instead of len u (the stopping rule compares r_i - r_{i-1} with u)
          double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
          int c = c0;
          for (; c + 3 < c1; c += 4) {
            d0 = fma(a[c], xs[c], d0);
            d1 = fma(a[c + 1], xs[c + 1], d1);
            d2 = fma(a[c + 2], xs[c + 2], d2);
            d3 = fma(a[c + 3], xs[c + 3], d3);
          }
          if (c < c1) d0 = fma(a[c], xs[c], d0);
          if (c + 1 < c1) d1 = fma(a[c + 1], xs[c + 1], d1);
          if (c + 2 < c1) d2 = fma(a[c + 2], xs[c + 2], d2);
          part1[tid] = (d0 + d1) + (d2 + d3);
        }
      }
      __syncthreads();
      double* rp = pl.r_prev + pr.rpoff + row0;
      if (tid < TR) {
        double v1 = 0.0, v2 = 0.0;
        if (tid < rows) {
          double dot = part1[tid];
          for (int sidx = 1; sidx < S; ++sidx) dot += part1[sidx * TR + tid];
          const double rj = __ldg(pr.b + row0 + tid) - dot;
          const double dl = rj - rp[tid];
          rp[tid] = rj;
          rt[tid] = rj;
          v1 = rj;
          v2 = dl;
        }
        q1[tid] = v1;
        q2[tid] = v2;
      }
      __syncthreads();
      // phase 2: c_k += sum_r A_rk r_r over the tile
      if (n >= kBThreads) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = tid + u * kBThreads;
          if (c < n)
            for (int r = 0; r < rows; ++r) acc[u] = fma(tl[(size_t)r * ss + c], rt[r], acc[u]);
        }
      } else if (g < G) {
        for (int r = g; r < rows; r += G) acc[0] = fma(tl[(size_t)r * ss + cg], rt[r], acc[0]);
      }
      if (warp < 2) {
        const double* q = warp ? q2 : q1;
        for (int r = lane; r < TR; r += 32) nv = fma(q[r], q[r], nv);
      }
      __syncthreads();                                // the buffer and rt are reused next
    }
    // the item's partial (c, ||r||^2, ||r - r_prev||^2)
    double* out = pl.part + pr.poff + (int64_t)cur.item * (n + 2);
    if (n >= kBThreads) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = tid + u * kBThreads;
        if (c < n) out[c] = acc[u];
      }
    } else {
      if (g < G) gs[g * n + cg] = acc[0];
      __syncthreads();
      for (int c = tid; c < n; c += kBThreads) {
        double t = 0.0;
        for (int gg = 0; gg < G; ++gg) t += gs[gg * n + c];
        out[c] = t;
      }
    }
    if (warp < 2) {
      nv = warp_sum(nv);
      if (lane == 0) out[n + warp] = nv;
    }
    __syncthreads();                                  // gs and xs are reused by the next item
    cur = nxt;
  }
}

// One 1-CTA cluster per problem: sum partials (item order), stopping rule,
// two substitutions, update.
__global__ void __launch_bounds__(256) k_b_step(const BProb* __restrict__ P, const int* __restrict__ alist,
                                                const int64_t* __restrict__ cnt, BPools pl, int use_stop, int extra,
                                                int q) {
  // only the problems the pass just served (the list k_b_compact made)
  if ((int64_t)blockIdx.x >= cnt[0]) return;
  const int p = alist[blockIdx.x];
  IterState S = pl.st[p];
  if (S.done) return;
  if (S.pad) {                      // rank deficient at factorization: report it now
    if (threadIdx.x == 0) {
      IterState& st = pl.st[p];
      st.done = 1;
      st.stop_reason = 4;
      b_record_done(pl, p, st);
    }
    return;
  }
  const BProb pr = P[p];
  const CL cl{0u, 1u};
  const int n = (int)pr.n;
  const double* part = pl.part + pr.poff;
  __shared__ double s_norm[2];
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int t = 0; t < pr.items; ++t) s += part[(int64_t)t * (n + 2) + n + threadIdx.x];
    s_norm[threadIdx.x] = s;
  }
  __syncthreads();
  const double rnorm = sqrt(s_norm[0]);
  const double dnorm = S.have_prev ? sqrt(s_norm[1]) : 0.0;
  const double u = 0x1.0p-53;
  int fired = S.fired, extra_left = S.extra_left, done = 0;
  if (use_stop && S.have_prev && !fired) {
    if (dnorm <= u * (S.gamma * S.normest * S.xnorm + S.rho * S.condest * rnorm)) {
      fired = 1;
      extra_left = extra;
    }
  }
  if (fired) {
    if (extra_left == 0) done = 1;
    else extra_left -= 1;
  }
  if (done) {
    if (threadIdx.x == 0) {
      IterState& st = pl.st[p];
      st.done = 1; st.fired = 1; st.stop_reason = 0;
      st.rnorm = rnorm; st.dnorm = dnorm;
      b_record_done(pl, p, st);
    }
    return;
  }
  double* work = bvec(pl, pr, V_WORK);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < pr.items; ++t) s += part[(int64_t)t * (n + 2) + i];
    __stcg(work + i, s);
  }
  __syncthreads();
  const double* invd = bvec(pl, pr, V_INVD);
  double* y = bvec(pl, pr, V_Y);
  double* dv = bvec(pl, pr, V_D);
  cl_solve_RT(cl, bRt(pl, pr), n, invd, work, y);
  cl_load_owned(cl, n, y, work);
  cl_solve_R(cl, bR(pl, pr), n, n, invd, work, dv);
  double xs = 0.0, bad = 0.0;
  double* xp = bvec(pl, pr, V_XPREV);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double xi = pr.x[i], xpi = xp[i], di = __ldcg(dv + i);
    const double xn = xi + S.alpha * di + S.beta * (xi - xpi);
    xp[i] = xi;
    pr.x[i] = xn;
    xs += xn * xn;
    if (!isfinite(xn)) bad = 1.0;
  }
  xs = cta_sum(xs);
  bad = cta_max(bad);
  if (threadIdx.x == 0) {
    IterState& st = pl.st[p];
    st.iter = S.iter + 1;
    st.fired = fired;
    st.extra_left = extra_left;
    st.have_prev = 1;
    st.xnorm = sqrt(xs);
    st.rnorm = rnorm;
    st.dnorm = dnorm;
    if (bad != 0.0) {
      st.nonfinite = 1; st.done = 1; st.stop_reason = 3;
    } else if (st.iter >= q) {
      st.done = 1; st.stop_reason = use_stop ? 1 : 2;
    }
    if (st.done) b_record_done(pl, p, st);
  }
}

// ---------------------------------------------------------------- host side

// Pass tile of a problem: shared-memory row stride ss = 2 mod 4 doubles (at
// most 2-way bank conflicts when threads read down a column), rows per tile
// tr = min(256, cap / ss), and S = 256 / tr column chunks per row dot.
static void pass_tile(int64_t n, int64_t lda, int tile, BProb& b) {
  const int ss = (int)((lda % 4 == 2) ? lda : lda + 2);
  b.ss = ss;
  b.rowcopy = (ss != lda) ? 1 : 0;
  b.tr = std::max(1, std::min(256, tile / ss));
  b.S = std::max(1, 256 / b.tr);
  (void)n;
}

int tune_cap(const PassTune& t) {
  int c = 0;
  for (int b = 0; b < kTuneBuckets; ++b) c = std::max(c, t.tile[b]);
  return c;
}

void batch_plan(const ls_problem* probs, int np, BProb* out, BatchPlan& pl, const PassTune& tune) {
  pl.np = np;
  pl.mtotal = pl.dtotal = pl.btotal = pl.rtotal = pl.vtotal = pl.ttotal = pl.ptotal = pl.wtotal = 0;
  pl.max_d = 0;
  pl.max_m = 0;
  pl.cap = 0;
  pl.max_fill = 0.0;
  pl.max_n = 0;
  pl.max_tile_doubles = 0;
  for (int p = 0; p < np; ++p) {
    const ls_problem& q = probs[p];
    BProb b{};
    b.A = q.A; b.b = q.b; b.x = q.x; b.m = q.m; b.n = q.n; b.lda = q.lda; b.d = q.d; b.seed = q.seed;
    b.moff = pl.mtotal; b.doff = pl.dtotal; b.boff = pl.btotal; b.roff = pl.rtotal; b.voff = pl.vtotal;
    b.rpoff = pl.mtotal;
    b.toff = pl.wtotal; b.poff = pl.ptotal;
    const int tb = tune_bucket(q.n);
    pass_tile(q.n, q.lda, tune.tile[tb], b);
    b.gw = (q.n + 1 > 16) ? 32 : (q.n + 1 > 8) ? 16 : (q.n + 1 > 4) ? 8 : 4;
    b.tiles = (int)((q.m + b.tr - 1) / b.tr);
    b.tpi = std::max(1, (tune.item_rows[tb] + b.tr - 1) / b.tr);
    pl.cap = std::max(pl.cap, b.tr * b.ss);
    b.items = (b.tiles + b.tpi - 1) / b.tpi;
    pl.mtotal += q.m; pl.dtotal += q.d; pl.btotal += q.d * (q.n + 1); pl.rtotal += 2 * q.n * q.n;
    pl.vtotal += V_COUNT * q.n; pl.ttotal += b.items; pl.ptotal += (int64_t)b.items * (q.n + 2);
    pl.wtotal += (q.d + (32 / b.gw) - 1) / (32 / b.gw);
    pl.max_d = std::max<int64_t>(pl.max_d, q.d);
    pl.max_m = std::max<int64_t>(pl.max_m, q.m);
    pl.max_fill = std::max<double>(pl.max_fill, (double)q.m / (double)q.d);
    pl.max_n = std::max<int>(pl.max_n, (int)q.n);

    out[p] = b;
  }
}

cudaError_t launch_cluster_grid(ls_ctx* ctx, const void* fn, void** args, int grid) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++ctx->launches;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_b_sketch_indices(ls_ctx* ctx, const BProb* dP, const int64_t* dmoffs, const BatchPlan& pl, int zeta,
                                    int32_t* rows, uint32_t* signs) {
  k_b_sparse_sign<<<(unsigned)((pl.mtotal + 255) / 256), 256, 0, ctx->stream>>>(dP, dmoffs, pl.np, pl.mtotal, zeta,
                                                                                 rows, signs);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_gather(ls_ctx* ctx, const BProb* dP, const int64_t* dwoffs, const BatchPlan& pl,
                            const int64_t* row_ptr, const uint32_t* ent, double scale, double* Bpool) {
  k_b_gather<double><<<(unsigned)((pl.wtotal + 7) / 8), 256, 0, ctx->stream>>>(dP, dwoffs, pl.np, pl.wtotal, row_ptr, ent,
                                                                       scale, Bpool);
  ++ctx->launches;
  return cudaGetLastError();
}

bool b_csr_fits(const BatchPlan& pl) { return pl.max_d <= kCsrMaxD; }
int64_t b_csr_max_d() { return kCsrMaxD; }
int64_t b_csr_global_entries() { return (int64_t)1 << 18; }

cudaError_t launch_b_csr(ls_ctx* ctx, const BProb* dP, const BatchPlan& pl, int zeta, const int32_t* rows,
                         const uint32_t* signs, int64_t* row_ptr, uint32_t* ent, uint32_t* scratch) {
  const size_t smem = sizeof(int) * kCsrMaxD + sizeof(uint32_t) * (kCsrThreads / 32) * kCsrWarpKeys;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_b_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  k_b_csr<<<pl.np, kCsrThreads, smem, ctx->stream>>>(dP, zeta, rows, signs, row_ptr, ent, scratch, ctx->d_status);
  ++ctx->launches;
  return cudaGetLastError();
}

// Factorization plan: problems with n >= kCQMinN (and n <= kCQMaxN) get a
// thread-block cluster each, the rest one CTA each in order of decreasing
// work (d n^2).  order[0 .. nsmall) = the one-CTA problems, order[nsmall ..
// np) = the cluster problems.  Returns nsmall.
int batch_order(const BProb* P, int np, int* order, bool clusters) {
  int ns = 0;
  for (int p = 0; p < np; ++p)
    if (!(clusters && P[p].n >= kCQMinN && P[p].n <= kCQMaxN)) order[ns++] = p;
  int nb = ns;
  for (int p = 0; p < np; ++p)
    if (clusters && P[p].n >= kCQMinN && P[p].n <= kCQMaxN) order[nb++] = p;
  std::stable_sort(order, order + ns, [&](int a, int b) {
    return (double)P[a].d * P[a].n * P[a].n > (double)P[b].d * P[b].n * P[b].n;
  });
  return ns;
}

size_t b_qr_cluster_smem() { return sizeof(double) * (2 * (size_t)kCQW + 256 * kHB + kHChunk * kHB); }
int b_qr_cluster_max_n() { return kCQMaxN; }

// CTAs per cluster for k_b_qr_cluster on this device: 16 where a 16-CTA
// cluster of this kernel fits, else 8, else 0 (not usable).
int b_qr_cluster_size(ls_ctx* ctx) {
  const size_t smem = b_qr_cluster_smem();
  if (cudaFuncSetAttribute(k_b_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  cudaFuncSetAttribute(k_b_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_b_qr_cluster, &cfg) == cudaSuccess && nclusters > 0) return c;
    cudaGetLastError();
  }
  return 0;
}

// Cluster QR of the `count` problems listed in dlist (device), csize CTAs each.
cudaError_t launch_b_qr_cluster(ls_ctx* ctx, const BProb* dP, const int* dlist, int count, int csize,
                                const BPools& pools) {
  if (count == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * csize));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = b_qr_cluster_smem();
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BProb* a0 = dP;
  const int* a1 = dlist;
  double* a2 = pools.B;
  unsigned int* a3 = pools.pstatus;
  void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3};
  ++ctx->launches;
  return cudaLaunchKernelExC(&cfg, (const void*)k_b_qr_cluster, args);
}

// Householder QR of `count` problems: the first `nsmall` entries of dorder
// one CTA each; `nbig` problems listed in dbig (may be null) one cluster
// each.  Then R, R^T, 1/diag(R), x0 and the estimates of all `count` listed
// problems (list; null = 0 .. count-1).
cudaError_t launch_b_factor2(ls_ctx* ctx, const BProb* dP, const int* dorder, int nsmall, const int* dbig, int nbig,
                             int csize, int count, const int* list, const BPools& pools) {
  cudaError_t e;
  if (nbig > 0 && (e = launch_b_qr_cluster(ctx, dP, dbig, nbig, csize, pools)) != cudaSuccess) return e;
  if (nsmall > 0) {
    k_b_householder<double><<<nsmall, 256, 0, ctx->stream>>>(dP, dorder, pools.B, pools.pstatus);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_b_prepare_R<<<std::min(count, ctx->num_sms * 8), 256, 0, ctx->stream>>>(dP, list, count, pools);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BPools pp = pools;
  const BProb* dPP = dP;
  const int* lp = list;
  void* args[] = {(void*)&dPP, (void*)&lp, &pp};
  return launch_cluster_grid(ctx, (const void*)k_b_post_factor, args, count);
}

cudaError_t launch_b_gather32(ls_ctx* ctx, const BProb* dP, const int64_t* dwoffs, const BatchPlan& pl,
                              const int64_t* row_ptr, const uint32_t* ent, double scale, float* B32) {
  k_b_gather<float><<<(unsigned)((pl.wtotal + 7) / 8), 256, 0, ctx->stream>>>(dP, dwoffs, pl.np, pl.wtotal, row_ptr,
                                                                              ent, scale, B32);
  ++ctx->launches;
  return cudaGetLastError();
}

// FP32 factorization of every problem (one CTA each, in dorder), then the
// FP64 R, R^T, x0 and estimates from the widened top rows (dP64: d = n,
// boff into Bc).
cudaError_t launch_b_factor_mixed(ls_ctx* ctx, const BProb* dP, const BProb* dP64, const int* dorder, int np,
                                  float* B32, double* Bc, const BPools& pools) {
  k_b_householder<float><<<np, 256, 0, ctx->stream>>>(dP, dorder, B32, pools.pstatus);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_b_widen_top<<<std::min(np, ctx->num_sms * 8), 256, 0, ctx->stream>>>(dP, dP64, np, B32, Bc);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BPools p64 = pools;
  p64.B = Bc;
  k_b_prepare_R<<<std::min(np, ctx->num_sms * 8), 256, 0, ctx->stream>>>(dP64, nullptr, np, p64);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const BProb* dPP = dP64;
  const int* lp = nullptr;
  void* args[] = {(void*)&dPP, (void*)&lp, &p64};
  return launch_cluster_grid(ctx, (const void*)k_b_post_factor, args, np);
}

cudaError_t launch_widen(ls_ctx* ctx, const float* src, double* dst, int64_t count) {
  k_widen<<<(unsigned)std::min<int64_t>((count + 255) / 256, (int64_t)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
      src, dst, count);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_factor(ls_ctx* ctx, const BProb* dP, const int* dorder, int count, const int* list,
                            const BPools& pools) {
  k_b_householder<double><<<count, 256, 0, ctx->stream>>>(dP, dorder, pools.B, pools.pstatus);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_b_prepare_R<<<std::min(count, ctx->num_sms * 8), 256, 0, ctx->stream>>>(dP, list, count, pools);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BPools pp = pools;
  const BProb* dPP = dP;
  const int* lp = list;
  void* args[] = {(void*)&dPP, (void*)&lp, &pp};
  return launch_cluster_grid(ctx, (const void*)k_b_post_factor, args, count);
}

cudaError_t launch_b_iter_init(ls_ctx* ctx, const BProb* dP, int count, const int* list, const BPools& pools,
                               double gamma, double rho, double alpha, double beta) {
  k_b_iter_init<<<std::min(count, ctx->num_sms * 8), 128, 0, ctx->stream>>>(dP, list, count, pools, gamma, rho,
                                                                           alpha, beta);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_compact(ls_ctx* ctx, const BProb* dP, int np, const BPools& pools, int* alist, int64_t* aoff,
                             int64_t* cnt) {
  k_b_compact<<<1, 1024, 0, ctx->stream>>>(dP, np, pools.st, alist, aoff, cnt);
  ++ctx->launches;
  return cudaGetLastError();
}

size_t b_pass_smem(int max_n, int cap) {
  return sizeof(double) * (2 * (size_t)cap + (size_t)((max_n + 1) & ~1) + 5 * kBThreads) + 2 * sizeof(uint64_t);
}

// Grid of the persistent pass for problems of up to max_n columns (also
// sets the kernel's shared-memory limit; call before capturing a launch).
int b_pass_grid(ls_ctx* ctx, int max_n, int cap) {
  const size_t smem = b_pass_smem(max_n, cap);
  if (cudaFuncSetAttribute(k_b_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pass, kBThreads, smem);
  return ctx->num_sms * std::max(1, per_sm);
}

cudaError_t launch_b_pass(ls_ctx* ctx, const BProb* dP, const int* alist, const int64_t* aoff, int64_t* cnt,
                          int max_n, int cap, int64_t max_items, const BPools& pools) {
  const size_t smem = b_pass_smem(max_n, cap);
  const int g = b_pass_grid(ctx, max_n, cap);
  if (g == 0) return cudaErrorInvalidValue;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(max_items, (int64_t)g));
  k_b_pass<<<(unsigned)grid, kBThreads, smem, ctx->stream>>>(dP, alist, aoff, cnt, pools, max_n, cap, ctx->d_status);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_step(ls_ctx* ctx, const BProb* dP, const int* alist, const int64_t* cnt, int np,
                          const BPools& pools, int use_stop, int extra, int q) {
  BPools pp = pools;
  const BProb* dPP = dP;
  const int* al = alist;
  const int64_t* cn = cnt;
  int us = use_stop, ex = extra, qq = q;
  void* args[] = {(void*)&dPP, (void*)&al, (void*)&cn, &pp, &us, &ex, &qq};
  return launch_cluster_grid(ctx, (const void*)k_b_step, args, np);
}

}  // namespace lsk
