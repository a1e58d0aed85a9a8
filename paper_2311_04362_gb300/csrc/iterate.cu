// iterate.cu -- the refinement loop of Algorithm 2:
//     r = b - A x,  c = A^T r,  d = R^{-1} (R^{-T} c),  x <- x + d
// with the Sec. 3.3 stopping rule and the App. B (Eq. (B.1)) damping /
// momentum update.
//
// k_fused_pass (a6): persistent, one CTA per SM.  A is streamed in row tiles
// (tr rows x all columns) by TMA (cp.async.bulk.tensor.2d) into a ring of
// shared-memory stages fed by one producer warp; eight consumer warps use each
// tile twice -- first the row dots A_j x (for n >= 32 every warp takes a
// rotated slice of every row's columns, a few lanes per row combined by two
// shuffles and the eight warps summed in warp order; for n < 32 a warp per
// row) and r_j = b_j - A_j x, then every thread adds r_j A_jk to its own
// columns of c -- so A is read from HBM exactly once per pass.  Each
// CTA writes one partial (c, ||r||^2, ||r - r_prev||^2); partials are summed
// over CTAs in index order by the next kernel, so results are bit-identical
// run to run.  Every wait is bounded by %globaltimer.
//
// k_fused_pass_ws: the warp-specialized form for n > 256 (below).
//
// k_iter_step / k_correct (a7): one thread-block cluster (16 CTAs where they
// fit) sums the partials, applies the stopping rule and performs the two
// triangular solves (the broadcast substitutions of cluster_la.cuh) and the
// update.
#include "cluster_la.cuh"

namespace lsk {

static constexpr int kConsumerWarps = 8;
static constexpr int kThreads = (kConsumerWarps + 1) * 32;

struct PassArgs {
  int64_t m;
  int n, boxw, nbox, tr, stages, ntiles;
  const double* b;
  const double* x;
  const double* r_prev;    // may be null
  double* r_out;           // may be null (may equal r_prev)
  double* part;            // gridDim.x * (n + 2)
  const IterState* st;     // null: always run
  unsigned int* status;
};

// OR of v over the `nthreads` threads (a multiple of 32) that meet at named
// barrier `id`: a group-uniform decision (e.g. to leave a loop after a
// bounded wait gave up) so that no warp is left at a later named barrier.
__device__ inline bool bar_any(bool v, int id, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Shared-memory offset (in doubles) of element (row r, column c) of a tile.
__device__ inline int tile_off(int r, int c, int boxw, int nbox, int tr) {
  return (nbox == 1) ? (r * boxw + c) : ((c >> 8) * (tr * 256) + r * 256 + (c & 255));
}

template <int NPT>
__global__ void __launch_bounds__(kThreads, 1) k_fused_pass(const __grid_constant__ CUtensorMap map, PassArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  const int n = a.n, tr = a.tr, boxw = a.boxw, nbox = a.nbox, S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t stage_doubles = (size_t)tr * nbox * boxw;
  // layout: [stages][stage_doubles] tiles | x[n] | rtile[2][tr] | red[...] | bars
  double* tiles = reinterpret_cast<double*>(smem_raw);
  double* xs = tiles + S * stage_doubles;
  double* rtile = xs + ((n + 1) & ~1);
  double* red = rtile + 2 * tr;                     // 2 * kConsumerWarps + 8
  double* p1 = red + 2 * kConsumerWarps + 8;         // kConsumerWarps * tr row-dot partials (n >= 32)
  uint64_t* full = reinterpret_cast<uint64_t*>(p1 + kConsumerWarps * tr);
  uint64_t* empty = full + S;
  __shared__ int s_abort;

  const int G = (n >= 256) ? 1 : max(1, 256 / n);   // row groups in phase 2 (n < 256)
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kConsumerWarps); }
    fence_mbar_init();
    s_abort = 0;
  }
  for (int i = tid; i < n; i += blockDim.x) xs[i] = a.x[i];
  __syncthreads();

  const uint32_t tile_bytes = (uint32_t)(stage_doubles * sizeof(double));
  const uint64_t deadline = gtimer() + LS_WAIT_NS;

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      prefetch_tmap(&map);
      int k = 0;
      for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
        const int s = k % S;
        if (k >= S) {
          if (!mbar_wait_bounded(&empty[s], ((k / S) - 1) & 1, deadline)) {
            atomicOr(a.status, LS_DEV_TIMEOUT);
            s_abort = 1;
            break;
          }
        }
        mbar_arrive_expect_tx(&full[s], tile_bytes);
        double* dst = tiles + (size_t)s * stage_doubles;
        for (int q = 0; q < nbox; ++q) tma_load_2d(dst + (size_t)q * tr * boxw, &map, q * boxw, t * tr, &full[s]);
      }
      // drain: wait until every issued copy has landed before the CTA can exit
      const int issued = k;
      for (int kk = max(0, issued - S); kk < issued; ++kk)
        mbar_wait_bounded(&full[kk % S], (kk / S) & 1, deadline + LS_WAIT_NS);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  double acc[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u) acc[u] = 0.0;
  double rn2 = 0.0, dn2 = 0.0;               // per-thread accumulators (rows this thread finishes)
  const int g = tid / max(n, 1);             // phase-2 row group (n < 256)
  const int cg = tid - g * n;                // phase-2 column (n < 256)

  int k = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
    const int s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], (k / S) & 1, deadline);
    if (bar_any(!ok, 1, kConsumerWarps * 32)) {        // every consumer warp leaves together
      if (!ok) atomicOr(a.status, LS_DEV_TIMEOUT);
      break;
    }
    const double* tl = tiles + (size_t)s * stage_doubles;
    double* rt = rtile + (k & 1) * tr;
    const int64_t row0 = (int64_t)t * tr;
    const int rows = (int)((a.m - row0 < (int64_t)tr) ? (a.m - row0) : (int64_t)tr);

    if (n >= 32) {
      // phase 1 (n >= 32): every warp takes all tr rows, in groups of RG = 8
      // rows (4 when tr = 4) with LPR = 32 / RG lanes per row; lane (r, q) of
      // warp w sums the columns c = LPR ((w + r) mod 8) + q (mod 8 LPR) --
      // each row's columns are covered once over the 8 warps, and the
      // rotation by r puts the rows of a warp on different banks.  The LPR
      // lanes are combined by shuffles, the 8 warps in warp order by one
      // thread per row.  Per row this costs ~3.5 FP64 instructions besides
      // the FMAs, against 9 for a warp per row (a 5-level shuffle tree and the
      // row's scalar work on one lane).
      const int RG = tr < 8 ? tr : 8;
      const int LPR = 32 / RG, CS = 8 * LPR;
      const int rl = lane / LPR, q = lane - rl * LPR;
      double bj = 0.0, rpj = 0.0;
      if (tid < rows) {                       // issue the row's loads before the dots
        bj = a.b[row0 + tid];
        if (a.r_prev) rpj = a.r_prev[row0 + tid];
      }
      for (int r0 = 0; r0 < tr; r0 += RG) {
        const int r = r0 + rl;
        double dot = 0.0;
        if (r < rows)
          for (int c = LPR * ((warp + rl) & 7) + q; c < n; c += CS) dot += tl[tile_off(r, c, boxw, nbox, tr)] * xs[c];
        for (int o = LPR >> 1; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (q == 0) p1[warp * tr + r] = dot;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32));
      if (tid < tr) {
        double rj = 0.0;
        if (tid < rows) {
          double d = 0.0;
#pragma unroll
          for (int w = 0; w < kConsumerWarps; ++w) d += p1[w * tr + tid];
          rj = bj - d;
          rn2 += rj * rj;
          if (a.r_prev) { const double dl = rj - rpj; dn2 += dl * dl; }
          if (a.r_out) a.r_out[row0 + tid] = rj;
        }
        rt[tid] = rj;
      }
    } else
    // phase 1: r_j = b_j - A_j x, one warp per row
    for (int r = warp; r < tr; r += kConsumerWarps) {
      double dot = 0.0, bj = 0.0, rpj = 0.0;
      if (lane == 0 && r < rows) {           // issue the row's loads before the dot
        bj = a.b[row0 + r];
        if (a.r_prev) rpj = a.r_prev[row0 + r];
      }
      if (r < rows) {
        for (int c = lane; c < n; c += 32) dot += tl[tile_off(r, c, boxw, nbox, tr)] * xs[c];
      }
      dot = warp_sum(dot);
      if (lane == 0) {
        double rj = 0.0;
        if (r < rows) {
          const int64_t j = row0 + r;
          rj = bj - dot;
          rn2 += rj * rj;
          if (a.r_prev) { const double dl = rj - rpj; dn2 += dl * dl; }
          if (a.r_out) a.r_out[j] = rj;
        }
        rt[r] = rj;
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32));

    // phase 2: c_k += A_jk r_j over the tile's rows
    if (NPT > 1 || n >= 256) {
      for (int r = 0; r < rows; ++r) {
        const double rj = rt[r];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
          const int c = tid + 256 * u;
          if (c < n) acc[u] += tl[tile_off(r, c, boxw, nbox, tr)] * rj;
        }
      }
    } else if (g < G) {
      for (int r = g; r < rows; r += G) acc[0] += tl[r * boxw + cg] * rt[r];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // ------------------------------------------------- per-CTA partial out
  double* out = a.part + (size_t)blockIdx.x * (n + 2);
  if (n >= 256 || NPT > 1) {
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
      const int c = tid + 256 * u;
      if (c < n) out[c] = acc[u];
    }
  } else {
    // reduce the G row groups of each column in group order (tile memory is
    // free now: all stages consumed)
    double* gsum = tiles;
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32));
    if (g < G) gsum[g * n + cg] = acc[0];
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32));
    for (int c = tid; c < n; c += kConsumerWarps * 32) {
      double sum = 0.0;
      for (int q = 0; q < G; ++q) sum += gsum[q * n + c];
      out[c] = sum;
    }
  }
  rn2 = warp_sum(rn2);
  dn2 = warp_sum(dn2);
  if (lane == 0) { red[warp] = rn2; red[kConsumerWarps + warp] = dn2; }
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32));
  if (tid == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < kConsumerWarps; ++w) { s1 += red[w]; s2 += red[kConsumerWarps + w]; }
    out[n] = s1;
    out[n + 1] = s2;
  }
  (void)s_abort;
}

// k_fused_pass_ws: the same pass for n > 256 (tr = 16, 8 or 4), warp-
// specialized so that the FP64 pipe does not idle at block-wide barriers
// between the two uses of a tile.  Warps 0-3 (row group) form the row dots of
// tile k -- lane (r, q) of warp w sums the columns c = LPR ((w + r) mod 4) + q
// (mod 4 LPR), LPR = 32 / tr, in two interleaved chains -- combine them (two
// shuffles, then the 4 warps in warp order by one thread per row), form r_j
// and the norms, and hand r to the column group through an mbarrier; warps
// 4-7 (column group) add r_j A_jk to their columns for tile k while the row
// group runs ahead.  r has one buffer per tile stage (so the row group may be
// up to S - 1 tiles ahead) and the row-dot partials two; the column group
// releases a tile's stage and its r buffer.  Deterministic orders within a
// CTA, as in k_fused_pass.
template <int NPT2>
__global__ void __launch_bounds__(kThreads, 1) k_fused_pass_ws(const __grid_constant__ CUtensorMap map, PassArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  constexpr int kRW = kConsumerWarps / 2;          // row-group warps (the rest: column group)
  const int n = a.n, tr = a.tr, boxw = a.boxw, nbox = a.nbox, S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const size_t stage_doubles = (size_t)tr * nbox * boxw;
  double* tiles = reinterpret_cast<double*>(smem_raw);
  double* xs = tiles + S * stage_doubles;
  double* rtile = xs + ((n + 1) & ~1);              // [S][tr]
  double* red = rtile + 4 * tr;
  double* p1 = red + 2 * kConsumerWarps + 8;        // [2][kRW][tr] row-dot partials
  uint64_t* full = reinterpret_cast<uint64_t*>(p1 + kConsumerWarps * tr);
  uint64_t* empty = full + S;
  uint64_t* rready = empty + S;                     // [S] r of a tile written
  uint64_t* rfree = rready + S;                     // [S] r of a tile consumed
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kConsumerWarps - kRW); }
    for (int i = 0; i < S; ++i) { mbar_init(&rready[i], 1); mbar_init(&rfree[i], kConsumerWarps - kRW); }
    fence_mbar_init();
  }
  for (int i = tid; i < n; i += blockDim.x) xs[i] = a.x[i];
  __syncthreads();
  const uint32_t tile_bytes = (uint32_t)(stage_doubles * sizeof(double));
  double* out = a.part + (size_t)blockIdx.x * (n + 2);

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      prefetch_tmap(&map);
      int k = 0;
      for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
        const int s = k % S;
        if (k >= S && !mbar_wait_bounded(&empty[s], ((k / S) - 1) & 1, gtimer() + LS_WAIT_NS)) {
          atomicOr(a.status, LS_DEV_TIMEOUT);
          break;
        }
        mbar_arrive_expect_tx(&full[s], tile_bytes);
        double* dst = tiles + (size_t)s * stage_doubles;
        for (int q = 0; q < nbox; ++q) tma_load_2d(dst + (size_t)q * tr * boxw, &map, q * boxw, t * tr, &full[s]);
      }
      const int issued = k;
      for (int kk = max(0, issued - S); kk < issued; ++kk)
        mbar_wait_bounded(&full[kk % S], (kk / S) & 1, gtimer() + LS_WAIT_NS);
    }
    return;
  }

  if (warp < kRW) {
    // ------------------------------------------------------------ row group
    const int LPR = 32 / tr, CS = kRW * LPR;
    const int rl = lane / LPR, q = lane - rl * LPR;
    const int rho = LPR * ((warp + rl) % kRW) + q;
    double rn2 = 0.0, dn2 = 0.0;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
      const int s = k % S;
      bool ok = mbar_wait_bounded(&full[s], (k / S) & 1, gtimer() + LS_WAIT_NS);
      if (ok && k >= S) ok = mbar_wait_bounded(&rfree[s], ((k / S) - 1) & 1, gtimer() + LS_WAIT_NS);
      if (bar_any(!ok, 3, kRW * 32)) {                // the row group leaves together
        if (!ok) atomicOr(a.status, LS_DEV_TIMEOUT);
        break;
      }
      const double* tl = tiles + (size_t)s * stage_doubles;
      const int64_t row0 = (int64_t)t * tr;
      const int rows = (int)((a.m - row0 < (int64_t)tr) ? (a.m - row0) : (int64_t)tr);
      double bj = 0.0, rpj = 0.0;
      if (tid < rows) {                               // issue the row's loads before the dots
        bj = a.b[row0 + tid];
        if (a.r_prev) rpj = a.r_prev[row0 + tid];
      }
      // two accumulators: a dependent chain of FP64 FMAs issues one per FMA
      // latency, so two interleaved chains keep the row group's pipe fed
      double d0 = 0.0, d1 = 0.0;
      if (rl < rows) {
        int c = rho;
        for (; c + CS < n; c += 2 * CS) {
          d0 += tl[tile_off(rl, c, boxw, nbox, tr)] * xs[c];
          d1 += tl[tile_off(rl, c + CS, boxw, nbox, tr)] * xs[c + CS];
        }
        if (c < n) d0 += tl[tile_off(rl, c, boxw, nbox, tr)] * xs[c];
      }
      double dot = d0 + d1;
      for (int o = LPR >> 1; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      double* pk = p1 + (size_t)(k & 1) * kRW * tr;
      if (q == 0) pk[warp * tr + rl] = dot;
      asm volatile("bar.sync 2, %0;" ::"n"(kRW * 32));
      if (tid < tr) {
        double rj = 0.0;
        if (tid < rows) {
          double d = 0.0;
#pragma unroll
          for (int w = 0; w < kRW; ++w) d += pk[w * tr + tid];
          rj = bj - d;
          rn2 += rj * rj;
          if (a.r_prev) { const double dl = rj - rpj; dn2 += dl * dl; }
          if (a.r_out) a.r_out[row0 + tid] = rj;
        }
        rtile[s * tr + tid] = rj;
      }
      if (warp == 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&rready[s]);
      }
    }
    if (warp == 0) {
      rn2 = warp_sum(rn2);
      dn2 = warp_sum(dn2);
      if (lane == 0) { out[n] = rn2; out[n + 1] = dn2; }
    }
    return;
  }

  // -------------------------------------------------------------- column group
  const int tc = tid - kRW * 32;
  constexpr int kCT2 = (kConsumerWarps - kRW) * 32;
  double acc[NPT2];
#pragma unroll
  for (int u = 0; u < NPT2; ++u) acc[u] = 0.0;
  int k = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
    const int s = k % S;
    if (!mbar_wait_bounded(&full[s], (k / S) & 1, gtimer() + LS_WAIT_NS) ||
        !mbar_wait_bounded(&rready[s], (k / S) & 1, gtimer() + LS_WAIT_NS)) {
      atomicOr(a.status, LS_DEV_TIMEOUT);
      break;
    }
    const double* tl = tiles + (size_t)s * stage_doubles;
    const double* rt = rtile + s * tr;
    const int64_t row0 = (int64_t)t * tr;
    const int rows = (int)((a.m - row0 < (int64_t)tr) ? (a.m - row0) : (int64_t)tr);
    for (int r = 0; r < rows; ++r) {
      const double rj = rt[r];
#pragma unroll
      for (int u = 0; u < NPT2; ++u) {
        const int c = tc + kCT2 * u;
        if (c < n) acc[u] += tl[tile_off(r, c, boxw, nbox, tr)] * rj;
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&rfree[s]);
      mbar_arrive(&empty[s]);
    }
  }
#pragma unroll
  for (int u = 0; u < NPT2; ++u) {
    const int c = tc + kCT2 * u;
    if (c < n) out[c] = acc[u];
  }
}

// Sum the per-CTA partials in CTA order: c[k], norms[0..1].
__global__ void k_reduce_partials(const double* __restrict__ part, int nparts, int n, double* __restrict__ c,
                                  double* __restrict__ norms) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n + 2) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(size_t)p * (n + 2) + k];
  if (k < n) c[k] = s;
  else norms[k - n] = s;
}

// ------------------------------------------------------------ cluster steps
// Sum partial column k over CTAs (fixed order).
__device__ inline double part_sum(const double* part, int nparts, int n, int k) {
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += __ldcg(part + (size_t)p * (n + 2) + k);
  return s;
}

template <int PP>
__global__ void __launch_bounds__(256) k_iter_step(StepArgs a) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  TsSmem& sm = *reinterpret_cast<TsSmem*>(ts_raw);
  const CL cl = cl_this();
  const int n = a.n;
  IterState S = *a.st;       // every CTA reads the state before anyone writes it
  if (!S.done) ts_setup(cl, sm, a.R, a.ldr, a.inv_diag, n);
  cl_sync();
  if (S.done) return;

  // ||r_i||, ||r_i - r_{i-1}|| (every CTA computes them identically)
  // (warp w < 2 sums column n + w: lane j takes the partials j, j + 32, ...,
  // then a fixed butterfly)
  __shared__ double s_norm[2];
  if (threadIdx.x < 64) {
    const int col = n + (threadIdx.x >> 5);
    double t = 0.0;
    for (int p = threadIdx.x & 31; p < a.nparts; p += 32) t += __ldcg(a.part + (size_t)p * (n + 2) + col);
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) s_norm[threadIdx.x >> 5] = t;
  }
  __syncthreads();
  const double rnorm = sqrt(s_norm[0]);
  const double dnorm = S.have_prev ? sqrt(s_norm[1]) : 0.0;
  const double u = 0x1.0p-53;
  int fired = S.fired, extra_left = S.extra_left, done = 0;
  if (a.use_stop && S.have_prev && !fired) {
    if (dnorm <= u * (S.gamma * S.normest * S.xnorm + S.rho * S.condest * rnorm)) {
      fired = 1;
      extra_left = a.extra;
    }
  }
  if (fired) {
    if (extra_left == 0) done = 1;
    else extra_left -= 1;
  }
  if (done) {                // uniform over the cluster; nothing has been pushed yet
    if (cl.rank == 0 && threadIdx.x == 0) {
      a.st->done = 1; a.st->fired = 1; a.st->stop_reason = 0;
      a.st->rnorm = rnorm; a.st->dnorm = dnorm;
    }
    return;
  }

  // c = sum of partials on the owned rows; y = R^{-T} c; d = R^{-1} y
  const uint64_t deadline = gtimer() + 2000000000ull;
  int tmo = 0;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, q = w >> 1, h = w & 1;
  const int nb = (n + 31) / 32, mine = ts_owned(cl, nb);
  double c[PP], y[PP], dv[PP];
#pragma unroll
  for (int s = 0; s < PP; ++s) {
    const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
    c[s] = (h == 0 && o < mine && i < n) ? part_sum(a.part, a.nparts, n, i) : 0.0;
  }
  ts_solve<PP, false>(cl, sm, 0, a.Rt, n, a.inv_diag, n, c, y, deadline, tmo);
  ts_solve<PP, true>(cl, sm, 1, a.R, a.ldr, a.inv_diag, n, y, dv, deadline, tmo);

  // x+ = x + alpha d + beta (x - x_prev) on owned rows; ||x+||^2
  double xs = 0.0, bad = 0.0;
  if (h == 0) {
#pragma unroll
    for (int s = 0; s < PP; ++s) {
      const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
      if (o < mine && i < n) {
        const double xi = __ldcg(a.x + i), xp = __ldcg(a.x_prev + i);
        const double xn = xi + S.alpha * dv[s] + S.beta * (xi - xp);
        __stcg(a.x_prev + i, xi);
        __stcg(a.x + i, xn);
        xs += xn * xn;
        if (!isfinite(xn)) bad = 1.0;
      }
    }
  }
  ts_drain(sm, n, deadline, tmo);
  if (tmo) atomicOr(a.status, LS_DEV_TIMEOUT);
  const double xn2 = cl_sum(cl, cta_sum(xs), a.slots);
  const double anybad = cl_max(cl, cta_max(bad), a.slots);
  if (cl.rank == 0 && threadIdx.x == 0) {
    a.st->iter = S.iter + 1;
    a.st->fired = fired;
    a.st->extra_left = extra_left;
    a.st->have_prev = 1;
    a.st->xnorm = sqrt(xn2);
    a.st->rnorm = rnorm;
    a.st->dnorm = dnorm;
    if (anybad != 0.0) {
      a.st->nonfinite = 1; a.st->done = 1; a.st->stop_reason = 3;
      atomicOr(a.status, LS_DEV_NONFINITE);
    }
  }
}

// y = R^{-T} c, d = R^{-1} y, x += d (standalone correction).
template <int PP>
__global__ void __launch_bounds__(256) k_correct(StepArgs a) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  TsSmem& sm = *reinterpret_cast<TsSmem*>(ts_raw);
  const CL cl = cl_this();
  const int n = a.n;
  ts_setup(cl, sm, a.R, a.ldr, a.inv_diag, n);
  cl_sync();
  const uint64_t deadline = gtimer() + 2000000000ull;
  int tmo = 0;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, q = w >> 1, h = w & 1;
  const int nb = (n + 31) / 32, mine = ts_owned(cl, nb);
  double c[PP], y[PP], dv[PP];
#pragma unroll
  for (int s = 0; s < PP; ++s) {
    const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
    c[s] = (h == 0 && o < mine && i < n) ? __ldcg(a.c_in + i) : 0.0;
  }
  ts_solve<PP, false>(cl, sm, 0, a.Rt, n, a.inv_diag, n, c, y, deadline, tmo);
  ts_solve<PP, true>(cl, sm, 1, a.R, a.ldr, a.inv_diag, n, y, dv, deadline, tmo);
  if (h == 0) {
#pragma unroll
    for (int s = 0; s < PP; ++s) {
      const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
      if (o < mine && i < n) {
        __stcg(a.x + i, __ldcg(a.x + i) + dv[s]);
        if (a.y_out) a.y_out[i] = y[s];
        if (a.d_out) a.d_out[i] = dv[s];
      }
    }
  }
  ts_drain(sm, n, deadline, tmo);
  if (tmo) atomicOr(a.status, LS_DEV_TIMEOUT);
  cl_sync();
}

// ------------------------------------------------------------ host side
PassGeom pass_geometry(const ls_ctx* ctx, int64_t n, int64_t m) {
  PassGeom g;
  if (n <= 256) {
    g.boxw = (int)((n + 1) & ~1LL);
    g.nbox = 1;
    const int rowbytes = g.boxw * 8;
    int tr = (48 * 1024) / rowbytes;
    tr = (tr / 8) * 8;
    tr = std::max(8, std::min(256, tr));
    g.tr = tr;
  } else {
    g.boxw = 256;
    g.nbox = (int)((n + 255) / 256);
    g.tr = (g.nbox <= 2) ? 16 : (g.nbox <= 4) ? 8 : 4;
  }
  const size_t stage = (size_t)g.tr * g.nbox * g.boxw * sizeof(double);
  g.stages = (int)std::max<size_t>(2, std::min<size_t>(4, (200 * 1024) / stage));
  const int64_t ntiles = (m + g.tr - 1) / g.tr;
  g.grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms, ntiles));
  g.smem = g.stages * stage + (size_t)((n + 1) & ~1LL) * 8 + 4 * g.tr * 8 + (2 * kConsumerWarps + 8) * 8 +
           (size_t)kConsumerWarps * g.tr * 8 + 4 * g.stages * 8 + 128;
  // phase-2 group sums for n < 256 reuse the tile memory
  return g;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t make_tensor_map(ls_ctx* ctx, CUtensorMap* map, const double* A, int64_t m, int64_t n, int64_t lda,
                            const PassGeom& g) {
  if (!ctx->encode_tiled) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    ctx->encode_tiled = fn;
  }
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(double)};
  cuuint32_t box[2] = {(cuuint32_t)g.boxw, (cuuint32_t)g.tr};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ((EncodeTiledFn)ctx->encode_tiled)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)A, dims, strides, box,
                                                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int NPT>
static cudaError_t launch_pass_t(ls_ctx* ctx, const CUtensorMap& map, const PassGeom& g, const PassArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(k_fused_pass<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  k_fused_pass<NPT><<<g.grid, kThreads, g.smem, ctx->stream>>>(map, a);
  ++ctx->launches;
  return cudaGetLastError();
}

template <int NPT2>
static cudaError_t launch_pass_ws(ls_ctx* ctx, const CUtensorMap& map, const PassGeom& g, const PassArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(k_fused_pass_ws<NPT2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  k_fused_pass_ws<NPT2><<<g.grid, kThreads, g.smem, ctx->stream>>>(map, a);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_fused_pass(ls_ctx* ctx, const CUtensorMap& map, const PassGeom& g, int64_t m, int64_t n,
                              const double* b, const double* x, const double* r_prev, double* r_out, double* part,
                              const IterState* st) {
  PassArgs a;
  a.m = m; a.n = (int)n; a.boxw = g.boxw; a.nbox = g.nbox; a.tr = g.tr; a.stages = g.stages;
  a.ntiles = (int)((m + g.tr - 1) / g.tr);
  a.b = b; a.x = x; a.r_prev = r_prev; a.r_out = r_out; a.part = part; a.st = st; a.status = ctx->d_status;
  if (g.nbox > 1) {                      // n > 256: the warp-specialized form
    const int npt2 = (int)((n + 127) / 128);
    if (npt2 <= 8) return launch_pass_ws<8>(ctx, map, g, a);
    if (npt2 <= 16) return launch_pass_ws<16>(ctx, map, g, a);
    return cudaErrorInvalidValue;
  }
  const int npt = (int)((n + 255) / 256);
  if (npt <= 1) return launch_pass_t<1>(ctx, map, g, a);
  if (npt <= 2) return launch_pass_t<2>(ctx, map, g, a);
  if (npt <= 4) return launch_pass_t<4>(ctx, map, g, a);
  if (npt <= 8) return launch_pass_t<8>(ctx, map, g, a);
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_partials(ls_ctx* ctx, const double* part, int nparts, int64_t n, double* c,
                                   double* norms) {
  const int threads = 256;
  const int grid = (int)((n + 2 + threads - 1) / threads);
  k_reduce_partials<<<grid, threads, 0, ctx->stream>>>(part, nparts, (int)n, c, norms);
  ++ctx->launches;
  return cudaGetLastError();
}

// Cluster size for kernels built on the broadcast substitutions: 16 CTAs
// where the device can hold such a cluster of every listed kernel with the
// solves' shared memory (TsSmem), else 8.  Sets the kernels' attributes.
int ts_cluster_size_of(const void* const* fns, int nfn) {
  bool ok16 = true;
  for (int f = 0; f < nfn; ++f) {
    cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TsSmem));
    if (cudaFuncSetAttribute(fns[f], cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ok16 = false;
  }
  cudaGetLastError();
  if (ok16) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sizeof(TsSmem);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    for (int f = 0; f < nfn; ++f)
      if (cudaOccupancyMaxActiveClusters(&nclusters, fns[f], &cfg) != cudaSuccess || nclusters < 1) ok16 = false;
    cudaGetLastError();
  }
  return ok16 ? 16 : 8;
}

int ts_cluster_size() {
  static int size = -1;
  if (size > 0) return size;
  const void* fns[] = {(const void*)k_iter_step<1>, (const void*)k_iter_step<2>, (const void*)k_correct<1>,
                       (const void*)k_correct<2>};
  size = ts_cluster_size_of(fns, 4);
  return size;
}

static cudaError_t launch_ts(ls_ctx* ctx, const void* f1, const void* f2, const StepArgs& a) {
  // the smallest power-of-two cluster, up to the largest that fits, that
  // still gives every CTA at most one block of 32 rows: small n then meets
  // fewer CTAs at every cluster barrier and pushes to fewer
  int P = ts_cluster_size();
  const int nb = (a.n + 31) / 32;
  while (P > 1 && P / 2 >= nb) P /= 2;
  const int pp = ts_slots(a.n, P);
  if (pp == 0 || a.n > kTsMaxN) return cudaErrorInvalidValue;
  StepArgs aa = a;
  void* args[] = {&aa};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sizeof(TsSmem);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++ctx->launches;
  return cudaLaunchKernelExC(&cfg, pp == 1 ? f1 : f2, args);
}

cudaError_t launch_iter_step(ls_ctx* ctx, const StepArgs& a) {
  return launch_ts(ctx, (const void*)k_iter_step<1>, (const void*)k_iter_step<2>, a);
}

cudaError_t launch_correct(ls_ctx* ctx, const StepArgs& a) {
  return launch_ts(ctx, (const void*)k_correct<1>, (const void*)k_correct<2>, a);
}

}  // namespace lsk
