// factor.cu -- Householder QR of the sketch B_aug = [S A  S b] (Algorithm 2,
// QR step; Sec. 3.2, Eq. (3.4)), the sketch-and-solve start
// x0 = R^{-1} (Q^T S b) (Sec. 2.3, Eq. (2.5)) and the two estimates of the
// Sec. 3.3 stopping rule.
//
// Three QR kernels, chosen by the rows per CTA (ch = ceil(d / P)):
//   k_householder_la (ch <= 436): blocked compact-WY with one panel of
//     lookahead (two panel buffers in shared memory);
//   k_householder_blocked (ch <= 600): the same steps, one panel buffer;
//   k_householder (taller slices): unblocked, described next.
//
// k_householder: one cooperative launch, P CTAs, each owning a contiguous
// slice of the d rows.  Column k is reduced with three bounded grid barriers:
//   1. partial sums of squares of column k below the diagonal  -> barrier
//   2. every CTA forms the same reflector (fixed-order sum of the partials),
//      scales its slice of v, and forms partial dots v^T B[:, j]  -> barrier
//   3. CTA p reduces the dots of columns j with (j-k-1) mod P == p -> barrier
//   4. every CTA updates its slice: B[:, j] -= (tau w_j) v
// The reflector convention is LAPACK's (beta = -sign(alpha) ||x||, sign(0) = +,
// tau = (beta - alpha)/beta, v = x / (alpha - beta) with v_k = 1); the same
// reflectors are applied to column n (S b), which yields Q^T S b.
//
// k_prepare_R: R (upper, strictly-lower part zeroed), its transpose Rt and
// the reciprocal diagonal used by every later substitution.
//
// k_post_factor: one thread-block cluster (16 CTAs where they fit).  Solves
// R x0 = (Q^T S b)[0:n], runs ceil(ln n) power steps on R (normest) and
// Hager's 1-norm estimator of ||R^{-1}||_1 times ||R||_1 (condest); the
// substitutions are the broadcast ones of cluster_la.cuh.
#include <algorithm>

#include "cluster_la.cuh"

namespace lsk {

__global__ void __launch_bounds__(256) k_householder(double* __restrict__ B, int64_t d, int n, int64_t ldb,
                                                     double* __restrict__ part, double* __restrict__ w,
                                                     GridBar gb) {
  extern __shared__ double vs[];  // this CTA's slice of the current v
  __shared__ double s_ab[4];      // alpha, beta, tau, scal
  __shared__ int s_bad;
  const int P = gridDim.x, p = blockIdx.x;
  const int ncols = n + 1;
  const int64_t chunk = (d + P - 1) / P;
  const int64_t r0 = (int64_t)p * chunk, r1 = min(d, r0 + chunk);
  const int PS = ncols + 1;          // stride of one CTA's partials
  double* alpha_slot = part + (size_t)P * PS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;

  for (int k = 0; k < n; ++k) {
    // ---- phase 1: partial ||B[k+1:, k]||^2, publish alpha
    const int64_t lo = max(r0, (int64_t)k + 1);
    double ss = 0.0;
    for (int64_t i = lo + threadIdx.x; i < r1; i += blockDim.x) {
      const double v = B[i + (int64_t)k * ldb];
      ss += v * v;
    }
    ss = cta_sum(ss);
    if (threadIdx.x == 0) {
      __stcg(part + (size_t)p * PS, ss);
      if (k >= r0 && k < r1) __stcg(alpha_slot, B[k + (int64_t)k * ldb]);
    }
    if (!grid_sync(gb, P)) return;

    // ---- phase 2: reflector (identical in every CTA), scale v, partial dots
    if (warp == 0) {
      double t = 0.0;
      for (int q = lane; q < P; q += 32) t += __ldcg(part + (size_t)q * PS);
      t = warp_sum(t);
      if (lane == 0) {
        const double alpha = __ldcg(alpha_slot);
        const double xnorm = sqrt(t);
        double beta, tau, scal;
        if (xnorm == 0.0) {
          beta = alpha; tau = 0.0; scal = 1.0;
        } else {
          const double h = hypot(alpha, xnorm);
          beta = (alpha >= 0.0) ? -h : h;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        s_ab[0] = alpha; s_ab[1] = beta; s_ab[2] = tau; s_ab[3] = scal;
        s_bad = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (s_bad) {
      if (p == 0 && threadIdx.x == 0) atomicOr(gb.status, LS_DEV_RANK);
      return;   // every CTA takes the same decision
    }
    const double tau = s_ab[2], scal = s_ab[3];
    const int64_t vlo = max(r0, (int64_t)k);   // rows of v in this slice (v_k = 1)
    for (int64_t i = vlo + threadIdx.x; i < r1; i += blockDim.x) {
      double v;
      if (i == k) {
        v = 1.0;
      } else {
        v = B[i + (int64_t)k * ldb];
        if (tau != 0.0) { v = v * scal; B[i + (int64_t)k * ldb] = v; }
      }
      vs[i - r0] = v;
    }
    if (threadIdx.x == 0 && k >= r0 && k < r1) B[k + (int64_t)k * ldb] = s_ab[1];
    __syncthreads();
    for (int j = k + 1 + warp; j < ncols; j += nwarp) {
      double s = 0.0;
      if (tau != 0.0)
        for (int64_t i = vlo + lane; i < r1; i += 32) s += vs[i - r0] * B[i + (int64_t)j * ldb];
      s = warp_sum(s);
      if (lane == 0) __stcg(part + (size_t)p * PS + 1 + j, s);
    }
    if (!grid_sync(gb, P)) return;

    // ---- phase 3: w_j = sum over CTAs (fixed order), columns dealt round robin
    if (tau != 0.0) {
      for (int j = k + 1 + p * nwarp + warp; j < ncols; j += P * nwarp) {
        double s = 0.0;
        for (int q = lane; q < P; q += 32) s += __ldcg(part + (size_t)q * PS + 1 + j);
        s = warp_sum(s);
        if (lane == 0) __stcg(w + j, s);
      }
    }
    if (!grid_sync(gb, P)) return;

    // ---- phase 4: B[:, j] -= (tau w_j) v on this slice
    if (tau != 0.0) {
      for (int j = k + 1 + warp; j < ncols; j += nwarp) {
        const double tw = tau * __ldcg(w + j);
        for (int64_t i = vlo + lane; i < r1; i += 32) {
          double* bp = B + i + (int64_t)j * ldb;
          *bp = *bp - tw * vs[i - r0];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ blocked QR
// k_householder_blocked: the same reflectors, applied panel by panel
// (Schreiber-Van Loan compact WY).  For each panel of kNB columns:
//   * the panel slice of this CTA's rows is factored in shared memory, one
//     column at a time (two grid barriers per column: norm partials, then dot
//     partials), exactly the unblocked steps restricted to the panel;
//   * the trailing columns (including S b) get C <- C - V (T^T (V^T C))
//     with T the Schreiber-Van Loan factor (T[b][b] = tau_b,
//     T[0:b, b] = -tau_b T[0:b, 0:b] G[0:b, b], G = V^T V).  T is not
//     formed: T^{-1} = diag(1 / tau) + striu(G), so W' = T^T W is a forward
//     substitution with G.  W = V^T C is summed over CTAs in CTA order, G's
//     strict upper triangle is summed by CTA e mod P for entry e (one more
//     grid barrier), and every CTA updates its own rows.  The products run
//     on (32 columns, quarter) tasks with V broadcast from shared memory:
//     an FP64 warp instruction costs its sub-partition the same time however
//     many lanes are active, so work is dealt in whole warps, evenly over the
//     four sub-partitions.
static constexpr int kNB = 32;

struct HhArgs {
  double* B; int64_t d; int n; int64_t ldb;
  double* part;   // householder_part_doubles()
  double* Wp;     // kNB * (n + 1)
  GridBar gb;
};

__device__ inline int panel_ld(int64_t ch) { return (int)(ch + 1 + (ch & 1)); }   // odd stride

__global__ void __launch_bounds__(256, 1) k_householder_blocked(HhArgs a) {
  extern __shared__ double sm[];
  __shared__ double s_tau[kNB], s_beta[kNB];
  __shared__ double s_par[3];
  __shared__ int s_bad;
  const int P = gridDim.x, p = blockIdx.x;
  const int n = a.n, ncols = n + 1;
  const int64_t ch = (a.d + P - 1) / P;
  const int64_t r0 = (int64_t)p * ch;
  const int64_t r1 = min(a.d, r0 + ch);
  const int nrow = (int)max((int64_t)0, r1 - r0);
  const int ldp = panel_ld(ch);
  double* Ps = sm;                           // kNB columns x ldp (column-major)
  double* Ts = Ps + (size_t)kNB * ldp;       // T, row-major kNB x kNB
  double* Gs = Ts + kNB * kNB;               // G, row-major kNB x kNB
  double* pnorm = a.part;                    // [P]
  double* alpha_slot = a.part + P;           // [1]
  double* pdot = a.part + P + 8;             // [P][kNB]
  double* pW = pdot + (size_t)P * kNB;       // [P][kNB][ncols]
  double* pG = pW + (size_t)P * kNB * ncols; // [P][kNB*kNB]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  double* B = a.B;
  const int64_t ldb = a.ldb;
  MonoBar mb{a.gb.count, a.gb.status, 0u};

  // norm partial of panel column kk (global column k) over own rows > k; owner publishes alpha
  auto norm_partial = [&](int kk, int k) {
    double ss = 0.0;
    for (int i = threadIdx.x; i < nrow; i += blockDim.x)
      if (r0 + i > k) { const double v = Ps[kk * ldp + i]; ss += v * v; }
    ss = cta_sum(ss);
    if (threadIdx.x == 0) {
      __stcg(pnorm + p, ss);
      if (k >= r0 && k < r1) __stcg(alpha_slot, Ps[kk * ldp + (k - r0)]);
    }
  };

  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int nbp = min(kNB, n - k0);
    for (int e = threadIdx.x; e < kNB * nrow; e += blockDim.x) {
      const int c = e / nrow, i = e - c * nrow;
      Ps[c * ldp + i] = (c < nbp) ? B[(r0 + i) + (int64_t)(k0 + c) * ldb] : 0.0;
    }
    __syncthreads();
    norm_partial(0, k0);
    mono_arrive(mb);

    // ---------------------------------------------------- panel factorization
    // Two grid barriers per column (norm partials, then dot partials).  The
    // next column is updated first and its norm partial published before the
    // rest of the panel is updated, so that update overlaps the barrier.
    for (int kk = 0; kk < nbp; ++kk) {
      const int k = k0 + kk;
      if (!mono_wait(mb, P)) return;
      if (warp == 0) {
        double t = 0.0;
        for (int q = lane; q < P; q += 32) t += __ldcg(pnorm + q);
        t = warp_sum(t);
        if (lane == 0) {
          const double alpha = __ldcg(alpha_slot);
          double beta, tau, scal;
          if (t == 0.0) {
            beta = alpha; tau = 0.0; scal = 1.0;
          } else {
            // ||[alpha; x]|| from the sum of squares already formed (the
            // partials overflow before this could)
            const double h = sqrt(alpha * alpha + t);
            beta = (alpha >= 0.0) ? -h : h;
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
          }
          s_par[0] = beta; s_par[1] = tau; s_par[2] = scal;
          s_tau[kk] = tau; s_beta[kk] = beta;
          s_bad = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        }
      }
      __syncthreads();
      if (s_bad) {
        if (p == 0 && threadIdx.x == 0) atomicOr(a.gb.status, LS_DEV_RANK);
        return;
      }
      const double tau = s_par[1], scal = s_par[2];
      for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
        const int64_t g = r0 + i;
        if (g == k) Ps[kk * ldp + i] = 1.0;
        else if (g > k && tau != 0.0) Ps[kk * ldp + i] *= scal;
      }
      __syncthreads();
      if (kk + 1 < nbp) {
        // dots of v with the remaining panel columns (own rows >= k)
        const int i0 = (int)max((int64_t)0, (int64_t)k - r0);
        for (int jj = kk + 1 + warp; jj < nbp; jj += nwarp) {
          double s = 0.0;
          if (tau != 0.0)
            for (int i = i0 + lane; i < nrow; i += 32) s += Ps[kk * ldp + i] * Ps[jj * ldp + i];
          s = warp_sum(s);
          if (lane == 0) __stcg(pdot + (size_t)p * kNB + jj, s);
        }
        if (!mono_sync(mb, P)) return;
        __shared__ double s_w[kNB];      // tau (v^T a_jj)
        for (int jj = kk + 1 + warp; jj < nbp; jj += nwarp) {
          double s = 0.0;
          for (int q = lane; q < P; q += 32) s += __ldcg(pdot + (size_t)q * kNB + jj);
          s = warp_sum(s);
          if (lane == 0) s_w[jj] = tau * s;
        }
        __syncthreads();
        if (tau != 0.0)
          for (int i = threadIdx.x; i < nrow; i += blockDim.x)
            if (r0 + i >= k) Ps[(kk + 1) * ldp + i] -= s_w[kk + 1] * Ps[kk * ldp + i];
        __syncthreads();
        norm_partial(kk + 1, k + 1);
        mono_arrive(mb);
        if (tau != 0.0) {
          for (int e = threadIdx.x; e < (nbp - kk - 2) * nrow; e += blockDim.x) {
            const int jj = kk + 2 + e / nrow, i = e % nrow;
            if (r0 + i >= k) Ps[jj * ldp + i] -= s_w[jj] * Ps[kk * ldp + i];
          }
        }
      }
    }
    __syncthreads();

    // ---------------------------------------------------- write back, form V
    for (int e = threadIdx.x; e < nbp * nrow; e += blockDim.x) {
      const int c = e / nrow, i = e - c * nrow;
      const int64_t g = r0 + i;
      const double v = Ps[c * ldp + i];
      B[g + (int64_t)(k0 + c) * ldb] = (g == k0 + c) ? s_beta[c] : v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNB * nrow; e += blockDim.x) {
      const int c = e / nrow, i = e - c * nrow;
      const int64_t g = r0 + i;
      if (c >= nbp || g < k0 + c) Ps[c * ldp + i] = 0.0;
      else if (g == k0 + c) Ps[c * ldp + i] = 1.0;
    }
    __syncthreads();

    // ---------------------------------------------------- partial G and W = V^T C
    // G: the 496 entries r < c of V^T V over own rows, packed as
    // e = c (c - 1) / 2 + r; 16 lane sets of 32 entries, two per warp, so that
    // every lane has work.  W: tasks (group of 32 columns, quarter h of the
    // kNB reflectors); warp w takes quarter w mod 4 of every other group, so
    // each sub-partition gets the same number of FP64 instructions.
    const int i0 = (int)max((int64_t)0, (int64_t)k0 - r0);
    for (int ls = 2 * warp; ls < 2 * warp + 2; ++ls) {
      const int e = 32 * ls + lane;
      if (e < kNB * (kNB - 1) / 2) {
        int c = 1;
        while ((c + 1) * c / 2 <= e) ++c;
        const int r = e - c * (c - 1) / 2;
        double g = 0.0;
        if (c < nbp)
          for (int i = i0; i < nrow; ++i) g += Ps[r * ldp + i] * Ps[c * ldp + i];
        __stcg(pG + (size_t)p * kNB * kNB + e, g);
      }
    }
    const int jt0 = k0 + nbp;
    const int ngroups = (ncols - jt0 + 31) / 32;
    {
      const int h = warp & 3;
      for (int g = warp >> 2; g < ngroups; g += 2) {
        const int j = jt0 + 32 * g + lane;
        if (j < ncols) {
          double acc[kNB / 4];
#pragma unroll
          for (int q = 0; q < kNB / 4; ++q) acc[q] = 0.0;
          const double* cp = B + (int64_t)j * ldb + r0;
          const double* vp = Ps + (size_t)(h * (kNB / 4)) * ldp;
#pragma unroll 2
          for (int i = i0; i < nrow; ++i) {
            const double c = cp[i];
#pragma unroll
            for (int q = 0; q < kNB / 4; ++q) acc[q] += vp[q * ldp + i] * c;
          }
          double* out = pW + ((size_t)p * kNB + h * (kNB / 4)) * ncols + j;
#pragma unroll
          for (int q = 0; q < kNB / 4; ++q) __stcg(out + (size_t)q * ncols, acc[q]);
        }
      }
    }
    if (!mono_sync(mb, P)) return;

    // ---------------------------------------------------- G summed over CTAs (CTA p: entries p, p + P, ...)
    double* Gred = a.Wp + (size_t)kNB * ncols + 8;
    for (int e = p + warp * P; e < kNB * (kNB - 1) / 2; e += nwarp * P) {
      double g = 0.0;
      for (int q = lane; q < P; q += 32) g += __ldcg(pG + (size_t)q * kNB * kNB + e);
      g = warp_sum(g);
      if (lane == 0) __stcg(Gred + e, g);
    }
    if (!mono_sync(mb, P)) return;

    // ---------------------------------------------------- W' = T^T W
    // T^{-1} = diag(1 / tau) + striu(V^T V) (Schreiber-Van Loan T, in the
    // Puglisi form), so W' solves (diag(1 / tau) + striu(G))^T W' = W by
    // forward substitution over the reflectors: W'_q = tau_q (W_q -
    // sum_{r<q} G_rq W'_r).  With M_rq = G_rq tau_r each step is one FMA:
    // lane q keeps W_q - sum_r M_rq (W_r - ...), scaled by tau_q at the end.
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, q = e - r * kNB;
      double mv = 0.0;
      if (r < q && q < nbp) mv = __ldcg(Gred + q * (q - 1) / 2 + r) * s_tau[r];
      Gs[e] = mv;
    }
    __syncthreads();
    {
      const double tq = (lane < nbp) ? s_tau[lane] : 0.0;
      for (int j = jt0 + p * nwarp + warp; j < ncols; j += P * nwarp) {
        double w = 0.0;
        for (int q = 0; q < P; ++q) w += __ldcg(pW + ((size_t)q * kNB + lane) * ncols + j);
        for (int r = 0; r + 1 < nbp; ++r) {
          const double t = __shfl_sync(0xffffffffu, w, r);
          if (lane > r) w = w - Gs[r * kNB + lane] * t;
        }
        __stcg(a.Wp + (size_t)lane * ncols + j, w * tq);
      }
    }
    if (!mono_sync(mb, P)) return;

    // ---------------------------------------------------- C -= V W' on own rows
    // tasks (group of 32 columns, quarter h of the rows i0..nrow)
    {
      const int h = warp & 3;
      const int len = nrow - i0;
      const int ia = i0 + (int)(((int64_t)len * h) / 4), ib = i0 + (int)(((int64_t)len * (h + 1)) / 4);
      for (int g = warp >> 2; g < ngroups; g += 2) {
        const int j = jt0 + 32 * g + lane;
        if (j < ncols && ia < ib) {
          double wv[kNB];
#pragma unroll
          for (int q = 0; q < kNB; ++q) wv[q] = __ldcg(a.Wp + (size_t)q * ncols + j);
          double* cp = B + (int64_t)j * ldb + r0;
          for (int i = ia; i < ib; ++i) {
            double c = cp[i];
#pragma unroll
            for (int q = 0; q < kNB; ++q) c -= Ps[q * ldp + i] * wv[q];
            cp[i] = c;
          }
        }
      }
    }
    __syncthreads();
    if (k0 + kNB < n) {
      // the next panel's first column was just updated by this CTA
    }
  }
}


// ------------------------------------------------------------ blocked QR with lookahead
// k_householder_la: the reflectors of k_householder_blocked, with the
// factorization of panel p+1 overlapped with the trailing update of panel p.
// Once W'_p is known, all warps first update panel p+1's columns on their own
// rows; then warps 0..w-1 of every CTA factor panel p+1 (into the second
// panel buffer, with the grid barriers of its columns) while the other warps
// -- and the panel's once it is done -- apply panel p to the remaining
// trailing columns, taking (32-column group, row chunk) tasks from a shared
// counter.  w is 2 or 4 while the update is long; once it is short the
// panel is factored by all 8 warps after the update.
// The panel is latency-bound and the update FP64-bound, so the two fill each
// other's idle time.  A panel column takes one grid barrier: every CTA
// publishes, for the column x below its diagonal row, the partial sum of
// squares and the partial dots x^T a_jj with the later panel columns (and
// the owner of the diagonal row publishes that row), so that after the
// barrier every CTA has the reflector and v^T a_jj = a_jj,k + scal x^T a_jj
// at once (two barriers per column before: 46.0 -> 43.4 ms at d = 20,000,
// n = 1000, with the lookahead thresholds retuned).  Panel 0 is factored by
// all warps.  Row dots of a panel column are summed per warp slice of the
// rows, then over warps in warp order; CTA partials in CTA-range order.
static constexpr int kLaTasksPerGroup = 8;

__global__ void __launch_bounds__(256, 1) k_householder_la(HhArgs a) {
  extern __shared__ double sm[];
  __shared__ double s_tau[kNB], s_beta[kNB], s_par[3], s_w[kNB];
  __shared__ double s_red[8][kNB];
  __shared__ int s_bad, s_task, s_abort, s_gok;
  const int P = gridDim.x, p = blockIdx.x;
  const int n = a.n, ncols = n + 1;
  const int64_t ch = (a.d + P - 1) / P;
  const int64_t r0 = (int64_t)p * ch;
  const int64_t r1 = min(a.d, r0 + ch);
  const int nrow = (int)max((int64_t)0, r1 - r0);
  const int ldp = panel_ld(ch);
  double* pbuf0 = sm;                                 // two panel buffers, kNB columns x ldp
  double* pbuf1 = sm + (size_t)kNB * ldp;
  double* Gs = sm + (size_t)2 * kNB * ldp;            // W' multipliers, kNB x kNB
  double* pdot = a.part + P + 8;             // [P][kNB]
  double* pW = pdot + (size_t)P * kNB;       // [P][kNB][ncols]
  double* pG = pW + (size_t)P * kNB * ncols; // [P][kNB*kNB]
  // column kk of a panel uses buffer kk & 1 of the dot partials and of row k
  // (a CTA writes column kk + 2's only after every CTA has read column kk's)
  double* rowk0 = pG + (size_t)P * kNB * kNB;     // [2][kNB]: row k of the panel
  double* pdot1 = rowk0 + 2 * kNB;                  // second buffer of pdot, [P][kNB]
  double* Gred = a.Wp + (size_t)kNB * ncols + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* B = a.B;
  const int64_t ldb = a.ldb;
  MonoBar mb{a.gb.count, a.gb.status, 0u};
  if (threadIdx.x == 0) s_abort = 0;

  // the nw warps 0..nw-1 meet (all 8: the CTA barrier)
  auto gsync = [&](int nw) {
    if (nw == 8) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"r"(32 * nw) : "memory");
  };
  auto g_arrive = [&](int nw) {
    gsync(nw);
    if (threadIdx.x == 0) { __threadfence(); atomicAdd(mb.count, 1u); }
    ++mb.epoch;
  };
  auto g_wait = [&](int nw) -> bool {
    if (threadIdx.x == 0) {
      const unsigned int target = mb.epoch * (unsigned int)P;
      int ok = 1;
      const uint64_t deadline = gtimer() + LS_WAIT_NS;
      uint32_t spins = 0;
      for (;;) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(mb.count) : "memory");
        if ((int)(v - target) >= 0) break;
        if ((++spins & 63u) == 0) {
          if (gtimer() > deadline) { atomicOr(mb.status, LS_DEV_TIMEOUT); ok = 0; break; }
          if (*(volatile unsigned int*)mb.status & LS_DEV_TIMEOUT) { ok = 0; break; }
        }
      }
      s_gok = ok;
    }
    gsync(nw);
    return s_gok != 0;
  };
  // Partials of panel column kk (global k) over own rows > k: lane 0 the sum
  // of squares, lane l its dot with panel column kk + l; the owner of row k
  // publishes row k of the panel (alpha and the a_jj,k).  One grid barrier
  // then gives every CTA the reflector and all its dots at once:
  // v^T a_jj = a_jj,k + scal (x^T a_jj) with x the column below row k.
  auto col_partials = [&](const double* Pn, int kk, int k, int nbp, int nw) {
    double* pd = (kk & 1) ? pdot1 : pdot;
    double* rowk = rowk0 + (kk & 1) * kNB;
    const int i0 = (int)max((int64_t)0, (int64_t)k + 1 - r0);
    const int len = max(0, nrow - i0);
    const int ia = i0 + (len * warp) / nw, ib = i0 + (len * (warp + 1)) / nw;
    const int jj = kk + lane;
    double s = 0.0;
    if (jj < nbp)
      for (int i = ia; i < ib; ++i) s += Pn[kk * ldp + i] * Pn[jj * ldp + i];
    s_red[warp][lane] = s;
    gsync(nw);
    if (warp == 0 && jj < nbp) {
      double d = 0.0;
      for (int w = 0; w < nw; ++w) d += s_red[w][lane];
      __stcg(pd + (size_t)p * kNB + jj, d);
      if (k >= r0 && k < r1) __stcg(rowk + jj, Pn[jj * ldp + (k - r0)]);
    }
  };

  // Factor the panel of columns k0 .. k0+nbp-1 (own rows) into Pn with warps
  // 0..nw-1; the CTA's other warps do not take part.  One grid barrier per
  // column.  False: rank deficiency or a timed-out barrier (status set).
  auto factor_panel = [&](double* Pn, int k0, int nbp, int nw) -> bool {
    const int nthr = 32 * nw;
    for (int e = threadIdx.x; e < kNB * nrow; e += nthr) {
      const int c = e / nrow, i = e - c * nrow;
      Pn[c * ldp + i] = (c < nbp) ? B[(r0 + i) + (int64_t)(k0 + c) * ldb] : 0.0;
    }
    gsync(nw);
    col_partials(Pn, 0, k0, nbp, nw);
    g_arrive(nw);
    for (int kk = 0; kk < nbp; ++kk) {
      const int k = k0 + kk;
      if (!g_wait(nw)) return false;
      // sums over CTAs: warp w takes a contiguous range of CTAs, lane l the
      // entry kk + l; then the reflector and the multipliers w_jj = tau v^T a_jj
      const int jj = kk + lane;
      const double* pd = (kk & 1) ? pdot1 : pdot;
      const double* rowk = rowk0 + (kk & 1) * kNB;
      double s = 0.0;
      if (jj < nbp)
        for (int q = (P * warp) / nw; q < (P * (warp + 1)) / nw; ++q) s += __ldcg(pd + (size_t)q * kNB + jj);
      s_red[warp][lane] = s;
      gsync(nw);
      if (warp == 0) {
        double d = 0.0;
        for (int w = 0; w < nw; ++w) d += s_red[w][lane];
        const double t = __shfl_sync(0xffffffffu, d, 0);
        const double alpha = __ldcg(rowk + kk);
        double beta, tau, scal;
        if (t == 0.0) {
          beta = alpha; tau = 0.0; scal = 1.0;
        } else {
          const double h = sqrt(alpha * alpha + t);
          beta = (alpha >= 0.0) ? -h : h;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        if (lane == 0) {
          s_par[1] = tau; s_par[2] = scal;
          s_tau[kk] = tau; s_beta[kk] = beta;
          s_bad = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        } else if (jj < nbp) {
          s_w[jj] = (tau != 0.0) ? tau * (__ldcg(rowk + jj) + scal * d) : 0.0;
        }
      }
      gsync(nw);
      if (s_bad) {
        if (p == 0 && threadIdx.x == 0) atomicOr(a.gb.status, LS_DEV_RANK);
        return false;
      }
      const double tau = s_par[1], scal = s_par[2];
      // v = [1; x scal] on own rows >= k; a_jj -= w_jj v for the later columns
      for (int i = threadIdx.x; i < nrow; i += nthr) {
        const int64_t g = r0 + i;
        if (g < k) continue;
        const double x = Pn[kk * ldp + i];
        const double v = (g == k) ? 1.0 : ((tau != 0.0) ? x * scal : x);
        if (tau != 0.0)
          for (int c = kk + 1; c < nbp; ++c) Pn[c * ldp + i] -= s_w[c] * v;
        Pn[kk * ldp + i] = v;
      }
      gsync(nw);
      if (kk + 1 < nbp) {
        col_partials(Pn, kk + 1, k + 1, nbp, nw);
        g_arrive(nw);
      }
    }
    gsync(nw);
    return true;
  };

  // C -= V W' for column group g (of 32 from jt0) on rows [ia, ib) of own rows
  auto update_rows = [&](const double* Ps, int jt0, int g, int ia, int ib) {
    const int j = jt0 + 32 * g + lane;
    if (j >= ncols || ia >= ib) return;
    double wv[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) wv[q] = __ldcg(a.Wp + (size_t)q * ncols + j);
    double* cp = B + (int64_t)j * ldb + r0;
    for (int i = ia; i < ib; ++i) {
      double c = cp[i];
#pragma unroll
      for (int q = 0; q < kNB; ++q) c -= Ps[q * ldp + i] * wv[q];
      cp[i] = c;
    }
  };

  if (!factor_panel(pbuf0, 0, min(kNB, n), 8)) return;
  int cur = 0;
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int nbp = min(kNB, n - k0);
    double* Ps = cur ? pbuf1 : pbuf0;

    // ---------------------------------------------------- write back, form V
    for (int e = threadIdx.x; e < nbp * nrow; e += blockDim.x) {
      const int c = e / nrow, i = e - c * nrow;
      const int64_t g = r0 + i;
      const double v = Ps[c * ldp + i];
      B[g + (int64_t)(k0 + c) * ldb] = (g == k0 + c) ? s_beta[c] : v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNB * nrow; e += blockDim.x) {
      const int c = e / nrow, i = e - c * nrow;
      const int64_t g = r0 + i;
      if (c >= nbp || g < k0 + c) Ps[c * ldp + i] = 0.0;
      else if (g == k0 + c) Ps[c * ldp + i] = 1.0;
    }
    __syncthreads();

    // ---------------------------------------------------- partial G and W = V^T C (as k_householder_blocked)
    const int i0 = (int)max((int64_t)0, (int64_t)k0 - r0);
    for (int ls = 2 * warp; ls < 2 * warp + 2; ++ls) {
      const int e = 32 * ls + lane;
      if (e < kNB * (kNB - 1) / 2) {
        int c = 1;
        while ((c + 1) * c / 2 <= e) ++c;
        const int r = e - c * (c - 1) / 2;
        double g = 0.0;
        if (c < nbp)
          for (int i = i0; i < nrow; ++i) g += Ps[r * ldp + i] * Ps[c * ldp + i];
        __stcg(pG + (size_t)p * kNB * kNB + e, g);
      }
    }
    const int jt0 = k0 + nbp;
    const int ngroups = (ncols - jt0 + 31) / 32;
    {
      const int h = warp & 3;
      for (int g = warp >> 2; g < ngroups; g += 2) {
        const int j = jt0 + 32 * g + lane;
        if (j < ncols) {
          double acc[kNB / 4];
#pragma unroll
          for (int q = 0; q < kNB / 4; ++q) acc[q] = 0.0;
          const double* cp = B + (int64_t)j * ldb + r0;
          const double* vp = Ps + (size_t)(h * (kNB / 4)) * ldp;
#pragma unroll 2
          for (int i = i0; i < nrow; ++i) {
            const double c = cp[i];
#pragma unroll
            for (int q = 0; q < kNB / 4; ++q) acc[q] += vp[q * ldp + i] * c;
          }
          double* out = pW + ((size_t)p * kNB + h * (kNB / 4)) * ncols + j;
#pragma unroll
          for (int q = 0; q < kNB / 4; ++q) __stcg(out + (size_t)q * ncols, acc[q]);
        }
      }
    }
    if (!mono_sync(mb, P)) return;
    for (int e = p + warp * P; e < kNB * (kNB - 1) / 2; e += 8 * P) {
      double g = 0.0;
      for (int q = lane; q < P; q += 32) g += __ldcg(pG + (size_t)q * kNB * kNB + e);
      g = warp_sum(g);
      if (lane == 0) __stcg(Gred + e, g);
    }
    if (!mono_sync(mb, P)) return;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e / kNB, q = e - r * kNB;
      double mv = 0.0;
      if (r < q && q < nbp) mv = __ldcg(Gred + q * (q - 1) / 2 + r) * s_tau[r];
      Gs[e] = mv;
    }
    __syncthreads();
    {
      const double tq = (lane < nbp) ? s_tau[lane] : 0.0;
      for (int j = jt0 + p * 8 + warp; j < ncols; j += P * 8) {
        double w = 0.0;
        for (int q = 0; q < P; ++q) w += __ldcg(pW + ((size_t)q * kNB + lane) * ncols + j);
        for (int r = 0; r + 1 < nbp; ++r) {
          const double t = __shfl_sync(0xffffffffu, w, r);
          if (lane > r) w = w - Gs[r * kNB + lane] * t;
        }
        __stcg(a.Wp + (size_t)lane * ncols + j, w * tq);
      }
    }
    if (!mono_sync(mb, P)) return;

    // ---------------------------------------------------- lookahead: panel p+1's columns first
    const int len = nrow - i0;
    if (ngroups > 0) update_rows(Ps, jt0, 0, i0 + (len * warp) / 8, i0 + (len * (warp + 1)) / 8);
    if (threadIdx.x == 0) s_task = 0;
    __syncthreads();
    const int k1 = k0 + kNB;
    const int nbp1 = (k1 < n) ? min(kNB, n - k1) : 0;
    // warps on the next panel: few while the update is long, all of them
    // (no overlap) once it is short (thresholds measured at d = 20,000,
    // n = 1000 with one grid barrier per panel column)
    const int grest = ngroups - 1;
    const int nw1 = (grest >= 12) ? 2 : (grest >= 5) ? 4 : 8;
    if (nbp1 > 0 && nw1 < 8 && warp < nw1) {
      if (!factor_panel(cur ? pbuf0 : pbuf1, k1, nbp1, nw1) && threadIdx.x == 0) s_abort = 1;
    }
    // ---------------------------------------------------- the rest of C -= V W' (groups 1 ..)
    const int ntask = (ngroups - 1) * kLaTasksPerGroup;
    for (;;) {
      int t = 0;
      if (lane == 0) t = atomicAdd(&s_task, 1);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= ntask) break;
      const int g = 1 + t / kLaTasksPerGroup, c = t % kLaTasksPerGroup;
      update_rows(Ps, jt0, g, i0 + (len * c) / kLaTasksPerGroup, i0 + (len * (c + 1)) / kLaTasksPerGroup);
    }
    __syncthreads();
    if (s_abort) return;
    if (nbp1 > 0 && nw1 == 8 && !factor_panel(cur ? pbuf0 : pbuf1, k1, nbp1, 8)) return;
    if (nbp1 > 0 && nw1 < 8 && warp >= nw1) mb.epoch += (unsigned int)nbp1;   // the panel's grid barriers
    cur ^= 1;
  }
}

// ------------------------------------------------------------ prepare R
// src: upper triangle of a column-major matrix (lds).  Writes R_out (if not
// null, ldr), Rt[a + b*n] = R[b, a], inv_diag[i] = 1 / R[i, i].
__global__ void k_prepare_R(const double* __restrict__ src, int64_t lds, int n, double* __restrict__ R_out,
                            int64_t ldr, double* __restrict__ Rt, double* __restrict__ inv_diag,
                            unsigned int* __restrict__ status) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    const double r = (i <= j) ? src[i + (int64_t)j * lds] : 0.0;
    if (R_out) R_out[i + (int64_t)j * ldr] = r;
    Rt[(size_t)j + (size_t)i * n] = r;
    if (i == j) {
      inv_diag[i] = 1.0 / r;
      if (r == 0.0 || !isfinite(r)) atomicOr(status, LS_DEV_RANK);
    }
  }
}

cudaError_t launch_prepare_R(ls_ctx* ctx, const double* src, int64_t lds, int64_t n, double* R_out, int64_t ldr,
                             double* Rt, double* inv_diag) {
  const int64_t total = n * n;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
  k_prepare_R<<<grid, 256, 0, ctx->stream>>>(src, lds, (int)n, R_out, ldr, Rt, inv_diag, ctx->d_status);
  ++ctx->launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------ post factor
struct PostArgs {
  const double* B; int64_t ldb; int n;
  const double* R; int64_t ldr;
  const double* Rt; const double* inv_diag;
  double* x0; uint64_t seed;
  double* v; double* w; double* xi; double* work;   // n-vectors
  double* slots;                                     // 2 * ncta
  double* est;                                       // [normest, condest]
  unsigned int* status;
};

template <int PP>
__global__ void __launch_bounds__(256) k_post_factor(PostArgs a) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  TsSmem& sm = *reinterpret_cast<TsSmem*>(ts_raw);
  const CL cl = cl_this();
  const int n = a.n;
  const int nb = (n + 31) / 32;
  ts_setup(cl, sm, a.R, a.ldr, a.inv_diag, n);
  cl_sync();
  const uint64_t deadline = gtimer() + 2000000000ull;
  int tmo = 0;
  uint32_t uses[2] = {0u, 0u};
  // out = R^{-1} rhs (back) or R^{-T} rhs, both n-vectors in global memory;
  // out is complete and visible cluster-wide on return
  auto solve = [&](bool back, const double* rhs_g, double* out_g) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, q = w >> 1, h = w & 1;
    const int mine = ts_owned(cl, nb);
    double rhs[PP], out[PP];
#pragma unroll
    for (int s = 0; s < PP; ++s) {
      const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
      rhs[s] = (h == 0 && o < mine && i < n) ? __ldcg(rhs_g + i) : 0.0;
    }
    const int sidx = back ? 1 : 0;
    const uint32_t par = uses[sidx] & 1u;
    if (back) ts_solve<PP, true>(cl, sm, 1, a.R, a.ldr, a.inv_diag, n, rhs, out, deadline, tmo, par);
    else ts_solve<PP, false>(cl, sm, 0, a.Rt, n, a.inv_diag, n, rhs, out, deadline, tmo, par);
#pragma unroll
    for (int s = 0; s < PP; ++s) {
      const int o = q + 4 * s, i = 32 * ((int)cl.rank + o * (int)cl.ncta) + l;
      if (h == 0 && o < mine && i < n) __stcg(out_g + i, out[s]);
    }
    ts_finish(sm, n, sidx, par, deadline, tmo);
    uses[sidx] += 1u;
    cl_sync();
  };

  // ---- x0 = R^{-1} z, z = (Q^T S b)[0:n] = column n of the factored B
  solve(true, a.B + (int64_t)n * a.ldb, a.x0);

  // ---- normest: power method on R^T R from a Philox start vector
  for_owned_rows(cl, n, [&](int i) { __stcg(a.v + i, power_start(a.seed, 1u, i)); });
  cl_sync();
  double nv = cl_norm2(cl, n, a.v, a.slots);
  for_owned_rows(cl, n, [&](int i) { __stcg(a.v + i, __ldcg(a.v + i) / nv); });
  cl_sync();
  const int steps = power_steps(n);
  for (int st = 0; st < steps; ++st) {
    cl_matvec_R(cl, a.Rt, n, a.v, a.w);
    cl_sync();
    cl_matvec_RT(cl, a.R, a.ldr, n, a.w, a.v);
    cl_sync();
    nv = cl_norm2(cl, n, a.v, a.slots);
    for_owned_rows(cl, n, [&](int i) { __stcg(a.v + i, __ldcg(a.v + i) / nv); });
    cl_sync();
  }
  cl_matvec_R(cl, a.Rt, n, a.v, a.w);
  cl_sync();
  const double normest = cl_norm2(cl, n, a.w, a.slots);

  // ---- condest = ||R||_1 * Hager estimate of ||R^{-1}||_1
  double colmax = 0.0;
  for (int b = cl.rank; b < nb; b += cl.ncta)
    for (int j = 32 * b + (int)threadIdx.x; j < min(n, 32 * b + 32); j += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i <= j; ++i) s += fabs(__ldg(a.R + i + (int64_t)j * a.ldr));
      colmax = fmax(colmax, s);
    }
  const double norm1 = cl_max(cl, cta_max(colmax), a.slots);

  double* x = a.v;   // reuse
  double* y = a.w;
  for_owned_rows(cl, n, [&](int i) { __stcg(a.work + i, 1.0 / (double)n); });
  cl_sync();
  solve(true, a.work, y);                                    // y = R^{-1} x
  double est;
  if (n == 1) {
    est = fabs(__ldcg(y));
  } else {
    est = cl_norm1(cl, n, y, a.slots);
    for_owned_rows(cl, n, [&](int i) { __stcg(a.xi + i, sgn1(__ldcg(y + i))); });
    cl_sync();
    solve(false, a.xi, x);                                   // x = R^{-T} xi
    int j = cl_argmax_abs(cl, n, x, a.slots);
    int iter = 2;
    for (;;) {
      for_owned_rows(cl, n, [&](int i) { __stcg(a.work + i, i == j ? 1.0 : 0.0); });
      cl_sync();
      solve(true, a.work, y);                                // y = R^{-1} e_j
      const double est_old = est;
      est = cl_norm1(cl, n, y, a.slots);
      double diff = 0.0;
      for_owned_rows(cl, n, [&](int i) { if (sgn1(__ldcg(y + i)) != __ldcg(a.xi + i)) diff = 1.0; });
      const double any_diff = cl_max(cl, cta_max(diff), a.slots);
      if (any_diff == 0.0 || est <= est_old) break;
      for_owned_rows(cl, n, [&](int i) { __stcg(a.xi + i, sgn1(__ldcg(y + i))); });
      cl_sync();
      solve(false, a.xi, x);                                 // x = R^{-T} xi
      const int jlast = j;
      j = cl_argmax_abs(cl, n, x, a.slots);
      if (__ldcg(x + jlast) != fabs(__ldcg(x + j)) && iter < 5) { iter += 1; continue; }
      break;
    }
    for_owned_rows(cl, n, [&](int i) {
      const double v = 1.0 + (double)i / (double)(n - 1);
      __stcg(a.work + i, (i % 2 == 0) ? v : -v);
    });
    cl_sync();
    solve(true, a.work, y);
    double alt = cl_norm1(cl, n, y, a.slots);
    alt = 2.0 * alt / (3.0 * (double)n);
    if (alt > est) est = alt;
  }
  if (tmo) atomicOr(a.status, LS_DEV_TIMEOUT);
  if (cl.rank == 0 && threadIdx.x == 0) {
    a.est[0] = normest;
    a.est[1] = norm1 * est;
  }
}

// ------------------------------------------------------------ host side
int householder_ctas(const ls_ctx* ctx, int64_t d) {
  int64_t p = (d + 63) / 64;
  if (p > ctx->num_sms) p = ctx->num_sms;
  if (p < 1) p = 1;
  return (int)p;
}

static constexpr int64_t kBlockedMaxChunk = 600;   // panel slice rows per CTA in shared memory
static constexpr int64_t kLaMaxChunk = 436;        // two panel buffers + W' multipliers in 227 KB

static size_t la_smem(int64_t ch) {
  const int64_t ldp = ch + 1 + (ch & 1);
  return (size_t)(2 * kNB * ldp + kNB * kNB) * sizeof(double);
}

static size_t blocked_smem(int64_t ch) {
  const int64_t ldp = ch + 1 + (ch & 1);
  return (size_t)(kNB * ldp + 2 * kNB * kNB) * sizeof(double);
}

cudaError_t launch_householder(ls_ctx* ctx, double* B, int64_t d, int64_t n, int64_t ldb, double* part,
                               double* w) {
  const int P = householder_ctas(ctx, d);
  const int64_t chunk = (d + P - 1) / P;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->d_status + 1, 0, 2 * sizeof(unsigned int), ctx->stream)) != cudaSuccess) return e;
  GridBar gb{ctx->d_status + 1, ctx->d_status + 2, ctx->d_status};
  if (chunk <= kLaMaxChunk && n >= 2) {
    const size_t smem = la_smem(chunk);
    if ((e = cudaFuncSetAttribute(k_householder_la, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    HhArgs ha{B, d, (int)n, ldb, part, w, gb};
    void* args[] = {&ha};
    ++ctx->launches;
    return cudaLaunchCooperativeKernel((const void*)k_householder_la, dim3(P), dim3(256), args, smem, ctx->stream);
  }
  if (chunk <= kBlockedMaxChunk && n >= 2) {
    const size_t smem = blocked_smem(chunk);
    if ((e = cudaFuncSetAttribute(k_householder_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    HhArgs ha{B, d, (int)n, ldb, part, w, gb};
    void* args[] = {&ha};
    ++ctx->launches;
    return cudaLaunchCooperativeKernel((const void*)k_householder_blocked, dim3(P), dim3(256), args, smem,
                                       ctx->stream);
  }
  const size_t smem = (size_t)chunk * sizeof(double);
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_householder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
  }
  int nn = (int)n;
  void* args[] = {&B, &d, &nn, &ldb, &part, &w, &gb};
  ++ctx->launches;
  return cudaLaunchCooperativeKernel((const void*)k_householder, dim3(P), dim3(256), args, smem, ctx->stream);
}

size_t householder_part_doubles(const ls_ctx* ctx, int64_t d, int64_t n) {
  const size_t P = (size_t)householder_ctas(ctx, d);
  const size_t unblocked = P * (size_t)(n + 2) + 1;
  const size_t blocked = P + 8 + P * kNB + P * kNB * (size_t)(n + 1) + P * kNB * kNB + 2 * kNB + P * kNB;
  return std::max(unblocked, blocked);
}

size_t householder_w_doubles(int64_t n) { return (size_t)kNB * (size_t)(n + 1) + 8 + kNB * kNB; }

cudaError_t launch_post_factor(ls_ctx* ctx, const double* B, int64_t d, int64_t n, int64_t ldb, const double* R,
                               int64_t ldr, double* x0, uint64_t seed, const double* Rt, const double* inv_diag,
                               double* vecs /* 4n + 64 */, double* est_out) {
  (void)d;
  static int P = -1;
  if (P < 0) {
    const void* fns[] = {(const void*)k_post_factor<1>, (const void*)k_post_factor<2>};
    P = ts_cluster_size_of(fns, 2);
  }
  const int pp = ts_slots((int)n, P);
  if (pp == 0 || n > kTsMaxN) return cudaErrorInvalidValue;
  PostArgs a;
  a.B = B; a.ldb = ldb; a.n = (int)n; a.R = R; a.ldr = ldr; a.Rt = Rt; a.inv_diag = inv_diag;
  a.x0 = x0; a.seed = seed;
  a.v = vecs; a.w = vecs + n; a.xi = vecs + 2 * n; a.work = vecs + 3 * n; a.slots = vecs + 4 * n;
  a.est = est_out; a.status = ctx->d_status;
  void* args[] = {&a};
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
  return cudaLaunchKernelExC(&cfg, pp == 1 ? (const void*)k_post_factor<1> : (const void*)k_post_factor<2>, args);
}

}  // namespace lsk
