// batched.cu -- many independent least-squares problems of different shapes
// solved together (Algorithm 2 with the Sec. 3.3 stopping rule per problem),
// one launch per phase for the whole batch.
//
//  * sketch: k_b_sparse_sign writes every column's zeta rows as global bucket
//    ids (problem offset + row), so the single-problem counting sort
//    (k_hist, k_scan, k_scatter, k_bucket_sort) runs unchanged over the
//    concatenated buckets; k_b_gather (one warp per bucket) forms B_p column
//    by column with the same left-to-right sums as the single-problem path,
//    so every B_p is bit-identical to ls_sketch of that problem.
//  * factor: one CTA per problem (k_b_householder: unblocked LAPACK-convention
//    Householder on B_p in L2), then k_prepare_R-like and post-factor work
//    per problem on 1-CTA clusters with the cluster_la.cuh routines.
//  * iterate: k_b_pass walks the (problem, row tile) items of all active
//    problems in a persistent grid (tile staged in shared memory, row dots by
//    warps, A^T r by column threads, one partial per item); k_b_step (one
//    CTA per problem) sums a problem's partials in item order, applies the
//    stopping rule and does the two substitutions and the update.
#include <algorithm>

#include "cluster_la.cuh"

namespace lsk {

struct BProb {
  const double* A; const double* b; double* x;
  int64_t m, n, lda, d;
  uint64_t seed;
  int64_t moff;      // sum of m over earlier problems (flattened columns of S)
  int64_t doff;      // sum of d (buckets)
  int64_t boff;      // sum of d (n + 1) (B pool)
  int64_t roff;      // sum of n^2 (R, Rt pools)
  int64_t voff;      // sum of n (vector pools)
  int64_t toff;      // sum of row tiles (pass items)
  int64_t poff;      // sum of tiles (n + 2) (partials)
  int tr;            // rows per tile
  int tiles;
};

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

// One warp per global bucket: B_p[t, c] = s * (left-to-right sum of +-A_p[j, c]).
__global__ void __launch_bounds__(256) k_b_gather(const BProb* __restrict__ P, const int64_t* __restrict__ doffs,
                                                  int np, int64_t dtotal, const int64_t* __restrict__ row_ptr,
                                                  const uint32_t* __restrict__ ent, double scale,
                                                  double* __restrict__ Bpool) {
  const int64_t tg = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tg >= dtotal) return;
  const int p = find_problem(doffs, np, tg);
  const BProb pr = P[p];
  const int64_t t = tg - pr.doff;
  const int64_t e0 = row_ptr[tg], e1 = row_ptr[tg + 1];
  double* B = Bpool + pr.boff;
  for (int64_t c0 = 0; c0 <= pr.n; c0 += 64) {
    const int64_t c = c0 + 2 * lane;
    // this lane's columns: c, c+1 of [A b] (c == n is b)
    const bool has0 = c <= pr.n, has1 = c + 1 <= pr.n;
    double a0 = 0.0, a1 = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t en = __ldg(ent + e);
      const int64_t j = (int64_t)(en >> 1) - pr.moff;
      double v0 = 0.0, v1 = 0.0;
      if (c + 1 < pr.n) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(pr.A + j * pr.lda + c));
        v0 = v.x; v1 = v.y;
      } else {
        if (has0) v0 = (c < pr.n) ? __ldg(pr.A + j * pr.lda + c) : __ldg(pr.b + j);
        if (has1) v1 = (c + 1 < pr.n) ? __ldg(pr.A + j * pr.lda + c + 1) : __ldg(pr.b + j);
      }
      if (en & 1u) { a0 = a0 - v0; a1 = a1 - v1; }
      else { a0 = a0 + v0; a1 = a1 + v1; }
    }
    if (has0) B[t + c * pr.d] = scale * a0;
    if (has1) B[t + (c + 1) * pr.d] = scale * a1;
  }
}

// ---------------------------------------------------------------- factor
// One CTA per problem: unblocked Householder QR of B_p (d x (n+1)), reflectors
// for the first n columns applied to all later columns.
__global__ void __launch_bounds__(256) k_b_householder(const BProb* __restrict__ P, double* __restrict__ Bpool,
                                                       unsigned int* __restrict__ pstatus) {
  const BProb pr = P[blockIdx.x];
  const int64_t d = pr.d;
  const int n = (int)pr.n;
  double* B = Bpool + pr.boff;
  __shared__ double s_par[3];
  __shared__ int s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    double* col = B + k + (int64_t)k * d;
    const int64_t len = d - k;
    double ss = 0.0;
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) ss += col[i] * col[i];
    ss = cta_sum(ss);
    if (threadIdx.x == 0) {
      const double alpha = col[0];
      const double xnorm = sqrt(ss);
      double beta, tau, scal;
      if (xnorm == 0.0) { beta = alpha; tau = 0.0; scal = 1.0; }
      else {
        const double h = hypot(alpha, xnorm);
        beta = (alpha >= 0.0) ? -h : h;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      s_par[0] = beta; s_par[1] = tau; s_par[2] = scal;
      s_bad = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
    }
    __syncthreads();
    if (s_bad) {
      if (threadIdx.x == 0) pstatus[blockIdx.x] |= LS_DEV_RANK;
      return;
    }
    const double tau = s_par[1], scal = s_par[2];
    if (tau != 0.0)
      for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) col[i] *= scal;
    __syncthreads();
    if (threadIdx.x == 0) col[0] = s_par[0];
    if (tau != 0.0) {
      for (int j = k + 1 + warp; j <= n; j += nw) {
        double* cj = B + k + (int64_t)j * d;
        double w = 0.0;
        for (int64_t i = lane; i < len; i += 32) w += ((i == 0) ? 1.0 : col[i]) * cj[i];
        w = warp_sum(w);
        const double tw = tau * w;
        for (int64_t i = lane; i < len; i += 32) cj[i] = cj[i] - tw * ((i == 0) ? 1.0 : col[i]);
      }
    }
    __syncthreads();
  }
}

// R_p, Rt_p, 1/diag(R_p) for every problem (grid-stride over all entries of all problems).
__global__ void k_b_prepare_R(const BProb* __restrict__ P, int np, const double* __restrict__ Bpool,
                              double* __restrict__ Rpool, double* __restrict__ Rtpool, double* __restrict__ invd,
                              unsigned int* __restrict__ pstatus) {
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const BProb pr = P[p];
    const int n = (int)pr.n;
    const double* B = Bpool + pr.boff;
    double* R = Rpool + pr.roff;
    double* Rt = Rtpool + pr.roff;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int j = e / n, i = e - j * n;
      const double r = (i <= j) ? B[i + (int64_t)j * pr.d] : 0.0;
      R[i + (int64_t)j * n] = r;
      Rt[j + (int64_t)i * n] = r;
      if (i == j) {
        invd[pr.voff + i] = 1.0 / r;
        if (r == 0.0 || !isfinite(r)) atomicOr(&pstatus[p], LS_DEV_RANK);
      }
    }
  }
}

// One 1-CTA cluster per problem: x0 = R^{-1} z, normest, condest (the same
// steps as the single-problem post-factor kernel).
__global__ void __launch_bounds__(256) k_b_post_factor(const BProb* __restrict__ P, BPools pl) {
  const int p = blockIdx.x;
  if (pl.pstatus[p] & LS_DEV_RANK) return;
  const BProb pr = P[p];
  const CL cl{0u, 1u};
  const int n = (int)pr.n;
  const double* B = pl.B + pr.boff;
  const double* R = pl.R + pr.roff;
  const double* Rt = pl.Rt + pr.roff;
  const double* invd = pl.inv_diag + pr.voff;
  double* work = pl.work + pr.voff;
  double* v = pl.v + pr.voff;
  double* w = pl.w + pr.voff;
  double* xi = pl.xi + pr.voff;
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
__global__ void k_b_iter_init(const BProb* __restrict__ P, int np, BPools pl, double gamma, double rho, double alpha,
                              double beta) {
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const BProb pr = P[p];
    for (int i = threadIdx.x; i < pr.n; i += blockDim.x) pl.x_prev[pr.voff + i] = pr.x[i];
    if (threadIdx.x == 0) {
      IterState s{};
      s.gamma = gamma; s.rho = rho; s.alpha = alpha; s.beta = beta;
      s.normest = pl.est[2 * p];
      s.condest = pl.est[2 * p + 1];
      if (pl.pstatus[p] & LS_DEV_RANK) { s.done = 1; s.stop_reason = 4; }
      pl.st[p] = s;
    }
  }
}

static constexpr int kBThreads = 256;

// Persistent pass over all (problem, tile) items of active problems.
__global__ void __launch_bounds__(kBThreads) k_b_pass(const BProb* __restrict__ P, const int64_t* __restrict__ toffs,
                                                      int np, int64_t items, BPools pl) {
  extern __shared__ double sb[];
  __shared__ double rt[256];
  __shared__ double red[2 * 8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int p = find_problem(toffs, np, it);
    if (pl.st[p].done) continue;                       // uniform in the CTA
    const BProb pr = P[p];
    const int n = (int)pr.n, tr = pr.tr;
    const int tile = (int)(it - pr.toff);
    const int64_t row0 = (int64_t)tile * tr;
    const int rows = (int)min((int64_t)tr, pr.m - row0);
    double* xs = sb;                                   // n
    double* ts = sb + ((n + 1) & ~1);                  // rows x n
    for (int i = threadIdx.x; i < n; i += kBThreads) xs[i] = pr.x[i];
    for (int e = threadIdx.x; e < rows * n; e += kBThreads) {
      const int r = e / n, c = e - r * n;
      ts[e] = __ldg(pr.A + (row0 + r) * pr.lda + c);
    }
    __syncthreads();
    // phase 1: r_j = b_j - A_j x (warp per row)
    double rn2 = 0.0, dn2 = 0.0;
    for (int r = warp; r < rows; r += kBThreads / 32) {
      double dot = 0.0;
      for (int c = lane; c < n; c += 32) dot += ts[r * n + c] * xs[c];
      dot = warp_sum(dot);
      if (lane == 0) {
        const int64_t j = row0 + r;
        const double rj = __ldg(pr.b + j) - dot;
        double* rp = pl.r_prev + pr.moff + j;
        const double dl = rj - *rp;
        *rp = rj;
        rn2 += rj * rj;
        dn2 += dl * dl;
        rt[r] = rj;
      }
    }
    if (lane == 0) { red[warp] = rn2; red[8 + warp] = dn2; }
    __syncthreads();
    // phase 2: c_k = sum_r A_rk r_r over the tile (column threads, row groups)
    double* out = pl.part + pr.poff + (int64_t)tile * (n + 2);
    if (n >= kBThreads) {
      for (int c = threadIdx.x; c < n; c += kBThreads) {
        double s = 0.0;
        for (int r = 0; r < rows; ++r) s += ts[r * n + c] * rt[r];
        out[c] = s;
      }
    } else {
      const int G = kBThreads / n;
      const int g = threadIdx.x / n, c = threadIdx.x - g * n;
      double s = 0.0;
      if (g < G)
        for (int r = g; r < rows; r += G) s += ts[r * n + c] * rt[r];
      __syncthreads();
      double* gs = ts;                                  // tile no longer needed
      if (g < G) gs[g * n + c] = s;
      __syncthreads();
      for (int cc = threadIdx.x; cc < n; cc += kBThreads) {
        double t = 0.0;
        for (int q = 0; q < G; ++q) t += gs[q * n + cc];
        out[cc] = t;
      }
    }
    if (threadIdx.x == 0) {
      double s1 = 0.0, s2 = 0.0;
      for (int w = 0; w < kBThreads / 32; ++w) { s1 += red[w]; s2 += red[8 + w]; }
      out[n] = s1;
      out[n + 1] = s2;
    }
    __syncthreads();
  }
}

// One 1-CTA cluster per problem: sum partials (item order), stopping rule,
// two substitutions, update.
__global__ void __launch_bounds__(256) k_b_step(const BProb* __restrict__ P, BPools pl, int use_stop, int extra,
                                                unsigned int* __restrict__ active) {
  const int p = blockIdx.x;
  IterState S = pl.st[p];
  if (S.done) return;
  const BProb pr = P[p];
  const CL cl{0u, 1u};
  const int n = (int)pr.n;
  const double* part = pl.part + pr.poff;
  __shared__ double s_norm[2];
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int t = 0; t < pr.tiles; ++t) s += part[(int64_t)t * (n + 2) + n + threadIdx.x];
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
      pl.st[p].done = 1; pl.st[p].fired = 1; pl.st[p].stop_reason = 0;
      pl.st[p].rnorm = rnorm; pl.st[p].dnorm = dnorm;
    }
    return;
  }
  double* work = pl.work + pr.voff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < pr.tiles; ++t) s += part[(int64_t)t * (n + 2) + i];
    __stcg(work + i, s);
  }
  __syncthreads();
  const double* invd = pl.inv_diag + pr.voff;
  double* y = pl.y + pr.voff;
  double* dv = pl.dvec + pr.voff;
  cl_solve_RT(cl, pl.Rt + pr.roff, n, invd, work, y);
  cl_load_owned(cl, n, y, work);
  cl_solve_R(cl, pl.R + pr.roff, n, n, invd, work, dv);
  double xs = 0.0, bad = 0.0;
  double* xp = pl.x_prev + pr.voff;
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
    if (bad != 0.0) { st.nonfinite = 1; st.done = 1; st.stop_reason = 3; }
    if (!st.done) atomicAdd(active, 1u);
  }
}

// ---------------------------------------------------------------- host side

static int tile_rows(int64_t n) {
  int64_t tr = 8192 / std::max<int64_t>(n, 1);
  tr = std::max<int64_t>(8, std::min<int64_t>(256, tr));
  return (int)tr;
}

void batch_plan(const ls_problem* probs, int np, BProb* out, BatchPlan& pl) {
  pl.np = np;
  pl.mtotal = pl.dtotal = pl.btotal = pl.rtotal = pl.vtotal = pl.ttotal = pl.ptotal = 0;
  pl.max_n = 0;
  pl.max_tile_doubles = 0;
  for (int p = 0; p < np; ++p) {
    const ls_problem& q = probs[p];
    BProb b{};
    b.A = q.A; b.b = q.b; b.x = q.x; b.m = q.m; b.n = q.n; b.lda = q.lda; b.d = q.d; b.seed = q.seed;
    b.moff = pl.mtotal; b.doff = pl.dtotal; b.boff = pl.btotal; b.roff = pl.rtotal; b.voff = pl.vtotal;
    b.toff = pl.ttotal; b.poff = pl.ptotal;
    b.tr = tile_rows(q.n);
    b.tiles = (int)((q.m + b.tr - 1) / b.tr);
    pl.mtotal += q.m; pl.dtotal += q.d; pl.btotal += q.d * (q.n + 1); pl.rtotal += q.n * q.n;
    pl.vtotal += q.n; pl.ttotal += b.tiles; pl.ptotal += (int64_t)b.tiles * (q.n + 2);
    pl.max_n = std::max<int>(pl.max_n, (int)q.n);
    pl.max_tile_doubles = std::max<int>(pl.max_tile_doubles, (int)(((q.n + 1) & ~1LL) + (int64_t)b.tr * q.n));
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

cudaError_t launch_b_gather(ls_ctx* ctx, const BProb* dP, const int64_t* ddoffs, const BatchPlan& pl,
                            const int64_t* row_ptr, const uint32_t* ent, double scale, double* Bpool) {
  k_b_gather<<<(unsigned)((pl.dtotal + 7) / 8), 256, 0, ctx->stream>>>(dP, ddoffs, pl.np, pl.dtotal, row_ptr, ent,
                                                                       scale, Bpool);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_factor(ls_ctx* ctx, const BProb* dP, const BatchPlan& pl, const BPools& pools) {
  k_b_householder<<<pl.np, 256, 0, ctx->stream>>>(dP, pools.B, pools.pstatus);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_b_prepare_R<<<std::min(pl.np, ctx->num_sms * 8), 256, 0, ctx->stream>>>(dP, pl.np, pools.B, pools.R, pools.Rt,
                                                                          pools.inv_diag, pools.pstatus);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BPools pp = pools;
  const BProb* dPP = dP;
  void* args[] = {(void*)&dPP, &pp};
  return launch_cluster_grid(ctx, (const void*)k_b_post_factor, args, pl.np);
}

cudaError_t launch_b_iter_init(ls_ctx* ctx, const BProb* dP, const BatchPlan& pl, const BPools& pools, double gamma,
                               double rho, double alpha, double beta) {
  k_b_iter_init<<<std::min(pl.np, ctx->num_sms * 8), 128, 0, ctx->stream>>>(dP, pl.np, pools, gamma, rho, alpha, beta);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_pass(ls_ctx* ctx, const BProb* dP, const int64_t* dtoffs, const BatchPlan& pl,
                          const BPools& pools) {
  const size_t smem = (size_t)pl.max_tile_doubles * sizeof(double);
  cudaError_t e;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_b_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pass, kBThreads, smem);
  const int64_t grid = std::min<int64_t>(pl.ttotal, (int64_t)ctx->num_sms * std::max(1, per_sm));
  k_b_pass<<<(unsigned)grid, kBThreads, smem, ctx->stream>>>(dP, dtoffs, pl.np, pl.ttotal, pools);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_b_step(ls_ctx* ctx, const BProb* dP, const BatchPlan& pl, const BPools& pools, int use_stop,
                          int extra, unsigned int* active) {
  BPools pp = pools;
  const BProb* dPP = dP;
  int us = use_stop, ex = extra;
  void* args[] = {(void*)&dPP, &pp, &us, &ex, &active};
  return launch_cluster_grid(ctx, (const void*)k_b_step, args, pl.np);
}

}  // namespace lsk
