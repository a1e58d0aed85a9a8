// sparse.cu -- Algorithm 2 for a sparse A given in CSR (the sparse workload of
// Sec. 3.5: a few nonzeros per row in random columns).  The sketch and the
// QR of the sketch are the dense method's; what changes is how A is read:
//
//  * k_sp_gather: B = s S [A b] with one warp per sketch row t.  The warp
//    walks the bucket's columns of S in ascending j and adds +-A[j, :] into a
//    shared-memory row accumulator (a row's nonzeros sit in distinct columns,
//    so its lanes never collide), then scales once.  Every entry of B is
//    therefore the dense left-to-right sum with its zero terms left out --
//    bit-identical to the dense sketch of the same matrix.
//  * CSC copy of A for A^T r, built deterministically: per block of rows a
//    column histogram, column starts and per-block offsets by prefix sums,
//    then each block scatters its rows in row order (a stable counting sort
//    by column), so every column lists its rows ascending.
//  * the pass: k_sp_residual forms r = b - A x row by row, keeps r in r_prev
//    and writes per-CTA partials of ||r||^2 and ||r - r_prev||^2;
//    k_sp_gradient forms A^T r column by column from the CSC copy (one warp
//    per column segment); k_sp_reduce sums both in fixed order into the
//    (n + 2)-vector that the dense path's step kernel consumes.
#include <algorithm>

#include "ls_internal.cuh"

namespace lsk {

static constexpr int kSpWarps = 8;
static constexpr int kSpBlockRows = 1024;   // rows per block of the CSC build

// ---------------------------------------------------------------- sketch
__global__ void __launch_bounds__(kSpWarps * 32) k_sp_gather(int64_t d, const int64_t* __restrict__ srow,
                                                             const uint32_t* __restrict__ sent,
                                                             const int64_t* __restrict__ arp,
                                                             const int32_t* __restrict__ acol,
                                                             const double* __restrict__ aval,
                                                             const double* __restrict__ b, int n, double scale,
                                                             double* __restrict__ B, int64_t ldb) {
  extern __shared__ double sp_acc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kSpWarps + warp;
  if (t >= d) return;
  double* acc = sp_acc + (size_t)warp * (n + 1);
  for (int c = lane; c <= n; c += 32) acc[c] = 0.0;
  __syncwarp();
  const int64_t e0 = srow[t], e1 = srow[t + 1];
  for (int64_t eb = e0; eb < e1; eb += 32) {
    // metadata of up to 32 entries at once, one per lane
    const int cnt = (int)min((int64_t)32, e1 - eb);
    uint32_t my = 0;
    int64_t mr0 = 0, mr1 = 0;
    if (lane < cnt) {
      my = __ldg(sent + eb + lane);
      const int64_t j = my >> 1;
      mr0 = __ldg(arp + j);
      mr1 = __ldg(arp + j + 1);
    }
    for (int i = 0; i < cnt; ++i) {
      const uint32_t en = __shfl_sync(0xffffffffu, my, i);
      const int64_t r0 = __shfl_sync(0xffffffffu, mr0, i), r1 = __shfl_sync(0xffffffffu, mr1, i);
      for (int64_t k = r0 + lane; k < r1; k += 32) {
        const int c = __ldg(acol + k);
        acc[c] = acc[c] + signed_by(__ldg(aval + k), en);
      }
      if (lane == 0) acc[n] = acc[n] + signed_by(__ldg(b + (en >> 1)), en);
      __syncwarp();
    }
  }
  for (int c = lane; c <= n; c += 32) B[t + (int64_t)c * ldb] = scale * acc[c];
}

// ---------------------------------------------------------------- CSC copy
// Column counts of each block of kSpBlockRows rows (one warp per block).
__global__ void __launch_bounds__(kSpWarps * 32) k_sp_block_count(int64_t m, int n, const int64_t* __restrict__ arp,
                                                                  const int32_t* __restrict__ acol,
                                                                  int32_t* __restrict__ cnt, int64_t nblocks) {
  extern __shared__ int32_t sp_cnt[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t blk = (int64_t)blockIdx.x * kSpWarps + warp;
  if (blk >= nblocks) return;
  int32_t* h = sp_cnt + (size_t)warp * n;
  for (int c = lane; c < n; c += 32) h[c] = 0;
  __syncwarp();
  const int64_t j0 = blk * kSpBlockRows, j1 = min(m, j0 + kSpBlockRows);
  for (int64_t j = j0; j < j1; ++j) {
    for (int64_t k = __ldg(arp + j) + lane; k < __ldg(arp + j + 1); k += 32) h[__ldg(acol + k)] += 1;
    __syncwarp();
  }
  for (int c = lane; c < n; c += 32) cnt[blk * n + c] = h[c];
}

// Per column: its total, and in place the running count of earlier blocks.
__global__ void k_sp_col_prefix(int n, int64_t nblocks, int32_t* __restrict__ cnt, int64_t* __restrict__ total) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int64_t run = 0;
  for (int64_t blk = 0; blk < nblocks; ++blk) {
    const int32_t v = cnt[blk * n + c];
    cnt[blk * n + c] = (int32_t)run;
    run += v;
  }
  total[c] = run;
}

// col_ptr = exclusive scan of the totals (one CTA; n <= 2048 here).
__global__ void __launch_bounds__(1024) k_sp_col_scan(int n, const int64_t* __restrict__ total,
                                                      int64_t* __restrict__ col_ptr) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int lo = tid * per, hi = min(n, lo + per);
  int64_t s = 0;
  for (int c = lo; c < hi; ++c) s += total[c];
  part[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = (tid >= off) ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;
  for (int c = lo; c < hi; ++c) {
    col_ptr[c] = run;
    run += total[c];
  }
  if (tid == 1023) col_ptr[n] = part[1023];
}

// Each block writes its rows in row order: (row, value) at col_ptr[c] + the
// running offset of column c.
__global__ void __launch_bounds__(kSpWarps * 32) k_sp_block_scatter(int64_t m, int n, const int64_t* __restrict__ arp,
                                                                    const int32_t* __restrict__ acol,
                                                                    const double* __restrict__ aval,
                                                                    const int32_t* __restrict__ cnt,
                                                                    const int64_t* __restrict__ col_ptr,
                                                                    int32_t* __restrict__ crow,
                                                                    double* __restrict__ cval, int64_t nblocks) {
  extern __shared__ int32_t sp_cur[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t blk = (int64_t)blockIdx.x * kSpWarps + warp;
  if (blk >= nblocks) return;
  int32_t* cur = sp_cur + (size_t)warp * n;
  for (int c = lane; c < n; c += 32) cur[c] = cnt[blk * n + c];
  __syncwarp();
  const int64_t j0 = blk * kSpBlockRows, j1 = min(m, j0 + kSpBlockRows);
  for (int64_t j = j0; j < j1; ++j) {
    for (int64_t k = __ldg(arp + j) + lane; k < __ldg(arp + j + 1); k += 32) {
      const int c = __ldg(acol + k);
      const int64_t p = col_ptr[c] + cur[c];
      cur[c] += 1;
      crow[p] = (int32_t)j;
      cval[p] = __ldg(aval + k);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- the pass
// r_j = b_j - A_j x (rows dealt to threads in a fixed pattern); r_prev <- r;
// per-CTA partials of ||r||^2, ||r - r_prev||^2 (first pass: the second is
// meaningless and ignored by the step kernel).
__global__ void __launch_bounds__(256) k_sp_residual(int64_t m, const int64_t* __restrict__ arp,
                                                     const int32_t* __restrict__ acol,
                                                     const double* __restrict__ aval, const double* __restrict__ b,
                                                     const double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ norms_part, const IterState* __restrict__ st) {
  if (st && st->done) return;
  double rn2 = 0.0, dn2 = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    double dot = 0.0;
    for (int64_t k = __ldg(arp + j); k < __ldg(arp + j + 1); ++k) dot += __ldg(aval + k) * x[__ldg(acol + k)];
    const double rj = __ldg(b + j) - dot;
    const double dl = rj - r[j];
    r[j] = rj;
    rn2 += rj * rj;
    dn2 += dl * dl;
  }
  // deterministic CTA sums (warp trees, then warps in order)
  __shared__ double red[2][8];
  rn2 = warp_sum(rn2);
  dn2 = warp_sum(dn2);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = rn2; red[1][w] = dn2; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    norms_part[2 * blockIdx.x + threadIdx.x] = s;
  }
}

// Segment sg of column c: sum of A_jc r_j over its rows (one warp).
__global__ void __launch_bounds__(256) k_sp_gradient(int n, int segs, const int64_t* __restrict__ col_ptr,
                                                     const int32_t* __restrict__ crow,
                                                     const double* __restrict__ cval, const double* __restrict__ r,
                                                     double* __restrict__ cpart, const IterState* __restrict__ st) {
  if (st && st->done) return;
  const int64_t wid = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)n * segs) return;
  const int c = (int)(wid % n), sg = (int)(wid / n);
  const int64_t lo = col_ptr[c], hi = col_ptr[c + 1];
  const int64_t len = hi - lo, per = (len + segs - 1) / segs;
  const int64_t s0 = lo + min(len, (int64_t)sg * per), s1 = lo + min(len, (int64_t)(sg + 1) * per);
  double acc = 0.0;
  for (int64_t e = s0 + lane; e < s1; e += 32) acc += __ldg(cval + e) * r[__ldg(crow + e)];
  acc = warp_sum(acc);
  if (lane == 0) cpart[(int64_t)sg * n + c] = acc;
}

// out[0..n) = sum over segments (in order); out[n], out[n+1] = sum of the
// per-CTA norm partials (in order).
__global__ void k_sp_reduce(int n, int segs, const double* __restrict__ cpart, int nnorm,
                            const double* __restrict__ norms_part, double* __restrict__ out,
                            const IterState* __restrict__ st) {
  if (st && st->done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    double s = 0.0;
    for (int sg = 0; sg < segs; ++sg) s += cpart[(int64_t)sg * n + k];
    out[k] = s;
  } else if (k < n + 2) {
    double s = 0.0;
    for (int q = 0; q < nnorm; ++q) s += norms_part[2 * q + (k - n)];
    out[k] = s;
  }
}

// ---------------------------------------------------------------- host side
size_t sp_gather_smem(int64_t n) { return sizeof(double) * kSpWarps * (size_t)(n + 1); }

cudaError_t launch_sp_gather(ls_ctx* ctx, int64_t d, const int64_t* srow, const uint32_t* sent, const int64_t* arp,
                             const int32_t* acol, const double* aval, const double* b, int64_t n, double scale,
                             double* B, int64_t ldb) {
  const size_t smem = sp_gather_smem(n);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sp_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  k_sp_gather<<<(unsigned)((d + kSpWarps - 1) / kSpWarps), kSpWarps * 32, smem, ctx->stream>>>(
      d, srow, sent, arp, acol, aval, b, (int)n, scale, B, ldb);
  ++ctx->launches;
  return cudaGetLastError();
}

int64_t sp_blocks(int64_t m) { return (m + kSpBlockRows - 1) / kSpBlockRows; }

cudaError_t launch_sp_csc(ls_ctx* ctx, int64_t m, int64_t n, const int64_t* arp, const int32_t* acol,
                          const double* aval, int32_t* cnt, int64_t* total, int64_t* col_ptr, int32_t* crow,
                          double* cval) {
  const int64_t nb = sp_blocks(m);
  const size_t smem = sizeof(int32_t) * kSpWarps * (size_t)n;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sp_block_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_sp_block_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  const unsigned grid = (unsigned)((nb + kSpWarps - 1) / kSpWarps);
  k_sp_block_count<<<grid, kSpWarps * 32, smem, ctx->stream>>>(m, (int)n, arp, acol, cnt, nb);
  k_sp_col_prefix<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>((int)n, nb, cnt, total);
  k_sp_col_scan<<<1, 1024, 0, ctx->stream>>>((int)n, total, col_ptr);
  k_sp_block_scatter<<<grid, kSpWarps * 32, smem, ctx->stream>>>(m, (int)n, arp, acol, aval, cnt, col_ptr, crow, cval,
                                                                 nb);
  ctx->launches += 4;
  return cudaGetLastError();
}

int sp_residual_grid(ls_ctx* ctx) { return ctx->num_sms * 8; }
int sp_segments(ls_ctx* ctx, int64_t n) {
  // about 8 warps per SM in total over the n columns
  return (int)std::max<int64_t>(1, ((int64_t)ctx->num_sms * 64 + n - 1) / n);
}

cudaError_t launch_sp_pass(ls_ctx* ctx, int64_t m, int64_t n, const int64_t* arp, const int32_t* acol,
                           const double* aval, const double* b, const double* x, double* r, const int64_t* col_ptr,
                           const int32_t* crow, const double* cval, double* norms_part, double* cpart, double* out,
                           const IterState* st) {
  const int g = sp_residual_grid(ctx), segs = sp_segments(ctx, n);
  k_sp_residual<<<g, 256, 0, ctx->stream>>>(m, arp, acol, aval, b, x, r, norms_part, st);
  const int64_t warps = n * segs;
  k_sp_gradient<<<(unsigned)((warps + 7) / 8), 256, 0, ctx->stream>>>((int)n, segs, col_ptr, crow, cval, r, cpart,
                                                                      st);
  k_sp_reduce<<<(unsigned)((n + 2 + 255) / 256), 256, 0, ctx->stream>>>((int)n, segs, cpart, g, norms_part, out, st);
  ctx->launches += 3;
  return cudaGetLastError();
}

}  // namespace lsk
