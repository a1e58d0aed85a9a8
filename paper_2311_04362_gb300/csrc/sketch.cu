// sketch.cu -- the sparse sign embedding and B_aug = S [A b] (Algorithm 2,
// sketch step; Sec. 2.2, Eq. (2.4)).
//
//  (a1) k_sparse_sign : one thread per column j of S.  Philox4x32-10 word
//       stream keyed by the seed (counter (j lo, j hi, block, 0)); word 0 is
//       the sign mask, the following words drive Floyd's subset sampling of
//       zeta distinct rows in [0, d) with Lemire's bounded draw; rows sorted
//       ascending, bit k of the mask is the sign of the k-th smallest row.
//  (a2) counting sort : integer histogram (atomics on integers only, so the
//       counts are exact), one-CTA exclusive scan, atomic scatter into the
//       buckets, then a bitonic sort of every bucket by its packed
//       (j << 1 | neg) keys -- the keys are distinct, so the sorted bucket is
//       unique and the CSR is bit-identical to a stable counting sort.
//  (a3) k_gather_add : B[t, c] = s * (sum over the bucket of row t, ascending
//       j, of +-A[j, c]) -- a segmented gather-add with 128-bit row loads and
//       no floating-point atomics; every entry is summed left to right from
//       +0.0, so the result is deterministic.
#include "ls_internal.cuh"

namespace lsk {

static constexpr int kSortCap = 8192;  // keys sorted in shared memory per bucket

// ---------------------------------------------------------------- (a1)
__global__ void __launch_bounds__(256) k_sparse_sign(int64_t m, int64_t d, int zeta, uint64_t seed,
                                                     int32_t* __restrict__ rows,
                                                     uint32_t* __restrict__ signs) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  WordStream s(seed, (uint64_t)j, 0u);
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
  int32_t* out = rows + j * zeta;
  for (int i = 0; i < cnt; ++i) out[i] = r[i];
  signs[j] = mask;
}

// ---------------------------------------------------------------- (a2)
__global__ void k_hist(int64_t total, const int32_t* __restrict__ rows, unsigned long long* __restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[rows[e]], 1ull);
}

// One CTA: row_ptr = exclusive scan of cnt (d entries); cnt <- row_ptr (fill
// cursors); misc[0] <- largest bucket.
__global__ void __launch_bounds__(1024) k_scan(int64_t d, unsigned long long* __restrict__ cnt,
                                               int64_t* __restrict__ row_ptr, int* __restrict__ misc) {
  __shared__ unsigned long long part[1024];
  __shared__ unsigned long long mx[1024];
  const int tid = threadIdx.x;
  const int64_t chunk = (d + 1023) / 1024;
  const int64_t lo = tid * chunk, hi = min(d, lo + chunk);
  unsigned long long s = 0, m = 0;
  for (int64_t t = lo; t < hi; ++t) { s += cnt[t]; m = max(m, cnt[t]); }
  part[tid] = s;
  mx[tid] = m;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // Hillis-Steele inclusive scan
    const unsigned long long v = (tid >= off) ? part[tid - off] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  for (int off = 512; off > 0; off >>= 1) {     // largest bucket
    if (tid < off) mx[tid] = max(mx[tid], mx[tid + off]);
    __syncthreads();
  }
  unsigned long long run = part[tid] - s;  // exclusive prefix of this chunk
  for (int64_t t = lo; t < hi; ++t) {
    const unsigned long long c = cnt[t];
    row_ptr[t] = (int64_t)run;
    cnt[t] = run;
    run += c;
  }
  if (tid == 1023) row_ptr[d] = (int64_t)part[1023];
  if (tid == 0) misc[0] = (int)mx[0];
}

__global__ void k_scatter(int64_t m, int zeta, const int32_t* __restrict__ rows, const uint32_t* __restrict__ signs,
                          unsigned long long* __restrict__ fill, uint32_t* __restrict__ ent) {
  const int64_t total = m * zeta;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / zeta;
    const int k = (int)(e - j * zeta);
    const uint32_t neg = (signs[j] >> k) & 1u;
    const unsigned long long pos = atomicAdd(&fill[rows[e]], 1ull);
    ent[pos] = ((uint32_t)j << 1) | neg;
  }
}

// One CTA per sketch row: sort its bucket ascending.  Buckets larger than
// kSortCap are sorted in global scratch at offset 2*row_ptr[t] (room for the
// next power of two of the bucket size).
__global__ void __launch_bounds__(256) k_bucket_sort(int64_t d, const int64_t* __restrict__ row_ptr,
                                                     uint32_t* __restrict__ ent, uint32_t* __restrict__ scratch,
                                                     unsigned int* __restrict__ status) {
  extern __shared__ uint32_t sk[];
  const int64_t t = blockIdx.x;
  if (t >= d) return;
  const int64_t b0 = row_ptr[t];
  const int64_t sz = row_ptr[t + 1] - b0;
  if (sz <= 1) return;
  int P = 1;
  while (P < sz) P <<= 1;
  uint32_t* buf = (P <= kSortCap) ? sk : (scratch + 2 * b0);
  if (P > kSortCap && scratch == nullptr) {        // the host sizes scratch from the largest bucket
    if (threadIdx.x == 0) atomicOr(status, LS_DEV_BADSIZE);
    return;
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) buf[i] = (i < sz) ? ent[b0 + i] : 0xFFFFFFFFu;
  __syncthreads();
  bitonic(buf, P);
  for (int i = threadIdx.x; i < sz; i += blockDim.x) ent[b0 + i] = buf[i];
}

// ---------------------------------------------------------------- (a3)
// CTA tile: 32 sketch rows x 64 columns of A; warp w owns rows 4w..4w+3 of
// the tile, lane l owns columns 2l, 2l+1 (one 16-byte load per bucket entry).
// With split != null only the entries of row piece `piece` of np are added:
// each bucket's running sum is kept unscaled in B between pieces (piece 0
// starts from 0, later pieces continue it) and the last piece applies the
// scale, so the sums and their order, and B, are those of one launch.
__global__ void __launch_bounds__(256) k_gather_add(const double* __restrict__ A, int64_t lda, int64_t n, int64_t d,
                                                    const int64_t* __restrict__ row_ptr,
                                                    const uint32_t* __restrict__ ent, double scale,
                                                    double* __restrict__ B, int64_t ldb,
                                                    const int64_t* __restrict__ split, int np, int piece) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.y * 64 + 2 * lane;
  const bool pair = (c + 1 < n), single = (c < n);
  const bool first = (split == nullptr) || piece == 0, last = (split == nullptr) || piece == np - 1;
  for (int tt = 0; tt < 4; ++tt) {
    const int64_t t = (int64_t)blockIdx.x * 32 + warp * 4 + tt;
    if (t >= d) break;
    int64_t e0, e1;
    if (split) {
      e0 = split[t * (np + 1) + piece];
      e1 = split[t * (np + 1) + piece + 1];
    } else {
      e0 = row_ptr[t];
      e1 = row_ptr[t + 1];
    }
    double a0 = 0.0, a1 = 0.0;
    if (!first) {
      if (single) a0 = B[t + c * ldb];
      if (pair) a1 = B[t + (c + 1) * ldb];
    }
    int64_t e = e0;
    for (; e + 8 <= e1; e += 8) {
      uint32_t en[8];
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) en[u] = __ldg(ent + e + u);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const double* p = A + (int64_t)(en[u] >> 1) * lda + c;
        if (pair) v[u] = __ldg(reinterpret_cast<const double2*>(p));
        else if (single) { v[u].x = __ldg(p); v[u].y = 0.0; }
        else { v[u].x = 0.0; v[u].y = 0.0; }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a0 = a0 + signed_by(v[u].x, en[u]);
        a1 = a1 + signed_by(v[u].y, en[u]);
      }
    }
    for (; e < e1; ++e) {
      const uint32_t en = __ldg(ent + e);
      const double* p = A + (int64_t)(en >> 1) * lda + c;
      double2 v = make_double2(0.0, 0.0);
      if (pair) v = __ldg(reinterpret_cast<const double2*>(p));
      else if (single) v.x = __ldg(p);
      a0 = a0 + signed_by(v.x, en);
      a1 = a1 + signed_by(v.y, en);
    }
    if (single) B[t + c * ldb] = last ? scale * a0 : a0;
    if (pair) B[t + (c + 1) * ldb] = last ? scale * a1 : a1;
  }
}

// split[t * (np + 1) + i] = the first entry of bucket t whose row is >=
// bnd.r[i] (a bucket's entries ascend by row; entry = row << 1 | sign).
__global__ void k_split_entries(int64_t d, const int64_t* __restrict__ row_ptr, const uint32_t* __restrict__ ent,
                                int np, PieceBounds bnd, int64_t* __restrict__ split) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d) return;
  const int64_t e0 = row_ptr[t], e1 = row_ptr[t + 1];
  split[t * (np + 1)] = e0;
  split[t * (np + 1) + np] = e1;
  for (int i = 1; i < np; ++i) {
    int64_t lo = e0, hi = e1;                       // first entry with row >= bnd.r[i]
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if ((int64_t)(__ldg(ent + mid) >> 1) < bnd.r[i]) lo = mid + 1;
      else hi = mid;
    }
    split[t * (np + 1) + i] = lo;
  }
}

// Column n of B_aug: S b, one thread per sketch row.
__global__ void k_gather_b(const double* __restrict__ b, int64_t d, const int64_t* __restrict__ row_ptr,
                           const uint32_t* __restrict__ ent, double scale, double* __restrict__ Bcol) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d) return;
  double acc = 0.0;
  for (int64_t e = row_ptr[t]; e < row_ptr[t + 1]; ++e) {
    const uint32_t en = __ldg(ent + e);
    const double v = __ldg(b + (en >> 1));
    acc = acc + signed_by(v, en);
  }
  Bcol[t] = scale * acc;
}

// ---------------------------------------------------------------- host side
cudaError_t launch_sketch_indices(ls_ctx* ctx, int64_t m, int64_t d, int zeta, uint64_t seed,
                                  int32_t* rows, uint32_t* signs) {
  if (m == 0) return cudaSuccess;
  const int64_t grid = (m + 255) / 256;
  k_sparse_sign<<<(unsigned)grid, 256, 0, ctx->stream>>>(m, d, zeta, seed, rows, signs);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_sketch_csr(ls_ctx* ctx, int64_t m, int64_t d, int zeta, const int32_t* rows,
                              const uint32_t* signs, int64_t* row_ptr, uint32_t* ent,
                              unsigned long long* fill, uint32_t* sort_scratch, int* max_bucket_host) {
  cudaError_t e;
  const int64_t total = m * zeta;
  if ((e = cudaMemsetAsync(fill, 0, sizeof(unsigned long long) * d, ctx->stream)) != cudaSuccess) return e;
  const int gridE = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
  if (total > 0) {
    k_hist<<<gridE, 256, 0, ctx->stream>>>(total, rows, fill);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_scan<<<1, 1024, 0, ctx->stream>>>(d, fill, row_ptr, ctx->d_misc);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (max_bucket_host) {
    // the caller needs the largest bucket before the sort (scratch sizing)
    if ((e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_misc, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return e;
    *max_bucket_host = *(int*)ctx->h_pinned;
    return cudaSuccess;
  }
  if (total > 0) {
    k_scatter<<<gridE, 256, 0, ctx->stream>>>(m, zeta, rows, signs, fill, ent);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bucket_sort<<<(unsigned)d, 256, kSortCap * sizeof(uint32_t), ctx->stream>>>(d, row_ptr, ent, sort_scratch,
                                                                                  ctx->d_status);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int sketch_sort_cap() { return kSortCap; }

cudaError_t launch_sketch_apply(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                                const double* b, int64_t d, const int64_t* row_ptr,
                                const uint32_t* ent, double scale, double* B, int64_t ldb) {
  (void)m;
  cudaError_t e;
  dim3 grid((unsigned)((d + 31) / 32), (unsigned)((n + 63) / 64));
  k_gather_add<<<grid, 256, 0, ctx->stream>>>(A, lda, n, d, row_ptr, ent, scale, B, ldb, nullptr, 1, 0);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_b<<<(unsigned)((d + 255) / 256), 256, 0, ctx->stream>>>(b, d, row_ptr, ent, scale, B + n * ldb);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_sketch_split(ls_ctx* ctx, int64_t d, const int64_t* row_ptr, const uint32_t* ent, int np,
                                const PieceBounds& bnd, int64_t* split) {
  if (np < 1 || np > kMaxPieces) return cudaErrorInvalidValue;
  k_split_entries<<<(unsigned)((d + 255) / 256), 256, 0, ctx->stream>>>(d, row_ptr, ent, np, bnd, split);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_sketch_gather_b(ls_ctx* ctx, const double* b, int64_t d, const int64_t* row_ptr,
                                   const uint32_t* ent, double scale, double* Bcol) {
  k_gather_b<<<(unsigned)((d + 255) / 256), 256, 0, ctx->stream>>>(b, d, row_ptr, ent, scale, Bcol);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_sketch_gather_piece(ls_ctx* ctx, const double* A, int64_t n, int64_t lda, int64_t d,
                                       const int64_t* split, int np, int piece, const uint32_t* ent, double scale,
                                       double* B, int64_t ldb) {
  dim3 grid((unsigned)((d + 31) / 32), (unsigned)((n + 63) / 64));
  k_gather_add<<<grid, 256, 0, ctx->stream>>>(A, lda, n, d, nullptr, ent, scale, B, ldb, split, np, piece);
  ++ctx->launches;
  return cudaGetLastError();
}

}  // namespace lsk
