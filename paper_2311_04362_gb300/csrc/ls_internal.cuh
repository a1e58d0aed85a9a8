// ls_internal.cuh -- shared declarations of the libls CUDA sources (sm_103a).
//
// Device helpers used by several kernels: the Philox4x32-10 counter hash
// (Salmon et al., SC'11), Lemire's bounded draw, bounded-time waits on
// mbarriers and on a grid barrier, and thin inline-PTX wrappers for TMA
// (cp.async.bulk.tensor), mbarrier and thread-block-cluster operations.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "../../include/ls.h"

// ---------------------------------------------------------------- status bits
// Written by kernels into ctx->d_status; mapped to ls_status on the host.
#define LS_DEV_TIMEOUT 1u
#define LS_DEV_RANK 2u
#define LS_DEV_NONFINITE 4u
#define LS_DEV_BADSIZE 8u

// A bounded wait gives up after this many nanoseconds of %globaltimer.
#define LS_WAIT_NS 2000000000ull

namespace lsk {

// --------------------------------------------------------------- Philox4x32-10
struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ inline u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    u32x4 n;
    n.x = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
    n.y = (uint32_t)p1;
    n.z = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
    n.w = (uint32_t)p0;
    c = n;
  }
  return c;
}

// Word stream of one counter family: block t = philox(lo(idx), hi(idx), t, dom).
struct WordStream {
  uint32_t k0, k1, c0, c1, dom, blk;
  uint32_t buf[4];
  int pos;
  __host__ __device__ WordStream(uint64_t seed, uint64_t idx, uint32_t domain)
      : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0((uint32_t)idx),
        c1((uint32_t)(idx >> 32)), dom(domain), blk(0), pos(4) {}
  __host__ __device__ uint32_t next() {
    if (pos == 4) {
      u32x4 o = philox10(u32x4{c0, c1, blk, dom}, k0, k1);
      buf[0] = o.x; buf[1] = o.y; buf[2] = o.z; buf[3] = o.w;
      ++blk;
      pos = 0;
    }
    return buf[pos++];
  }
  // Uniform in [0, range), range >= 1 (Lemire's multiply-shift with rejection).
  __host__ __device__ uint32_t below(uint32_t range) {
    uint64_t p = (uint64_t)next() * range;
    uint32_t lo = (uint32_t)p;
    if (lo < range) {
      const uint32_t thr = (uint32_t)(0u - range) % range;
      while (lo < thr) { p = (uint64_t)next() * range; lo = (uint32_t)p; }
    }
    return (uint32_t)(p >> 32);
  }
};

// ------------------------------------------------------------------ timers
__device__ inline uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// --------------------------------------------------------------- mbarrier
__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ inline void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false if the deadline passed.
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0 && gtimer() > deadline) return false;
  }
  return true;
}

// ------------------------------------------------------------------- TMA
__device__ inline void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ inline void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// ---------------------------------------------------------------- clusters
__device__ inline uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ inline uint32_t cluster_nctas() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ inline void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of `p` (this CTA's shared memory) in the shared window of CTA `rank`.
__device__ inline uint32_t map_shared(const void* p, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}
__device__ inline void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ inline double ld_cluster_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

// Store v into the shared memory of a cluster peer (addresses from
// map_shared); the 8 bytes count toward the peer's mbarrier transaction.
__device__ inline void st_async_f64(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
               "l"(__double_as_longlong(v)), "r"(bar)
               : "memory");
}

// ------------------------------------------------------------- grid barrier
// Sense-free generation barrier for a cooperative launch (all CTAs are
// co-resident).  Every wait is bounded; on timeout the status word gets
// LS_DEV_TIMEOUT and all CTAs return false from then on.
struct GridBar {
  unsigned int* count;   // zero-initialised
  unsigned int* gen;
  unsigned int* status;
};

__device__ inline bool grid_sync(const GridBar& gb, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = gb.gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(gb.count, 1u);
    if (arrived == nblocks - 1) {
      *gb.count = 0;
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      const uint64_t deadline = gtimer() + LS_WAIT_NS;
      uint32_t spins = 0;
      while (*vgen == g) {
        if ((++spins & 63u) == 0) {
          if (gtimer() > deadline) { atomicOr(gb.status, LS_DEV_TIMEOUT); ok = 0; break; }
          if (*(volatile unsigned int*)gb.status & LS_DEV_TIMEOUT) { ok = 0; break; }
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Monotonic grid barrier for a cooperative launch.  The counter only grows
// (zeroed before the launch): a CTA's e-th barrier completes when it reaches
// e * nblocks.  Arriving is one fenced add per CTA and waiting polls with
// acquire loads, so a barrier costs about two L2 round trips; arrive and
// wait are separate so that a CTA can do local work while the others
// arrive.  Waits are bounded like grid_sync's.  Every thread of every CTA
// calls both, in the same order.
struct MonoBar {
  unsigned int* count;   // zero-initialised
  unsigned int* status;
  unsigned int epoch;
};

__device__ inline void mono_arrive(MonoBar& b) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(b.count, 1u);
  }
  ++b.epoch;
}

__device__ inline bool mono_wait(MonoBar& b, unsigned int nblocks) {
  __shared__ int s_mono_ok;
  if (threadIdx.x == 0) {
    const unsigned int target = b.epoch * nblocks;
    int ok = 1;
    const uint64_t deadline = gtimer() + LS_WAIT_NS;
    uint32_t spins = 0;
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(b.count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 63u) == 0) {
        if (gtimer() > deadline) { atomicOr(b.status, LS_DEV_TIMEOUT); ok = 0; break; }
        if (*(volatile unsigned int*)b.status & LS_DEV_TIMEOUT) { ok = 0; break; }
      }
    }
    s_mono_ok = ok;
  }
  __syncthreads();
  return s_mono_ok != 0;
}

__device__ inline bool mono_sync(MonoBar& b, unsigned int nblocks) {
  mono_arrive(b);
  return mono_wait(b, nblocks);
}

// v with its sign flipped when bit 0 of en is set (an integer XOR on the sign
// bit), so that acc + signed_by(v, en) is acc + v or acc - v exactly (IEEE
// subtraction is addition of the negation) with a single FP64 add.
__device__ inline double signed_by(double v, uint32_t en) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(en & 1u) << 63));
}
__device__ inline float signed_by(float v, uint32_t en) {
  return __int_as_float(__float_as_int(v) ^ (int)((en & 1u) << 31));
}

// ------------------------------------------------------------ reductions
// Block-wide bitonic sort of s[0..P) ascending (P a power of two; every
// thread of the block calls it).
__device__ inline void bitonic(uint32_t* s, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = s[i], b = s[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { s[i] = b; s[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lsk

// -------------------------------------------------------------------- context
// Geometry of the batched fused pass, per class of n (the autotuner's table).
constexpr int kTuneBuckets = 6;   // n in [1,32), [32,64), [64,128), [128,256), [256,512), [512,1024]
struct PassTune {
  int tile[kTuneBuckets];       // doubles of one tile (tr * stride <= tile)
  int item_rows[kTuneBuckets];  // rows per pass item (one partial per item)
  int tuned[kTuneBuckets];      // 1 where a measurement chose the entry
};
inline int tune_bucket(int64_t n) {
  int b = 0;
  while (b < kTuneBuckets - 1 && n >= (32ll << b)) ++b;
  return b;
}
inline PassTune default_tune() {
  PassTune t;
  for (int b = 0; b < kTuneBuckets; ++b) { t.tile[b] = 3840; t.item_rows[b] = 128; t.tuned[b] = 0; }
  return t;
}

struct ls_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // device arena (grown on demand, never shrunk)
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // small persistent device buffers
  unsigned int* d_status = nullptr;    // [0] status bits, [1..3] barrier counters
  int* d_misc = nullptr;               // small integer scratch (max bucket size, ...)
  // pinned host mirror for readbacks
  void* h_pinned = nullptr;
  // staging for host inputs of ls_solve
  char* stage = nullptr;
  size_t stage_bytes = 0;
  // sort scratch for sketch rows with more than the shared-memory capacity
  void* aux = nullptr;
  size_t aux_bytes = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> pass_ev;    // two per fused-pass launch of ls_iterate
  long long launches = 0;              // kernels launched (for ls_info)
  // TMA encode entry point
  void* encode_tiled = nullptr;
  // batched pass geometry (ls_tune_batched)
  PassTune tune = default_tune();
  // host inputs of ls_solve*: A is uploaded on a stream of its own while the
  // sketch's indices and CSR (which do not read A) run on `stream`
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_done = nullptr;
  cudaEvent_t piece_done[4] = {nullptr, nullptr, nullptr, nullptr};   // host A uploaded piece by piece
  // ls_solve*: A is put in fixed point on this stream while the QR runs
  cudaStream_t fx_stream = nullptr;
  cudaEvent_t fx_done = nullptr;
  // bounded device waits of the fixed-point pass give up after this long
  unsigned long long wait_ns = LS_WAIT_NS;
  // failure injection for tests (ls_inject_fault): the next fixed-point pass's
  // CTA 0 skips this tile (-1: none); the next device allocation fails (0: none)
  int inject_skip_tile = -1;
  int inject_alloc_fail = 0;
};

// ------------------------------------------------------------ launch helpers
// Implemented in sketch.cu / factor.cu / iterate.cu; all enqueue on ctx->stream
// and return cudaSuccess or the first launch error.
namespace lsk {

cudaError_t launch_sketch_indices(ls_ctx* ctx, int64_t m, int64_t d, int zeta, uint64_t seed,
                                  int32_t* rows, uint32_t* signs);
// With max_bucket_host != null: histogram + scan only, returns the largest
// bucket (synchronises).  Otherwise histogram, scan, scatter and bucket sort.
cudaError_t launch_sketch_csr(ls_ctx* ctx, int64_t m, int64_t d, int zeta, const int32_t* rows,
                              const uint32_t* signs, int64_t* row_ptr, uint32_t* ent,
                              unsigned long long* fill, uint32_t* sort_scratch, int* max_bucket_host);
int sketch_sort_cap();
cudaError_t launch_sketch_apply(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                                const double* b, int64_t d, const int64_t* row_ptr,
                                const uint32_t* ent, double scale, double* B, int64_t ldb);
// Gather by row pieces of A (as they are uploaded): bounds[0] = 0 <
// bounds[1] < ... < bounds[np] = m; split gets d * (np + 1) entry offsets.
constexpr int kMaxPieces = 4;
struct PieceBounds { int64_t r[kMaxPieces + 1]; };
cudaError_t launch_sketch_split(ls_ctx* ctx, int64_t d, const int64_t* row_ptr, const uint32_t* ent, int np,
                                const PieceBounds& bnd, int64_t* split);
cudaError_t launch_sketch_gather_b(ls_ctx* ctx, const double* b, int64_t d, const int64_t* row_ptr,
                                   const uint32_t* ent, double scale, double* Bcol);
cudaError_t launch_sketch_gather_piece(ls_ctx* ctx, const double* A, int64_t n, int64_t lda, int64_t d,
                                       const int64_t* split, int np, int piece, const uint32_t* ent, double scale,
                                       double* B, int64_t ldb);

int householder_ctas(const ls_ctx* ctx, int64_t d);
size_t householder_part_doubles(const ls_ctx* ctx, int64_t d, int64_t n);
size_t householder_w_doubles(int64_t n);
cudaError_t launch_householder(ls_ctx* ctx, double* B, int64_t d, int64_t n, int64_t ldb,
                               double* part, double* w);
cudaError_t launch_prepare_R(ls_ctx* ctx, const double* src, int64_t lds, int64_t n, double* R_out,
                             int64_t ldr, double* Rt, double* inv_diag);
cudaError_t launch_post_factor(ls_ctx* ctx, const double* B, int64_t d, int64_t n, int64_t ldb,
                               const double* R, int64_t ldr, double* x0, uint64_t seed,
                               const double* Rt, const double* inv_diag, double* vecs /* 4n+64 */,
                               double* est_out /* 2 */);

// Iteration state on the device.
struct IterState {
  int iter;          // updates applied
  int done;          // 1: stop (rule held and extra updates done) or error
  int fired;         // the stopping rule has held
  int extra_left;    // updates remaining after the rule held
  int stop_reason;   // 0 rule held, 1 q reached, 3 non-finite
  int nonfinite;
  int have_prev;     // r_prev holds r(x_{i-1})
  int pad;           // batched path: 1 = rank deficient, to be reported
  double xnorm;      // ||x_i||
  double rnorm;      // ||r(x_i)||
  double dnorm;      // ||r(x_i) - r(x_{i-1})||
  double normest, condest, gamma, rho, alpha, beta;
};

struct PassGeom {
  int boxw;      // TMA box width (columns), even, <= 256
  int nbox;      // boxes per row
  int tr;        // rows per tile
  int stages;    // pipeline stages
  size_t smem;   // dynamic shared memory bytes
  int grid;      // CTAs (one per SM)
};
PassGeom pass_geometry(const ls_ctx* ctx, int64_t n, int64_t m);
cudaError_t make_tensor_map(ls_ctx* ctx, CUtensorMap* map, const double* A, int64_t m, int64_t n,
                            int64_t lda, const PassGeom& g);
cudaError_t launch_fused_pass(ls_ctx* ctx, const CUtensorMap& map, const PassGeom& g, int64_t m,
                              int64_t n, const double* b, const double* x, const double* r_prev,
                              double* r_out, double* part, const IterState* st);
cudaError_t launch_reduce_partials(ls_ctx* ctx, const double* part, int nparts, int64_t n,
                                   double* c, double* norms);

struct StepArgs {
  const double* part; int nparts;
  const double* Rt; const double* R; int64_t ldr; const double* inv_diag; int n;
  double* x; double* x_prev;
  double* y; double* dvec; double* work; double* slots;
  IterState* st;
  int use_stop; int extra;
  unsigned int* status;
  const double* c_in;     // k_correct: c given directly
  double* y_out; double* d_out;
};
cudaError_t launch_iter_step(ls_ctx* ctx, const StepArgs& a);
int ts_cluster_size_of(const void* const* fns, int nfn);

// sparse A (sparse.cu)
size_t sp_gather_smem(int64_t n);
cudaError_t launch_sp_gather(ls_ctx* ctx, int64_t d, const int64_t* srow, const uint32_t* sent, const int64_t* arp,
                             const int32_t* acol, const double* aval, const double* b, int64_t n, double scale,
                             double* B, int64_t ldb);
int64_t sp_blocks(int64_t m);
cudaError_t launch_sp_csc(ls_ctx* ctx, int64_t m, int64_t n, const int64_t* arp, const int32_t* acol,
                          const double* aval, int32_t* cnt, int64_t* total, int64_t* col_ptr, int32_t* crow,
                          double* cval);
int sp_residual_grid(ls_ctx* ctx);
int sp_segments(ls_ctx* ctx, int64_t n);
cudaError_t launch_sp_pass(ls_ctx* ctx, int64_t m, int64_t n, const int64_t* arp, const int32_t* acol,
                           const double* aval, const double* b, const double* x, double* r, const int64_t* col_ptr,
                           const int32_t* crow, const double* cval, double* norms_part, double* cpart, double* out,
                           const IterState* st);

// fixed-point fused pass (fxpass.cu)
struct FxGeom {
  int boxw, nbox, tr, stages;
  size_t smem;
  int grid;
};
FxGeom fx_geometry(const ls_ctx* ctx, int64_t n, int64_t m);
size_t fx_part_words(const FxGeom& g, int64_t n);
constexpr int64_t kFxMaxN = 1024;
cudaError_t launch_to_fixed(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, int2* Af, int64_t ldf,
                            int* rexp);
cudaError_t make_fx_tensor_map(ls_ctx* ctx, CUtensorMap* map, const int2* Af, int64_t m, int64_t n, int64_t ldf,
                               const FxGeom& g);
cudaError_t launch_fx_pass(ls_ctx* ctx, const CUtensorMap& map, const FxGeom& g, int64_t m, int64_t n,
                           const int* rexp, const double* b, const double* x, const double* r_prev, double* r_out,
                           long long* part, const IterState* st);
cudaError_t launch_fx_reduce(ls_ctx* ctx, const long long* part, int nparts, int64_t n, double* c, double* norms,
                             const IterState* st);

// batched path (batched.cu)
// One problem of a batched solve or one server slot: caller's arrays, sizes,
// offsets of its parts in the pools, and its pass tile geometry.
struct BProb {
  const double* A; const double* b; double* x;
  int64_t m, n, lda, d;
  uint64_t seed;
  int64_t moff;      // sum of m over earlier problems (flattened columns of S)
  int64_t doff;      // sum of d (buckets)
  int64_t boff;      // sum of d (n + 1) (B pool)
  int64_t roff;      // R at roff, R^T at roff + n^2 (R pool)
  int64_t voff;      // 8 n-vectors at voff (V pool): 1/diag R, x_prev, y, d, work, v, w, xi
  int64_t rpoff;     // r_prev (m doubles) in the r_prev pool
  int64_t toff;      // sum of gather warps (k_b_gather)
  int64_t poff;      // sum of tiles (n + 2) (partials)
  int tr;            // rows per pass tile
  int tiles;         // pass tiles
  int ss;            // shared-memory row stride of a tile (doubles, = 2 mod 4)
  int S;             // column chunks per row in the row-dot phase (S * tr <= 256)
  int rowcopy;       // 1: one bulk copy per row (lda != ss), 0: one per tile
  int gw;            // gather lanes per bucket (32, 16, 8 or 4)
  int tpi;           // pass tiles per item (one partial per item)
  int items;         // pass items
};
// Completion record of a problem (server mode).
struct BDone {
  int slot, iters, stop_reason, pad;
  double res_norm, step_norm, normest, condest;
};
struct BPools {
  double* B;        // sketches [S A, S b] at boff
  double* R;        // R at roff, R^T at roff + n^2
  double* V;        // 8 n-vectors at voff
  double* part;     // pass partials at poff
  double* r_prev;   // previous residuals at rpoff
  double* slots;    // 64 per problem (cluster reductions)
  double* est;      // normest, condest per problem
  IterState* st;
  unsigned int* pstatus;
  BDone* done_rec;            // completion queue (null: not recorded)
  unsigned int* done_count;
};
struct BatchPlan {
  int np;
  int64_t mtotal, dtotal, btotal, rtotal, vtotal, ttotal, ptotal;
  int64_t wtotal;                // gather warps
  int max_n, max_tile_doubles;   // max_tile_doubles: unused
  int64_t max_d, max_m;
  int cap;                       // doubles per pass buffer (largest tile used)
  double max_fill;               // largest m / d (mean bucket size / zeta)
};
bool b_csr_fits(const BatchPlan& pl);
int64_t b_csr_global_entries();
cudaError_t launch_b_csr(ls_ctx* ctx, const BProb* dP, const BatchPlan& pl, int zeta, const int32_t* rows,
                         const uint32_t* signs, int64_t* row_ptr, uint32_t* ent, uint32_t* scratch);
size_t bprob_bytes();
void batch_plan(const ls_problem* probs, int np, BProb* out, BatchPlan& pl, const PassTune& tune);
int tune_cap(const PassTune& t);   // the largest tile of the table (doubles per pass buffer)
void batch_offsets(const BProb* P, int np, int64_t* moffs, int64_t* doffs, int64_t* toffs);
int64_t batch_boff(const BProb* P, int p);
int64_t batch_roff(const BProb* P, int p);
cudaError_t launch_b_sketch_indices(ls_ctx* ctx, const BProb* dP, const int64_t* dmoffs, const BatchPlan& pl,
                                    int zeta, int32_t* rows, uint32_t* signs);
cudaError_t launch_b_gather(ls_ctx* ctx, const BProb* dP, const int64_t* dwoffs, const BatchPlan& pl,
                            const int64_t* row_ptr, const uint32_t* ent, double scale, double* Bpool);
int batch_order(const BProb* P, int np, int* order, bool clusters);
cudaError_t launch_b_factor(ls_ctx* ctx, const BProb* dP, const int* dorder, int count, const int* list,
                            const BPools& pools);
int b_qr_cluster_size(ls_ctx* ctx);
int b_qr_cluster_max_n();
cudaError_t launch_b_factor2(ls_ctx* ctx, const BProb* dP, const int* dorder, int nsmall, const int* dbig, int nbig,
                             int csize, int count, const int* list, const BPools& pools);
cudaError_t launch_b_gather32(ls_ctx* ctx, const BProb* dP, const int64_t* dwoffs, const BatchPlan& pl,
                              const int64_t* row_ptr, const uint32_t* ent, double scale, float* B32);
cudaError_t launch_b_factor_mixed(ls_ctx* ctx, const BProb* dP, const BProb* dP64, const int* dorder, int np,
                                  float* B32, double* Bc, const BPools& pools);
cudaError_t launch_widen(ls_ctx* ctx, const float* src, double* dst, int64_t count);
cudaError_t launch_b_iter_init(ls_ctx* ctx, const BProb* dP, int count, const int* list, const BPools& pools,
                               double gamma, double rho, double alpha, double beta);
cudaError_t launch_b_compact(ls_ctx* ctx, const BProb* dP, int np, const BPools& pools, int* alist, int64_t* aoff,
                             int64_t* cnt);
int b_pass_grid(ls_ctx* ctx, int max_n, int cap);
cudaError_t launch_b_pass(ls_ctx* ctx, const BProb* dP, const int* alist, const int64_t* aoff, int64_t* cnt,
                          int max_n, int cap, int64_t max_items, const BPools& pools);
cudaError_t launch_b_step(ls_ctx* ctx, const BProb* dP, const int* alist, const int64_t* cnt, int np,
                          const BPools& pools, int use_stop, int extra, int q);
cudaError_t launch_correct(ls_ctx* ctx, const StepArgs& a);

}  // namespace lsk
