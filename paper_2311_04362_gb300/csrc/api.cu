// api.cu -- the extern "C" entry points declared in include/ls.h: argument
// checks, the context's scratch arena, and the order of kernel launches for
// each step of Algorithm 2 (sketch, factor, start, iterate).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <string>
#include <vector>

#include "ls_internal.cuh"

using namespace lsk;

namespace {

ls_status fail(ls_ctx* ctx, ls_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

#define CUDA_TRY(ctx, call)                                                                       \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      if (e_ == cudaErrorMemoryAllocation) return fail(ctx, LS_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_)); \
      return fail(ctx, LS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                     \
    }                                                                                             \
  } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over the context arena; `plan` first measures, then carves.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += align256(count * sizeof(T));
    return p;
  }
};

ls_status ensure_arena(ls_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->arena_bytes) return LS_OK;
  if (ctx->inject_alloc_fail) {                 // test hook (ls_inject_fault)
    ctx->inject_alloc_fail = 0;
    return fail(ctx, LS_ENOMEM, "device scratch of %zu bytes could not be allocated (injected failure)", bytes);
  }
  if (ctx->arena) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&ctx->arena, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, LS_ENOMEM, "device scratch of %zu bytes could not be allocated", want);
  }
  ctx->arena_bytes = want;
  return LS_OK;
}

ls_status ensure_stage(ls_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return LS_OK;
  if (ctx->stage) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
  }
  if (cudaMalloc(&ctx->stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, LS_ENOMEM, "device staging of %zu bytes could not be allocated", bytes);
  }
  ctx->stage_bytes = bytes;
  return LS_OK;
}

// Separate buffer for the large-bucket sort scratch (sized after the
// histogram, so growing it never moves the arena).
ls_status ensure_aux(ls_ctx* ctx, void** aux, size_t* aux_bytes, size_t bytes) {
  if (bytes <= *aux_bytes) return LS_OK;
  if (*aux) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(*aux);
    *aux = nullptr;
    *aux_bytes = 0;
  }
  if (cudaMalloc(aux, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, LS_ENOMEM, "sort scratch of %zu bytes could not be allocated", bytes);
  }
  *aux_bytes = bytes;
  return LS_OK;
}

// status word handling -------------------------------------------------------
ls_status reset_status(ls_ctx* ctx) {
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, 4 * sizeof(unsigned int), ctx->stream));
  return LS_OK;
}

ls_status sync_and_check(ls_ctx* ctx) {
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const unsigned int st = *reinterpret_cast<unsigned int*>(ctx->h_pinned);
  if (st & LS_DEV_TIMEOUT) return fail(ctx, LS_ETIMEOUT, "a bounded device wait gave up (pipeline stalled)");
  if (st & LS_DEV_RANK) return fail(ctx, LS_ERANK, "R has a zero or non-finite diagonal entry (rank deficient)");
  if (st & LS_DEV_NONFINITE) return fail(ctx, LS_ENONFINITE, "the iterate became non-finite");
  if (st & LS_DEV_BADSIZE) return fail(ctx, LS_ECUDA, "internal: sort scratch missing for a large bucket");
  return LS_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// argument checks -------------------------------------------------------------
ls_status check_sketch_args(ls_ctx* ctx, int64_t m, int64_t d, int zeta) {
  if (m < 1 || m > INT32_MAX) return fail(ctx, LS_EINVAL, "m = %lld out of range [1, 2^31-1]", (long long)m);
  if (d < 1 || d > INT32_MAX) return fail(ctx, LS_EINVAL, "d = %lld out of range [1, 2^31-1]", (long long)d);
  if (zeta < 1 || zeta > 32 || zeta > d)
    return fail(ctx, LS_EINVAL, "zeta = %d must satisfy 1 <= zeta <= min(d, 32)", zeta);
  return LS_OK;
}

ls_status check_A(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda) {
  if (!A) return fail(ctx, LS_EINVAL, "A is null");
  if (n < 1 || n > m) return fail(ctx, LS_EINVAL, "need 1 <= n <= m (n = %lld, m = %lld)", (long long)n, (long long)m);
  if (lda < n || (lda & 1)) return fail(ctx, LS_EINVAL, "lda = %lld must be even and >= n", (long long)lda);
  if (reinterpret_cast<uintptr_t>(A) & 15) return fail(ctx, LS_EINVAL, "A must be 16-byte aligned");
  return LS_OK;
}

constexpr int64_t kMaxN = 2048;   // fused pass keeps up to 8 columns per thread

// scratch layouts ---------------------------------------------------------------
struct SketchScratch {
  int32_t* rows; uint32_t* signs; int64_t* row_ptr; uint32_t* ent; unsigned long long* fill;
  int64_t* split;   // entry offsets of the upload pieces, d * (kMaxPieces + 1)
};
SketchScratch carve_sketch(Carve& c, int64_t m, int64_t d, int zeta) {
  SketchScratch s;
  s.rows = c.take<int32_t>((size_t)m * zeta);
  s.signs = c.take<uint32_t>((size_t)m);
  s.row_ptr = c.take<int64_t>((size_t)d + 1);
  s.ent = c.take<uint32_t>((size_t)m * zeta);
  s.fill = c.take<unsigned long long>((size_t)d);
  s.split = c.take<int64_t>((size_t)d * (kMaxPieces + 1));
  return s;
}

struct FactorScratch {
  double* part; double* w; double* Rt; double* inv_diag; double* vecs; double* est;
};
FactorScratch carve_factor(Carve& c, const ls_ctx* ctx, int64_t d, int64_t n) {
  FactorScratch f;
  f.part = c.take<double>(householder_part_doubles(ctx, d, n));
  f.w = c.take<double>(householder_w_doubles(n));
  f.Rt = c.take<double>((size_t)n * n);
  f.inv_diag = c.take<double>((size_t)n);
  f.vecs = c.take<double>(4 * (size_t)n + 64);
  f.est = c.take<double>(2);
  return f;
}

struct IterScratch {
  double* part; double* Rt; double* inv_diag; double* x_prev; double* y; double* dvec; double* work;
  double* slots; IterState* st; double* r_prev;
};
IterScratch carve_iter(Carve& c, const PassGeom& g, int64_t m, int64_t n) {
  IterScratch s;
  s.part = c.take<double>((size_t)g.grid * (n + 2));
  s.Rt = c.take<double>((size_t)n * n);
  s.inv_diag = c.take<double>((size_t)n);
  s.x_prev = c.take<double>((size_t)n);
  s.y = c.take<double>((size_t)n);
  s.dvec = c.take<double>((size_t)n);
  s.work = c.take<double>((size_t)n);
  s.slots = c.take<double>(64);
  s.st = c.take<IterState>(1);
  s.r_prev = c.take<double>((size_t)m);
  return s;
}

// Fixed-point pass (fxpass.cu): A in 55-bit fixed point, row exponents and
// the per-CTA partials.  Used by the iteration for n <= kFxMaxN.
bool use_fx_pass(int64_t n) { return n <= kFxMaxN; }

struct FxScratch {
  int2* Af; int* rexp; long long* part; int64_t ldf;
};
FxScratch carve_fx(Carve& c, const ls_ctx* ctx, int64_t m, int64_t n) {
  FxScratch f;
  f.ldf = (n + 1) & ~1LL;
  const FxGeom g = fx_geometry(ctx, n, m);
  f.Af = c.take<int2>((size_t)m * f.ldf);
  f.rexp = c.take<int>((size_t)m);
  f.part = c.take<long long>(fx_part_words(g, n));
  return f;
}

}  // namespace

// ============================================================ public API
extern "C" {

void ls_default_opts(ls_opts* o) {
  if (!o) return;
  o->gamma = 1.0;
  o->rho = 0.04;
  o->extra_iters = 3;
  o->use_stop = 1;
  o->alpha = 1.0;
  o->beta = 0.0;
}

void ls_opts_damping(ls_opts* o, int64_t n, int64_t d) {
  if (!o || n < 1 || d < 1) return;
  const double e2 = (double)n / (double)d;   // e = sqrt(n/d)
  o->alpha = (1.0 - e2) * (1.0 - e2) / (1.0 + e2);
  o->beta = 0.0;
}

void ls_opts_momentum(ls_opts* o, int64_t n, int64_t d) {
  if (!o || n < 1 || d < 1) return;
  const double e2 = (double)n / (double)d;
  o->alpha = (1.0 - e2) * (1.0 - e2);
  o->beta = e2;
}

ls_status ls_create(ls_ctx** out, int device, void* cuda_stream) {
  if (!out) return LS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LS_ECUDA;
  }
  if (device < 0 || device >= ndev) return LS_EINVAL;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return LS_ECUDA;
  if (prop.major != 10 || prop.minor != 3) return LS_ECUDA;   // built for sm_103a only
  ls_ctx* ctx = new ls_ctx();
  ctx->device = device;
  ctx->num_sms = prop.multiProcessorCount;
  if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return LS_ECUDA; }
  if (cuda_stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return LS_ECUDA; }
    ctx->own_stream = true;
  }
  if (cudaMalloc(&ctx->d_status, 16 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_misc, 16 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_pinned, 4096) != cudaSuccess) {
    ls_destroy(ctx);
    return LS_ENOMEM;
  }
  cudaMemset(ctx->d_status, 0, 16 * sizeof(unsigned int));
  for (auto& e : ctx->ev) cudaEventCreate(&e);
  *out = ctx;
  return LS_OK;
}

ls_status ls_destroy(ls_ctx* ctx) {
  if (!ctx) return LS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_misc) cudaFree(ctx->d_misc);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->fx_stream) cudaStreamDestroy(ctx->fx_stream);
  if (ctx->fx_done) cudaEventDestroy(ctx->fx_done);
  if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
  for (auto& e : ctx->piece_done) if (e) cudaEventDestroy(e);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  for (auto& e : ctx->ev) if (e) cudaEventDestroy(e);
  for (auto& e : ctx->pass_ev) if (e) cudaEventDestroy(e);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return LS_OK;
}

const char* ls_last_error(const ls_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t ls_workspace_bytes(int64_t m, int64_t n, int64_t d, int zeta) {
  if (m < 1 || n < 1 || d < 1 || zeta < 1) return 0;
  ls_ctx probe;
  probe.num_sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) probe.num_sms = p.multiProcessorCount;
  }
  cudaGetLastError();
  Carve c(nullptr);
  c.take<double>((size_t)d * (n + 1));   // B_aug
  c.take<double>((size_t)n * n);         // R
  c.take<double>((size_t)n);             // x0
  const size_t mark = c.off;
  carve_sketch(c, m, d, zeta);
  size_t sk = c.off;
  c.off = mark;
  carve_factor(c, &probe, d, n);
  size_t fa = c.off;
  c.off = mark;
  PassGeom g = pass_geometry(&probe, n, m);
  carve_iter(c, g, m, n);
  if (use_fx_pass(n)) carve_fx(c, &probe, m, n);
  size_t it = c.off;
  size_t need = std::max(sk, std::max(fa, it));
  return need;
}

ls_status ls_sketch_indices(ls_ctx* ctx, int64_t m, int64_t d, int zeta, uint64_t seed, int32_t* rows,
                            uint32_t* signs) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st = check_sketch_args(ctx, m, d, zeta);
  if (st) return st;
  if (!rows || !signs) return fail(ctx, LS_EINVAL, "rows/signs are null");
  cudaSetDevice(ctx->device);
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, launch_sketch_indices(ctx, m, d, zeta, seed, rows, signs));
  return sync_and_check(ctx);
}

static ls_status sketch_csr_impl(ls_ctx* ctx, int64_t m, int64_t d, int zeta, const int32_t* rows,
                                 const uint32_t* signs, int64_t* row_ptr, uint32_t* ent, unsigned long long* fill) {
  int maxb = 0;
  CUDA_TRY(ctx, launch_sketch_csr(ctx, m, d, zeta, rows, signs, row_ptr, ent, fill, nullptr, &maxb));
  uint32_t* scratch = nullptr;
  int P = 1;
  while (P < maxb) P <<= 1;
  if (P > sketch_sort_cap()) {
    ls_status st = ensure_aux(ctx, &ctx->aux, &ctx->aux_bytes, sizeof(uint32_t) * 2 * (size_t)m * zeta);
    if (st) return st;
    scratch = reinterpret_cast<uint32_t*>(ctx->aux);
  }
  // histogram + scan again (cheap) and then scatter + sort
  CUDA_TRY(ctx, launch_sketch_csr(ctx, m, d, zeta, rows, signs, row_ptr, ent, fill, scratch, nullptr));
  return LS_OK;
}

ls_status ls_sketch_csr(ls_ctx* ctx, int64_t m, int64_t d, int zeta, const int32_t* rows, const uint32_t* signs,
                        int64_t* row_ptr, uint32_t* ent) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st = check_sketch_args(ctx, m, d, zeta);
  if (st) return st;
  if (!rows || !signs || !row_ptr || !ent) return fail(ctx, LS_EINVAL, "null pointer argument");
  cudaSetDevice(ctx->device);
  Carve c(nullptr);
  unsigned long long* fill_probe = c.take<unsigned long long>((size_t)d);
  (void)fill_probe;
  if ((st = ensure_arena(ctx, c.off))) return st;
  Carve cc(ctx->arena);
  unsigned long long* fill = cc.take<unsigned long long>((size_t)d);
  if ((st = reset_status(ctx))) return st;
  if ((st = sketch_csr_impl(ctx, m, d, zeta, rows, signs, row_ptr, ent, fill))) return st;
  return sync_and_check(ctx);
}

// Host A uploaded in row pieces: piece i (rows bnd.r[i] .. bnd.r[i+1]) may be
// read after event ev[i].
struct UploadPieces {
  int np;
  PieceBounds bnd;
  cudaEvent_t ev[kMaxPieces];
};

// wait_A (may be null): an event after which A may be read (an upload in
// flight); the indices and the CSR, which do not read A, run before it.
static ls_status sketch_impl(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                             int64_t d, int zeta, uint64_t seed, double* B, int64_t ldb, Carve& cc,
                             cudaEvent_t wait_A = nullptr, const UploadPieces* up = nullptr) {
  SketchScratch s = carve_sketch(cc, m, d, zeta);
  CUDA_TRY(ctx, launch_sketch_indices(ctx, m, d, zeta, seed, s.rows, s.signs));
  ls_status st = sketch_csr_impl(ctx, m, d, zeta, s.rows, s.signs, s.row_ptr, s.ent, s.fill);
  if (st) return st;
  const double scale = 1.0 / std::sqrt((double)zeta);
  if (up) {
    // gather each piece of A as it lands; the running sums continue in B
    CUDA_TRY(ctx, launch_sketch_split(ctx, d, s.row_ptr, s.ent, up->np, up->bnd, s.split));
    CUDA_TRY(ctx, launch_sketch_gather_b(ctx, b, d, s.row_ptr, s.ent, scale, B + n * ldb));
    for (int i = 0; i < up->np; ++i) {
      CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, up->ev[i], 0));
      CUDA_TRY(ctx, launch_sketch_gather_piece(ctx, A, n, lda, d, s.split, up->np, i, s.ent, scale, B, ldb));
    }
    return LS_OK;
  }
  if (wait_A) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, wait_A, 0));
  CUDA_TRY(ctx, launch_sketch_apply(ctx, A, m, n, lda, b, d, s.row_ptr, s.ent, scale, B, ldb));
  return LS_OK;
}

ls_status ls_sketch(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                    int zeta, uint64_t seed, double* B, int64_t ldb) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if ((st = check_sketch_args(ctx, m, d, zeta))) return st;
  if ((st = check_A(ctx, A, m, n, lda))) return st;
  if (!b || !B) return fail(ctx, LS_EINVAL, "b/B is null");
  if (ldb < d) return fail(ctx, LS_EINVAL, "ldb < d");
  if (d < n) return fail(ctx, LS_EINVAL, "d = %lld must be >= n = %lld", (long long)d, (long long)n);
  cudaSetDevice(ctx->device);
  Carve probe(nullptr);
  carve_sketch(probe, m, d, zeta);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  if ((st = reset_status(ctx))) return st;
  if ((st = sketch_impl(ctx, A, m, n, lda, b, d, zeta, seed, B, ldb, cc))) return st;
  return sync_and_check(ctx);
}

static ls_status factor_impl(ls_ctx* ctx, double* B, int64_t d, int64_t n, int64_t ldb, double* R, int64_t ldr,
                             double* x0, uint64_t seed, Carve& cc, double* est_host) {
  FactorScratch f = carve_factor(cc, ctx, d, n);
  CUDA_TRY(ctx, launch_householder(ctx, B, d, n, ldb, f.part, f.w));
  CUDA_TRY(ctx, launch_prepare_R(ctx, B, ldb, n, R, ldr, f.Rt, f.inv_diag));
  CUDA_TRY(ctx, launch_post_factor(ctx, B, d, n, ldb, R, ldr, x0, seed, f.Rt, f.inv_diag, f.vecs, f.est));
  CUDA_TRY(ctx, cudaMemcpyAsync(reinterpret_cast<char*>(ctx->h_pinned) + 64, f.est, 2 * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
  ls_status st = sync_and_check(ctx);
  if (st) return st;
  std::memcpy(est_host, reinterpret_cast<char*>(ctx->h_pinned) + 64, 2 * sizeof(double));
  return LS_OK;
}

ls_status ls_factor(ls_ctx* ctx, double* B, int64_t d, int64_t n, int64_t ldb, double* R, int64_t ldr, double* x0,
                    uint64_t seed, ls_info* info) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  if (!B || !R || !x0) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (n < 1 || d < n) return fail(ctx, LS_EINVAL, "need 1 <= n <= d");
  if (ldb < d || ldr < n) return fail(ctx, LS_EINVAL, "ldb < d or ldr < n");
  if (n > 1000000) return fail(ctx, LS_EINVAL, "n too large");
  cudaSetDevice(ctx->device);
  ls_status st;
  Carve probe(nullptr);
  carve_factor(probe, ctx, d, n);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  if ((st = reset_status(ctx))) return st;
  double est[2];
  const long long l0 = ctx->launches;
  st = factor_impl(ctx, B, d, n, ldb, R, ldr, x0, seed, cc, est);
  if (st) return st;
  if (info) {
    std::memset(info, 0, sizeof *info);
    info->normest = est[0];
    info->condest = est[1];
    info->launches = (int)(ctx->launches - l0);
  }
  return LS_OK;
}

ls_status ls_residual_gradient(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                               const double* x, const double* r_prev, double* r_out, double* c, double* norms) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if (m < 1) return fail(ctx, LS_EINVAL, "m must be >= 1");
  if ((st = check_A(ctx, A, m, n, lda))) return st;
  if (n > kMaxN) return fail(ctx, LS_EINVAL, "n = %lld above the fused-pass limit %lld", (long long)n, (long long)kMaxN);
  if (!b || !x || !c || !norms) return fail(ctx, LS_EINVAL, "null pointer argument");
  cudaSetDevice(ctx->device);
  PassGeom g = pass_geometry(ctx, n, m);
  Carve probe(nullptr);
  probe.take<double>((size_t)g.grid * (n + 2));
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  double* part = cc.take<double>((size_t)g.grid * (n + 2));
  CUtensorMap map;
  CUDA_TRY(ctx, make_tensor_map(ctx, &map, A, m, n, lda, g));
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, launch_fused_pass(ctx, map, g, m, n, b, x, r_prev, r_out, part, nullptr));
  CUDA_TRY(ctx, launch_reduce_partials(ctx, part, g.grid, n, c, norms));
  if (!r_prev) CUDA_TRY(ctx, cudaMemsetAsync(norms + 1, 0, sizeof(double), ctx->stream));
  return sync_and_check(ctx);
}

ls_status ls_fixed_point(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, int32_t* A_fx,
                         int64_t ldf, int32_t* row_exp) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if (m < 1 || m > INT32_MAX) return fail(ctx, LS_EINVAL, "m = %lld out of range [1, 2^31-1]", (long long)m);
  if ((st = check_A(ctx, A, m, n, lda))) return st;
  if (!A_fx || !row_exp) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (ldf < n || (ldf & 1)) return fail(ctx, LS_EINVAL, "ldf = %lld must be even and >= n", (long long)ldf);
  if (reinterpret_cast<uintptr_t>(A_fx) & 15) return fail(ctx, LS_EINVAL, "A_fx must be 16-byte aligned");
  cudaSetDevice(ctx->device);
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, launch_to_fixed(ctx, A, m, n, lda, reinterpret_cast<int2*>(A_fx), ldf, row_exp));
  return sync_and_check(ctx);
}

ls_status ls_residual_gradient_fx(ls_ctx* ctx, const int32_t* A_fx, const int32_t* row_exp, int64_t m, int64_t n,
                                  int64_t ldf, const double* b, const double* x, const double* r_prev, double* r_out,
                                  double* c, double* norms) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if (m < 1 || m > INT32_MAX) return fail(ctx, LS_EINVAL, "m = %lld out of range [1, 2^31-1]", (long long)m);
  if (n < 1 || n > m) return fail(ctx, LS_EINVAL, "need 1 <= n <= m (n = %lld, m = %lld)", (long long)n, (long long)m);
  if (n > kFxMaxN) return fail(ctx, LS_EINVAL, "n = %lld above the fixed-point pass limit %lld", (long long)n,
                               (long long)kFxMaxN);
  if (!A_fx || !row_exp || !b || !x || !c || !norms) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (ldf < n || (ldf & 1)) return fail(ctx, LS_EINVAL, "ldf = %lld must be even and >= n", (long long)ldf);
  if (reinterpret_cast<uintptr_t>(A_fx) & 15) return fail(ctx, LS_EINVAL, "A_fx must be 16-byte aligned");
  cudaSetDevice(ctx->device);
  const FxGeom g = fx_geometry(ctx, n, m);
  Carve probe(nullptr);
  probe.take<long long>(fx_part_words(g, n));
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  long long* part = cc.take<long long>(fx_part_words(g, n));
  CUtensorMap map;
  CUDA_TRY(ctx, make_fx_tensor_map(ctx, &map, reinterpret_cast<const int2*>(A_fx), m, n, ldf, g));
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, launch_fx_pass(ctx, map, g, m, n, row_exp, b, x, r_prev, r_out, part, nullptr));
  CUDA_TRY(ctx, launch_fx_reduce(ctx, part, g.grid, n, c, norms, nullptr));
  if (!r_prev) CUDA_TRY(ctx, cudaMemsetAsync(norms + 1, 0, sizeof(double), ctx->stream));
  return sync_and_check(ctx);
}

ls_status ls_set_wait_limit(ls_ctx* ctx, uint64_t ns) {
  if (!ctx) return LS_EINVAL;
  ctx->wait_ns = ns ? ns : LS_WAIT_NS;
  return LS_OK;
}

ls_status ls_inject_fault(ls_ctx* ctx, int kind, int64_t arg) {
  if (!ctx) return LS_EINVAL;
  if (kind == LS_FAULT_NONE) { ctx->inject_skip_tile = -1; ctx->inject_alloc_fail = 0; return LS_OK; }
  if (kind == LS_FAULT_SKIP_TILE) {
    if (arg < 0 || arg > INT32_MAX) return fail(ctx, LS_EINVAL, "tile index out of range");
    ctx->inject_skip_tile = (int)arg;
    return LS_OK;
  }
  if (kind == LS_FAULT_ALLOC) { ctx->inject_alloc_fail = 1; return LS_OK; }
  return fail(ctx, LS_EINVAL, "unknown fault kind %d", kind);
}

ls_status ls_correct(ls_ctx* ctx, const double* R, int64_t ldr, int64_t n, const double* c, double* x, double* y_out,
                     double* d_out) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  if (!R || !c || !x) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (n < 1 || ldr < n) return fail(ctx, LS_EINVAL, "need n >= 1 and ldr >= n");
  cudaSetDevice(ctx->device);
  ls_status st;
  Carve probe(nullptr);
  probe.take<double>((size_t)n * n);
  for (int i = 0; i < 4; ++i) probe.take<double>((size_t)n);
  probe.take<double>(64);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  StepArgs a{};
  double* Rt = cc.take<double>((size_t)n * n);
  double* inv_diag = cc.take<double>((size_t)n);
  a.y = cc.take<double>((size_t)n);
  a.dvec = cc.take<double>((size_t)n);
  a.work = cc.take<double>((size_t)n);
  a.slots = cc.take<double>(64);
  a.Rt = Rt; a.R = R; a.ldr = ldr; a.inv_diag = inv_diag; a.n = (int)n;
  a.x = x; a.c_in = c; a.y_out = y_out; a.d_out = d_out; a.status = ctx->d_status;
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, launch_prepare_R(ctx, R, ldr, n, nullptr, n, Rt, inv_diag));
  CUDA_TRY(ctx, launch_correct(ctx, a));
  return sync_and_check(ctx);
}

// pre (may be null): A already in fixed point (ls_solve_ex converts it on a
// second stream while the QR runs; the caller has made ctx->stream wait).
static ls_status iterate_impl(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                              const double* R, int64_t ldr, double* x, int q, const ls_opts* opts, double normest,
                              double condest, Carve& cc, ls_info* info, const FxScratch* pre = nullptr) {
  ls_opts o;
  ls_default_opts(&o);
  if (opts) o = *opts;
  PassGeom g = pass_geometry(ctx, n, m);
  IterScratch s = carve_iter(cc, g, m, n);
  const bool fx = use_fx_pass(n);
  CUtensorMap map;
  FxScratch fs{};
  FxGeom fg{};
  if (fx) {
    // A in fixed point once per call; every pass then reads the 8-byte limbs
    fg = fx_geometry(ctx, n, m);
    if (pre) {
      fs = *pre;
    } else {
      fs = carve_fx(cc, ctx, m, n);
      CUDA_TRY(ctx, launch_to_fixed(ctx, A, m, n, lda, fs.Af, fs.ldf, fs.rexp));
    }
    CUDA_TRY(ctx, make_fx_tensor_map(ctx, &map, fs.Af, m, n, fs.ldf, fg));
  } else {
    CUDA_TRY(ctx, make_tensor_map(ctx, &map, A, m, n, lda, g));
  }
  CUDA_TRY(ctx, launch_prepare_R(ctx, R, ldr, n, nullptr, n, s.Rt, s.inv_diag));
  IterState h{};
  h.gamma = o.gamma; h.rho = o.rho; h.alpha = o.alpha; h.beta = o.beta;
  h.normest = normest; h.condest = condest;
  IterState* hs = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 256);
  *hs = h;
  CUDA_TRY(ctx, cudaMemcpyAsync(s.st, hs, sizeof(IterState), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(s.x_prev, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(s.r_prev, 0, sizeof(double) * m, ctx->stream));
  StepArgs a{};
  a.part = s.part; a.nparts = fx ? 1 : g.grid; a.Rt = s.Rt; a.R = R; a.ldr = ldr; a.inv_diag = s.inv_diag; a.n = (int)n;
  a.x = x; a.x_prev = s.x_prev; a.y = s.y; a.dvec = s.dvec; a.work = s.work; a.slots = s.slots; a.st = s.st;
  a.use_stop = o.use_stop; a.extra = o.extra_iters; a.status = ctx->d_status;
  // launch in chunks; between chunks read the done flag.  Each fused pass is
  // bracketed by two events on the launching stream (its device time).
  if ((int)ctx->pass_ev.size() < 2 * q) {
    const size_t old = ctx->pass_ev.size();
    ctx->pass_ev.resize(2 * (size_t)q);
    for (size_t i = old; i < ctx->pass_ev.size(); ++i) CUDA_TRY(ctx, cudaEventCreate(&ctx->pass_ev[i]));
  }
  const int chunk = 8;
  int launched = 0;
  IterState* hread = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 1024);
  while (launched < q) {
    const int k = std::min(chunk, q - launched);
    for (int i = 0; i < k; ++i) {
      CUDA_TRY(ctx, cudaEventRecord(ctx->pass_ev[2 * (launched + i)], ctx->stream));
      if (fx) {
        CUDA_TRY(ctx, launch_fx_pass(ctx, map, fg, m, n, fs.rexp, b, x, s.r_prev, s.r_prev, fs.part, s.st));
        CUDA_TRY(ctx, cudaEventRecord(ctx->pass_ev[2 * (launched + i) + 1], ctx->stream));
        CUDA_TRY(ctx, launch_fx_reduce(ctx, fs.part, fg.grid, n, s.part, s.part + n, s.st));
      } else {
        CUDA_TRY(ctx, launch_fused_pass(ctx, map, g, m, n, b, x, s.r_prev, s.r_prev, s.part, s.st));
        CUDA_TRY(ctx, cudaEventRecord(ctx->pass_ev[2 * (launched + i) + 1], ctx->stream));
      }
      CUDA_TRY(ctx, launch_iter_step(ctx, a));
    }
    launched += k;
    if (launched < q) {
      CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (hread->done) break;
    }
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
  ls_status st = sync_and_check(ctx);
  if (st) return st;
  const bool by_rule = hread->done && !hread->nonfinite;
  const int active = std::min(launched, by_rule ? hread->iter + 1 : hread->iter);
  float ms_pass = 0.0f;
  for (int i = 0; i < active; ++i) {
    float ms = 0.0f;
    CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->pass_ev[2 * i], ctx->pass_ev[2 * i + 1]));
    ms_pass += ms;
  }
  if (info) {
    info->iters = hread->iter;
    info->res_norm = hread->rnorm;
    info->step_norm = hread->dnorm;
    info->normest = normest;
    info->condest = condest;
    info->stop_reason = hread->done ? (hread->nonfinite ? 3 : 0) : (o.use_stop ? 1 : 2);
    info->ms_pass = ms_pass;
    info->n_pass = active;
  }
  if (hread->nonfinite) return fail(ctx, LS_ENONFINITE, "the iterate became non-finite");
  if (!hread->done && o.use_stop) return LS_ENOTCONV;
  return LS_OK;
}

// Row-sharded iteration on one device: part p holds rows m_parts[p] of A and
// b.  Each iteration runs the fixed-point pass on every part into its own
// block of per-CTA partials (what one GPU of a row-sharded run computes),
// then one reduction over all blocks in part order (the exchange: exact
// integer sums of the column partials, FP64 norms in order), then the step.
static ls_status iterate_rows_impl(ls_ctx* ctx, int np, const double* const* A_parts, const int64_t* m_parts,
                                   int64_t n, int64_t lda, const double* const* b_parts, const double* R, int64_t ldr,
                                   double* x, int q, const ls_opts* opts, double normest, double condest, Carve& cc,
                                   ls_info* info) {
  ls_opts o;
  ls_default_opts(&o);
  if (opts) o = *opts;
  int64_t mtot = 0;
  for (int p = 0; p < np; ++p) mtot += m_parts[p];
  PassGeom g0 = pass_geometry(ctx, n, mtot);
  IterScratch s = carve_iter(cc, g0, mtot, n);        // step scratch; r_prev for all rows
  std::vector<FxScratch> fs(np);
  std::vector<FxGeom> fg(np);
  std::vector<CUtensorMap> maps(np);
  std::vector<int64_t> roff(np), poff(np);
  int64_t rsum = 0, psum = 0;
  for (int p = 0; p < np; ++p) {
    fg[p] = fx_geometry(ctx, n, m_parts[p]);
    fs[p] = carve_fx(cc, ctx, m_parts[p], n);
    roff[p] = rsum;
    poff[p] = psum;
    rsum += m_parts[p];
    psum += (int64_t)fx_part_words(fg[p], n);
  }
  long long* allpart = cc.take<long long>((size_t)psum);
  int ctas = 0;
  for (int p = 0; p < np; ++p) {
    CUDA_TRY(ctx, launch_to_fixed(ctx, A_parts[p], m_parts[p], n, lda, fs[p].Af, fs[p].ldf, fs[p].rexp));
    CUDA_TRY(ctx, make_fx_tensor_map(ctx, &maps[p], fs[p].Af, m_parts[p], n, fs[p].ldf, fg[p]));
    ctas += fg[p].grid;
  }
  CUDA_TRY(ctx, launch_prepare_R(ctx, R, ldr, n, nullptr, n, s.Rt, s.inv_diag));
  IterState h{};
  h.gamma = o.gamma; h.rho = o.rho; h.alpha = o.alpha; h.beta = o.beta;
  h.normest = normest; h.condest = condest;
  IterState* hs = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 256);
  *hs = h;
  CUDA_TRY(ctx, cudaMemcpyAsync(s.st, hs, sizeof(IterState), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(s.x_prev, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(s.r_prev, 0, sizeof(double) * mtot, ctx->stream));
  StepArgs a{};
  a.part = s.part; a.nparts = 1; a.Rt = s.Rt; a.R = R; a.ldr = ldr; a.inv_diag = s.inv_diag; a.n = (int)n;
  a.x = x; a.x_prev = s.x_prev; a.y = s.y; a.dvec = s.dvec; a.work = s.work; a.slots = s.slots; a.st = s.st;
  a.use_stop = o.use_stop; a.extra = o.extra_iters; a.status = ctx->d_status;
  const int chunk = 8;
  int launched = 0;
  IterState* hread = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 1024);
  while (launched < q) {
    const int k = std::min(chunk, q - launched);
    for (int i = 0; i < k; ++i) {
      for (int p = 0; p < np; ++p)
        CUDA_TRY(ctx, launch_fx_pass(ctx, maps[p], fg[p], m_parts[p], n, fs[p].rexp, b_parts[p], x,
                                     s.r_prev + roff[p], s.r_prev + roff[p], allpart + poff[p], s.st));
      CUDA_TRY(ctx, launch_fx_reduce(ctx, allpart, ctas, n, s.part, s.part + n, s.st));
      CUDA_TRY(ctx, launch_iter_step(ctx, a));
    }
    launched += k;
    if (launched < q) {
      CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (hread->done) break;
    }
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
  ls_status st = sync_and_check(ctx);
  if (st) return st;
  if (info) {
    info->iters = hread->iter;
    info->res_norm = hread->rnorm;
    info->step_norm = hread->dnorm;
    info->normest = normest;
    info->condest = condest;
    info->stop_reason = hread->done ? (hread->nonfinite ? 3 : 0) : (o.use_stop ? 1 : 2);
  }
  if (hread->nonfinite) return fail(ctx, LS_ENONFINITE, "the iterate became non-finite");
  if (!hread->done && o.use_stop) return LS_ENOTCONV;
  return LS_OK;
}

ls_status ls_iterate_rows(ls_ctx* ctx, int nparts, const double* const* A_parts, const int64_t* m_parts, int64_t n,
                          int64_t lda, const double* const* b_parts, const double* R, int64_t ldr, double* x, int q,
                          const ls_opts* opts, ls_info* info) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if (nparts < 1 || nparts > 64 || !A_parts || !m_parts || !b_parts)
    return fail(ctx, LS_EINVAL, "need 1 <= nparts <= 64 and the part arrays");
  if (n < 1 || n > kFxMaxN) return fail(ctx, LS_EINVAL, "need 1 <= n <= %lld", (long long)kFxMaxN);
  int64_t mtot = 0;
  for (int p = 0; p < nparts; ++p) {
    if (m_parts[p] < 1 || m_parts[p] > INT32_MAX) return fail(ctx, LS_EINVAL, "part %d: m out of range", p);
    if (!A_parts[p] || !b_parts[p]) return fail(ctx, LS_EINVAL, "part %d: null pointer", p);
    if (lda < n || (lda & 1)) return fail(ctx, LS_EINVAL, "lda = %lld must be even and >= n", (long long)lda);
    mtot += m_parts[p];
  }
  if (n > mtot) return fail(ctx, LS_EINVAL, "need n <= total rows");
  if (!R || !x || !info) return fail(ctx, LS_EINVAL, "null pointer argument (info is required)");
  if (ldr < n) return fail(ctx, LS_EINVAL, "ldr < n");
  if (q < 0) return fail(ctx, LS_EINVAL, "q < 0");
  cudaSetDevice(ctx->device);
  Carve probe(nullptr);
  carve_iter(probe, pass_geometry(ctx, n, mtot), mtot, n);
  int64_t psum = 0;
  for (int p = 0; p < nparts; ++p) {
    carve_fx(probe, ctx, m_parts[p], n);
    psum += (int64_t)fx_part_words(fx_geometry(ctx, n, m_parts[p]), n);
  }
  probe.take<long long>((size_t)psum);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  if ((st = reset_status(ctx))) return st;
  const double ne = info->normest, ce = info->condest;
  const long long l0 = ctx->launches;
  st = iterate_rows_impl(ctx, nparts, A_parts, m_parts, n, lda, b_parts, R, ldr, x, q, opts, ne, ce, cc, info);
  info->launches = (int)(ctx->launches - l0);
  return st;
}

ls_status ls_iterate(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                     const double* R, int64_t ldr, double* x, int q, const ls_opts* opts, ls_info* info) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if (m < 1) return fail(ctx, LS_EINVAL, "m must be >= 1");
  if ((st = check_A(ctx, A, m, n, lda))) return st;
  if (n > kMaxN) return fail(ctx, LS_EINVAL, "n = %lld above the fused-pass limit %lld", (long long)n, (long long)kMaxN);
  if (!b || !R || !x || !info) return fail(ctx, LS_EINVAL, "null pointer argument (info is required)");
  if (ldr < n) return fail(ctx, LS_EINVAL, "ldr < n");
  if (q < 0) return fail(ctx, LS_EINVAL, "q < 0");
  cudaSetDevice(ctx->device);
  PassGeom g = pass_geometry(ctx, n, m);
  Carve probe(nullptr);
  carve_iter(probe, g, m, n);
  if (use_fx_pass(n)) carve_fx(probe, ctx, m, n);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  if ((st = reset_status(ctx))) return st;
  const double ne = info->normest, ce = info->condest;
  const long long l0 = ctx->launches;
  st = iterate_impl(ctx, A, m, n, lda, b, R, ldr, x, q, opts, ne, ce, cc, info);
  info->launches = (int)(ctx->launches - l0);
  return st;
}

}  // extern "C"

// The batched solve; mixed = FP32 sketch and QR (one CTA per problem), FP64
// iteration.
static ls_status solve_batched_impl(ls_ctx* ctx, const ls_problem* probs, int np, int zeta, int q,
                                    const ls_opts* opts, ls_info* infos, bool mixed) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  if (np < 0 || (np > 0 && !probs)) return fail(ctx, LS_EINVAL, "invalid problem array");
  if (np == 0) return LS_OK;
  if (zeta < 1 || zeta > 32) return fail(ctx, LS_EINVAL, "zeta = %d must be in [1, 32]", zeta);
  if (q <= 0) q = 100;
  ls_opts o;
  ls_default_opts(&o);
  if (opts) o = *opts;
  int64_t msum = 0, dsum = 0;
  for (int p = 0; p < np; ++p) {
    const ls_problem& pr = probs[p];
    ls_status st;
    if (!pr.b || !pr.x) return fail(ctx, LS_EINVAL, "problem %d: null b or x", p);
    if ((st = check_A(ctx, pr.A, pr.m, pr.n, pr.lda))) {
      const std::string why = ctx->err;
      return fail(ctx, st, "problem %d: %s", p, why.c_str());
    }
    if (pr.d < pr.n || pr.d > INT32_MAX || zeta > pr.d)
      return fail(ctx, LS_EINVAL, "problem %d: need n <= d, zeta <= d", p);
    if (pr.n > 1024) return fail(ctx, LS_EINVAL, "problem %d: n = %lld above the batched limit 1024", p, (long long)pr.n);
    msum += pr.m;
    dsum += pr.d;
  }
  if (msum > INT32_MAX || dsum > INT32_MAX) return fail(ctx, LS_EINVAL, "sum of m or of d reaches 2^31");
  cudaSetDevice(ctx->device);
  std::vector<char> hP(bprob_bytes() * (size_t)np);
  BProb* hp = reinterpret_cast<BProb*>(hP.data());
  BatchPlan pl;
  batch_plan(probs, np, hp, pl, ctx->tune);
  std::vector<int64_t> hoffs(3 * (size_t)np);
  batch_offsets(hp, np, hoffs.data(), hoffs.data() + np, hoffs.data() + 2 * np);
  std::vector<int> horder((size_t)np);
  const int csize = mixed ? 0 : b_qr_cluster_size(ctx);
  const int nsmall = batch_order(hp, np, horder.data(), csize > 0);
  // mixed: the FP64 stage reads a compact n x (n+1) copy of the factored top rows
  std::vector<char> hP64;
  int64_t ctotal = 0;
  if (mixed) {
    hP64.assign(hP.begin(), hP.end());
    BProb* h64 = reinterpret_cast<BProb*>(hP64.data());
    for (int p = 0; p < np; ++p) {
      h64[p].d = h64[p].n;
      h64[p].boff = ctotal;
      ctotal += h64[p].n * (h64[p].n + 1);
    }
  }

  BProb* dP64 = nullptr;
  float* B32 = nullptr;
  double* Bc = nullptr;
  auto carve_all = [&](Carve& c, BProb** dP, int64_t** doff3, SketchScratch* sk, BPools* pools, int** dorder,
                       int** alist, int64_t** aoff, int64_t** cnt) {
    *dP = reinterpret_cast<BProb*>(c.take<char>(bprob_bytes() * (size_t)np));
    if (mixed) {
      dP64 = reinterpret_cast<BProb*>(c.take<char>(bprob_bytes() * (size_t)np));
      B32 = c.take<float>((size_t)pl.btotal);
      Bc = c.take<double>((size_t)ctotal);
    }
    *doff3 = c.take<int64_t>(3 * (size_t)np);
    *sk = carve_sketch(c, pl.mtotal, pl.dtotal, zeta);
    pools->B = mixed ? nullptr : c.take<double>((size_t)pl.btotal);
    pools->R = c.take<double>((size_t)pl.rtotal);
    pools->V = c.take<double>((size_t)pl.vtotal);
    pools->done_rec = nullptr;
    pools->done_count = nullptr;
    pools->slots = c.take<double>(64 * (size_t)np);
    pools->est = c.take<double>(2 * (size_t)np);
    pools->part = c.take<double>((size_t)pl.ptotal);
    pools->r_prev = c.take<double>((size_t)pl.mtotal);
    pools->st = c.take<IterState>((size_t)np);
    pools->pstatus = c.take<unsigned int>((size_t)np);
    *dorder = c.take<int>((size_t)np);
    *alist = c.take<int>((size_t)np);
    *aoff = c.take<int64_t>((size_t)np);
    *cnt = c.take<int64_t>(4);
  };
  BProb* dP; int64_t* doff3; SketchScratch sk; BPools pools; int* dorder; int* alist; int64_t* aoff; int64_t* cnt;
  Carve probe(nullptr);
  carve_all(probe, &dP, &doff3, &sk, &pools, &dorder, &alist, &aoff, &cnt);
  ls_status st;
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  carve_all(cc, &dP, &doff3, &sk, &pools, &dorder, &alist, &aoff, &cnt);
  if ((st = reset_status(ctx))) return st;
  CUDA_TRY(ctx, cudaMemcpyAsync(dP, hp, bprob_bytes() * (size_t)np, cudaMemcpyHostToDevice, ctx->stream));
  if (mixed)
    CUDA_TRY(ctx, cudaMemcpyAsync(dP64, hP64.data(), bprob_bytes() * (size_t)np, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(doff3, hoffs.data(), sizeof(int64_t) * 3 * np, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(dorder, horder.data(), sizeof(int) * np, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(pools.pstatus, 0, sizeof(unsigned int) * np, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(pools.r_prev, 0, sizeof(double) * pl.mtotal, ctx->stream));
  const long long l0 = ctx->launches;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
  // sketch
  CUDA_TRY(ctx, launch_b_sketch_indices(ctx, dP, doff3, pl, zeta, sk.rows, sk.signs));
  // one CTA per problem builds small problems' CSR fastest; a problem with
  // millions of entries would keep one CTA busy for a long time, so batches
  // holding one use the device-wide counting sort
  if (b_csr_fits(pl) && pl.max_m * zeta <= b_csr_global_entries()) {
    // buckets above 1024 entries are sorted in global scratch; expect them
    // only when some problem's mean bucket exceeds ~600
    uint32_t* scratch = nullptr;
    if (pl.max_fill * zeta > 600.0) {
      if ((st = ensure_aux(ctx, &ctx->aux, &ctx->aux_bytes, sizeof(uint32_t) * 2 * (size_t)pl.mtotal * zeta)))
        return st;
      scratch = reinterpret_cast<uint32_t*>(ctx->aux);
    }
    CUDA_TRY(ctx, launch_b_csr(ctx, dP, pl, zeta, sk.rows, sk.signs, sk.row_ptr, sk.ent, scratch));
  } else if ((st = sketch_csr_impl(ctx, pl.mtotal, pl.dtotal, zeta, sk.rows, sk.signs, sk.row_ptr, sk.ent,
                                   sk.fill))) {
    return st;
  }
  const double scale = 1.0 / std::sqrt((double)zeta);
  if (mixed)
    CUDA_TRY(ctx, launch_b_gather32(ctx, dP, doff3 + 2 * np, pl, sk.row_ptr, sk.ent, scale, B32));
  else
    CUDA_TRY(ctx, launch_b_gather(ctx, dP, doff3 + 2 * np, pl, sk.row_ptr, sk.ent, scale, pools.B));
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
  for (int p = 0; p < np; ++p)
    if (probs[p].B_out) {
      const size_t cntB = (size_t)probs[p].d * (probs[p].n + 1);
      if (mixed)
        CUDA_TRY(ctx, launch_widen(ctx, B32 + batch_boff(hp, p), probs[p].B_out, (int64_t)cntB));
      else
        CUDA_TRY(ctx, cudaMemcpyAsync(probs[p].B_out, pools.B + batch_boff(hp, p), sizeof(double) * cntB,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
  // factor
  if (mixed)
    CUDA_TRY(ctx, launch_b_factor_mixed(ctx, dP, dP64, dorder, np, B32, Bc, pools));
  else
    CUDA_TRY(ctx, launch_b_factor2(ctx, dP, dorder, nsmall, dorder + nsmall, np - nsmall, csize, np, nullptr, pools));
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
  for (int p = 0; p < np; ++p)
    if (probs[p].R_out)
      CUDA_TRY(ctx, cudaMemcpyAsync(probs[p].R_out, pools.R + batch_roff(hp, p),
                                    sizeof(double) * (size_t)probs[p].n * probs[p].n, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
  // iterate
  CUDA_TRY(ctx, launch_b_iter_init(ctx, dP, np, nullptr, pools, o.gamma, o.rho, o.alpha, o.beta));
  CUDA_TRY(ctx, launch_b_compact(ctx, dP, np, pools, alist, aoff, cnt));
  int64_t* hcnt = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(ctx->h_pinned) + 2048);
  for (int i = 0; i < q; ++i) {
    CUDA_TRY(ctx, launch_b_pass(ctx, dP, alist, aoff, cnt, pl.max_n, pl.cap, pl.ttotal, pools));
    CUDA_TRY(ctx, launch_b_step(ctx, dP, alist, cnt, np, pools, o.use_stop, o.extra_iters, q));
    CUDA_TRY(ctx, launch_b_compact(ctx, dP, np, pools, alist, aoff, cnt));
    if ((i & 7) == 7 && i + 1 < q) {
      CUDA_TRY(ctx, cudaMemcpyAsync(hcnt, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (*hcnt == 0) break;
    }
  }
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[3], ctx->stream));
  std::vector<IterState> hst((size_t)np);
  std::vector<double> hest(2 * (size_t)np);
  CUDA_TRY(ctx, cudaMemcpyAsync(hst.data(), pools.st, sizeof(IterState) * np, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(hest.data(), pools.est, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, ctx->stream));
  if ((st = sync_and_check(ctx))) return st;
  if (infos) {
    float ms[3] = {0, 0, 0};
    cudaEventElapsedTime(&ms[0], ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&ms[1], ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&ms[2], ctx->ev[2], ctx->ev[3]);
    for (int p = 0; p < np; ++p) {
      ls_info& in = infos[p];
      std::memset(&in, 0, sizeof in);
      const IterState& s = hst[p];
      in.iters = s.iter;
      in.stop_reason = s.done ? s.stop_reason : (o.use_stop ? 1 : 2);
      in.res_norm = s.rnorm;
      in.step_norm = s.dnorm;
      in.normest = hest[2 * p];
      in.condest = hest[2 * p + 1];
      in.ms_sketch = ms[0]; in.ms_factor = ms[1]; in.ms_iterate = ms[2];
      in.launches = (int)(ctx->launches - l0);
    }
  }
  return LS_OK;
}

extern "C" {

ls_status ls_solve_batched(ls_ctx* ctx, const ls_problem* probs, int np, int zeta, int q, const ls_opts* opts,
                           ls_info* infos) {
  return solve_batched_impl(ctx, probs, np, zeta, q, opts, infos, false);
}

// Time `reps` passes (after one warm-up) over the problems `sub` with pass
// table t; *ms = the average.  The pass reads A and b and writes only
// scratch (x = 0 of its own).
static ls_status time_pass(ls_ctx* ctx, const std::vector<ls_problem>& sub, const PassTune& t, int reps, float* ms) {
  const int ns = (int)sub.size();
  std::vector<char> hP(bprob_bytes() * (size_t)ns);
  BProb* hp = reinterpret_cast<BProb*>(hP.data());
  BatchPlan pl;
  batch_plan(sub.data(), ns, hp, pl, t);
  auto carve_t = [&](Carve& c, BProb** dP, BPools* pools, double** xs, int** alist, int64_t** aoff, int64_t** cnt) {
    *dP = reinterpret_cast<BProb*>(c.take<char>(bprob_bytes() * (size_t)ns));
    *pools = BPools{};
    pools->part = c.take<double>((size_t)pl.ptotal);
    pools->r_prev = c.take<double>((size_t)pl.mtotal);
    pools->st = c.take<IterState>((size_t)ns);
    *xs = c.take<double>((size_t)pl.vtotal);
    *alist = c.take<int>((size_t)ns);
    *aoff = c.take<int64_t>((size_t)ns);
    *cnt = c.take<int64_t>(4);
  };
  BProb* dP; BPools pools; double* xs; int* alist; int64_t* aoff; int64_t* cnt;
  Carve probe(nullptr);
  carve_t(probe, &dP, &pools, &xs, &alist, &aoff, &cnt);
  ls_status st;
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  carve_t(cc, &dP, &pools, &xs, &alist, &aoff, &cnt);
  int64_t xo = 0;
  for (int i = 0; i < ns; ++i) {
    hp[i].x = xs + xo;
    xo += hp[i].n;
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(dP, hp, bprob_bytes() * (size_t)ns, cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(xs, 0, sizeof(double) * (size_t)pl.vtotal, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(pools.r_prev, 0, sizeof(double) * (size_t)pl.mtotal, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(pools.st, 0, sizeof(IterState) * (size_t)ns, ctx->stream));
  CUDA_TRY(ctx, launch_b_compact(ctx, dP, ns, pools, alist, aoff, cnt));
  CUDA_TRY(ctx, launch_b_pass(ctx, dP, alist, aoff, cnt, pl.max_n, pl.cap, pl.ttotal, pools));   // warm
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
  for (int r = 0; r < reps; ++r) {
    CUDA_TRY(ctx, launch_b_compact(ctx, dP, ns, pools, alist, aoff, cnt));
    CUDA_TRY(ctx, launch_b_pass(ctx, dP, alist, aoff, cnt, pl.max_n, pl.cap, pl.ttotal, pools));
  }
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
  if ((st = sync_and_check(ctx))) return st;
  float t_ms = 0.0f;
  cudaEventElapsedTime(&t_ms, ctx->ev[0], ctx->ev[1]);
  *ms = t_ms / (float)reps;
  return LS_OK;
}

ls_status ls_tune_batched(ls_ctx* ctx, const ls_problem* probs, int np, int reps, char* report, size_t report_len) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  if (np < 1 || !probs) return fail(ctx, LS_EINVAL, "invalid problem array");
  if (reps < 1) reps = 3;
  for (int p = 0; p < np; ++p) {
    ls_status st;
    if (!probs[p].b) return fail(ctx, LS_EINVAL, "problem %d: null b", p);
    if ((st = check_A(ctx, probs[p].A, probs[p].m, probs[p].n, probs[p].lda))) return st;
    if (probs[p].n > 1024) return fail(ctx, LS_EINVAL, "problem %d: n above 1024", p);
  }
  cudaSetDevice(ctx->device);
  // a sample with up to 64 problems of every class present: the launch-wide
  // buffer size couples the classes, so candidates are timed on the mix
  std::vector<int> per(kTuneBuckets, 0);
  std::vector<ls_problem> sub;
  for (int p = 0; p < np; ++p) {
    const int b = tune_bucket(probs[p].n);
    if (per[b] < 64) { sub.push_back(probs[p]); ++per[b]; }
  }
  static const int kTiles[] = {1536, 2560, 3840, 6144};
  static const int kItems[] = {64, 128, 256};
  PassTune table = ctx->tune;
  float best = 0.0f;
  ls_status st;
  if ((st = time_pass(ctx, sub, table, reps, &best))) return st;
  const float start = best;
  std::string rep;
  // one sweep of coordinate descent over the classes present
  for (int bkt = 0; bkt < kTuneBuckets; ++bkt) {
    if (per[bkt] == 0) continue;
    for (int tile : kTiles) {
      for (int items : kItems) {
        if (tile == table.tile[bkt] && items == table.item_rows[bkt]) continue;
        PassTune t = table;
        t.tile[bkt] = tile;
        t.item_rows[bkt] = items;
        float ms = 0.0f;
        if ((st = time_pass(ctx, sub, t, reps, &ms))) return st;
        if (ms < 0.99f * best) { best = ms; table = t; }
      }
    }
    table.tuned[bkt] = 1;
    char line[160];
    snprintf(line, sizeof line, "n<%d: tile %d doubles, %d rows per item\n", 32 << bkt, table.tile[bkt],
             table.item_rows[bkt]);
    rep += line;
  }
  char tail[160];
  snprintf(tail, sizeof tail, "pass over the %d-problem sample: %.3f ms -> %.3f ms\n", (int)sub.size(), start, best);
  rep += tail;
  ctx->tune = table;
  if (report && report_len) {
    std::strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = 0;
  }
  return LS_OK;
}

ls_status ls_reset_tuning(ls_ctx* ctx) {
  if (!ctx) return LS_EINVAL;
  ctx->tune = default_tune();
  return LS_OK;
}

ls_status ls_solve_batched_mixed(ls_ctx* ctx, const ls_problem* probs, int np, int zeta, int q, const ls_opts* opts,
                                 ls_info* infos) {
  return solve_batched_impl(ctx, probs, np, zeta, q, opts, infos, true);
}

ls_status ls_sketch_sparse(ls_ctx* ctx, const int64_t* row_ptr, const int32_t* col, const double* val, int64_t m,
                           int64_t n, const double* b, int64_t d, int zeta, uint64_t seed, double* B, int64_t ldb) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if ((st = check_sketch_args(ctx, m, d, zeta))) return st;
  if (!row_ptr || !col || !val || !b || !B) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (n < 1 || n > kMaxN) return fail(ctx, LS_EINVAL, "need 1 <= n <= %lld", (long long)kMaxN);
  if (ldb < d) return fail(ctx, LS_EINVAL, "ldb < d");
  cudaSetDevice(ctx->device);
  Carve probe(nullptr);
  carve_sketch(probe, m, d, zeta);
  if ((st = ensure_arena(ctx, probe.off))) return st;
  Carve cc(ctx->arena);
  if ((st = reset_status(ctx))) return st;
  SketchScratch sk = carve_sketch(cc, m, d, zeta);
  CUDA_TRY(ctx, launch_sketch_indices(ctx, m, d, zeta, seed, sk.rows, sk.signs));
  if ((st = sketch_csr_impl(ctx, m, d, zeta, sk.rows, sk.signs, sk.row_ptr, sk.ent, sk.fill))) return st;
  CUDA_TRY(ctx, launch_sp_gather(ctx, d, sk.row_ptr, sk.ent, row_ptr, col, val, b, n, 1.0 / std::sqrt((double)zeta),
                                 B, ldb));
  return sync_and_check(ctx);
}

ls_status ls_solve_sparse(ls_ctx* ctx, const int64_t* row_ptr, const int32_t* col, const double* val, int64_t m,
                          int64_t n, int64_t nnz, const double* b, int64_t d, int zeta, int q, uint64_t seed,
                          const ls_opts* opts, double* x, ls_info* info) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if ((st = check_sketch_args(ctx, m, d, zeta))) return st;
  if (!row_ptr || !col || !val || !b || !x) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (n < 1 || n > m) return fail(ctx, LS_EINVAL, "need 1 <= n <= m");
  if (n > kMaxN) return fail(ctx, LS_EINVAL, "n = %lld above the limit %lld", (long long)n, (long long)kMaxN);
  if (d < n) return fail(ctx, LS_EINVAL, "d must be >= n");
  if (nnz < 1 || nnz > INT32_MAX) return fail(ctx, LS_EINVAL, "nnz out of range");
  if (q <= 0) q = 100;
  ls_opts o;
  ls_default_opts(&o);
  if (opts) o = *opts;
  cudaSetDevice(ctx->device);
  const int64_t nb = sp_blocks(m);
  const int g = sp_residual_grid(ctx), segs = sp_segments(ctx, n);
  auto carve = [&](Carve& c, double** B, double** R, int32_t** cnt, int64_t** total, int64_t** col_ptr,
                   int32_t** crow, double** cval, double** norms_part, double** cpart, double** out) {
    *B = c.take<double>((size_t)d * (n + 1));
    *R = c.take<double>((size_t)n * n);
    *cnt = c.take<int32_t>((size_t)nb * n);
    *total = c.take<int64_t>((size_t)n);
    *col_ptr = c.take<int64_t>((size_t)n + 1);
    *crow = c.take<int32_t>((size_t)nnz);
    *cval = c.take<double>((size_t)nnz);
    *norms_part = c.take<double>(2 * (size_t)g);
    *cpart = c.take<double>((size_t)segs * n);
    *out = c.take<double>((size_t)n + 2);
  };
  double *B, *R, *cval, *norms_part, *cpart, *outp;
  int32_t *cnt, *crow;
  int64_t *total, *col_ptr;
  Carve probe(nullptr);
  carve(probe, &B, &R, &cnt, &total, &col_ptr, &crow, &cval, &norms_part, &cpart, &outp);
  const size_t mark = probe.off;
  carve_sketch(probe, m, d, zeta);
  size_t need = probe.off;
  probe.off = mark;
  carve_factor(probe, ctx, d, n);
  need = std::max(need, probe.off);
  probe.off = mark;
  PassGeom pg1{};
  pg1.grid = 1;
  carve_iter(probe, pg1, m, n);
  need = std::max(need, probe.off);
  if ((st = ensure_arena(ctx, need))) return st;
  Carve cc(ctx->arena);
  carve(cc, &B, &R, &cnt, &total, &col_ptr, &crow, &cval, &norms_part, &cpart, &outp);
  const size_t mark2 = cc.off;
  if ((st = reset_status(ctx))) return st;
  const long long l0 = ctx->launches;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
  {  // sketch: indices, CSR of S, sparse gather-add
    SketchScratch sk = carve_sketch(cc, m, d, zeta);
    CUDA_TRY(ctx, launch_sketch_indices(ctx, m, d, zeta, seed, sk.rows, sk.signs));
    if ((st = sketch_csr_impl(ctx, m, d, zeta, sk.rows, sk.signs, sk.row_ptr, sk.ent, sk.fill))) return st;
    CUDA_TRY(ctx, launch_sp_gather(ctx, d, sk.row_ptr, sk.ent, row_ptr, col, val, b, n,
                                   1.0 / std::sqrt((double)zeta), B, d));
  }
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
  cc.off = mark2;
  double est[2];
  if ((st = factor_impl(ctx, B, d, n, d, R, n, x, seed, cc, est))) return st;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
  cc.off = mark2;
  // CSC copy of A for A^T r, then the iteration
  CUDA_TRY(ctx, launch_sp_csc(ctx, m, n, row_ptr, col, val, cnt, total, col_ptr, crow, cval));
  IterScratch s = carve_iter(cc, pg1, m, n);
  CUDA_TRY(ctx, launch_prepare_R(ctx, R, n, n, nullptr, n, s.Rt, s.inv_diag));
  IterState h{};
  h.gamma = o.gamma; h.rho = o.rho; h.alpha = o.alpha; h.beta = o.beta;
  h.normest = est[0]; h.condest = est[1];
  IterState* hs = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 256);
  *hs = h;
  CUDA_TRY(ctx, cudaMemcpyAsync(s.st, hs, sizeof(IterState), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(s.x_prev, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(s.r_prev, 0, sizeof(double) * m, ctx->stream));
  StepArgs a{};
  a.part = outp; a.nparts = 1; a.Rt = s.Rt; a.R = R; a.ldr = n; a.inv_diag = s.inv_diag; a.n = (int)n;
  a.x = x; a.x_prev = s.x_prev; a.y = s.y; a.dvec = s.dvec; a.work = s.work; a.slots = s.slots; a.st = s.st;
  a.use_stop = o.use_stop; a.extra = o.extra_iters; a.status = ctx->d_status;
  IterState* hread = reinterpret_cast<IterState*>(reinterpret_cast<char*>(ctx->h_pinned) + 1024);
  int launched = 0;
  while (launched < q) {
    const int k = std::min(8, q - launched);
    for (int i = 0; i < k; ++i) {
      CUDA_TRY(ctx, launch_sp_pass(ctx, m, n, row_ptr, col, val, b, x, s.r_prev, col_ptr, crow, cval, norms_part,
                                   cpart, outp, s.st));
      CUDA_TRY(ctx, launch_iter_step(ctx, a));
    }
    launched += k;
    if (launched < q) {
      CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (hread->done) break;
    }
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(hread, s.st, sizeof(IterState), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[3], ctx->stream));
  if ((st = sync_and_check(ctx))) return st;
  if (info) {
    std::memset(info, 0, sizeof *info);
    info->iters = hread->iter;
    info->res_norm = hread->rnorm;
    info->step_norm = hread->dnorm;
    info->normest = est[0];
    info->condest = est[1];
    info->stop_reason = hread->done ? (hread->nonfinite ? 3 : 0) : (o.use_stop ? 1 : 2);
    cudaEventElapsedTime(&info->ms_sketch, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&info->ms_factor, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&info->ms_iterate, ctx->ev[2], ctx->ev[3]);
    info->launches = (int)(ctx->launches - l0);
  }
  if (hread->nonfinite) return fail(ctx, LS_ENONFINITE, "the iterate became non-finite");
  if (!hread->done && o.use_stop) return LS_ENOTCONV;
  return LS_OK;
}

ls_status ls_solve(ls_ctx* ctx, const double* A, const double* b, int64_t m, int64_t n, int64_t lda, int64_t d,
                   int zeta, int q, uint64_t seed, double* x, ls_info* info) {
  return ls_solve_ex(ctx, A, b, m, n, lda, d, zeta, q, seed, nullptr, x, info);
}

ls_status ls_solve_ex(ls_ctx* ctx, const double* A, const double* b, int64_t m, int64_t n, int64_t lda, int64_t d,
                      int zeta, int q, uint64_t seed, const ls_opts* opts, double* x, ls_info* info) {
  if (!ctx) return LS_EINVAL;
  ctx->err.clear();
  ls_status st;
  if ((st = check_sketch_args(ctx, m, d, zeta))) return st;
  if (!A || !b || !x) return fail(ctx, LS_EINVAL, "null pointer argument");
  if (n < 1 || n > m) return fail(ctx, LS_EINVAL, "need 1 <= n <= m");
  if (lda < n || (lda & 1)) return fail(ctx, LS_EINVAL, "lda must be even and >= n");
  if (d < n) return fail(ctx, LS_EINVAL, "d must be >= n");
  if (n > kMaxN) return fail(ctx, LS_EINVAL, "n = %lld above the fused-pass limit %lld", (long long)n, (long long)kMaxN);
  if (q <= 0) q = 100;
  cudaSetDevice(ctx->device);
  const bool dA = is_device_ptr(A), db = is_device_ptr(b), dx = is_device_ptr(x);
  // staging for host arrays
  size_t stage = 0;
  if (!dA) stage += align256(sizeof(double) * (size_t)m * lda);
  if (!db) stage += align256(sizeof(double) * (size_t)m);
  if (!dx) stage += align256(sizeof(double) * (size_t)n);
  if (stage && (st = ensure_stage(ctx, stage))) return st;
  if (dA && (reinterpret_cast<uintptr_t>(A) & 15)) return fail(ctx, LS_EINVAL, "A must be 16-byte aligned");
  Carve sc(ctx->stage);
  const double* Ad = A;
  const double* bd = b;
  double* xd = x;
  // b first: a copy queued behind the 16 GB of A in the copy engine would
  // hold the stream (and the sketch's indices and CSR) until A has landed
  if (!db) {
    double* p = sc.take<double>((size_t)m);
    CUDA_TRY(ctx, cudaMemcpyAsync(p, b, sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
    bd = p;
  }
  cudaEvent_t wait_A = nullptr;
  UploadPieces pieces{};
  if (!dA) {
    // upload A on the copy stream in a few large pieces (one 16 GB copy
    // measured ~30% slower than four), overlapping the sketch's indices and
    // CSR; the gather takes each piece as it lands
    if (!ctx->copy_stream) {
      CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming));
      for (auto& e : ctx->piece_done) CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    double* p = sc.take<double>((size_t)m * lda);
    CUDA_TRY(ctx, cudaEventRecord(ctx->copy_done, ctx->stream));      // after earlier work on the stream
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_done, 0));
    const int64_t rows = (m + kMaxPieces - 1) / kMaxPieces;
    pieces.np = 0;
    for (int64_t r0 = 0; r0 < m; r0 += rows) {
      const int64_t nr = std::min(rows, m - r0);
      CUDA_TRY(ctx, cudaMemcpyAsync(p + r0 * lda, A + r0 * lda, sizeof(double) * (size_t)nr * lda,
                                    cudaMemcpyHostToDevice, ctx->copy_stream));
      CUDA_TRY(ctx, cudaEventRecord(ctx->piece_done[pieces.np], ctx->copy_stream));
      pieces.bnd.r[pieces.np] = r0;
      pieces.ev[pieces.np] = ctx->piece_done[pieces.np];
      ++pieces.np;
    }
    pieces.bnd.r[pieces.np] = m;
    CUDA_TRY(ctx, cudaEventRecord(ctx->copy_done, ctx->copy_stream));
    wait_A = ctx->copy_done;
    Ad = p;
  }
  if (!dx) xd = sc.take<double>((size_t)n);

  // arena: B_aug, R, the fixed-point A (n <= 1024) | max(sketch, factor,
  // iterate) scratch
  const bool prefx = use_fx_pass(n);
  Carve probe(nullptr);
  probe.take<double>((size_t)d * (n + 1));
  probe.take<double>((size_t)n * n);
  if (prefx) carve_fx(probe, ctx, m, n);
  const size_t mark = probe.off;
  carve_sketch(probe, m, d, zeta);
  size_t need = probe.off;
  probe.off = mark;
  carve_factor(probe, ctx, d, n);
  need = std::max(need, probe.off);
  probe.off = mark;
  PassGeom g = pass_geometry(ctx, n, m);
  carve_iter(probe, g, m, n);
  need = std::max(need, probe.off);
  if ((st = ensure_arena(ctx, need))) return st;
  Carve cc(ctx->arena);
  double* B = cc.take<double>((size_t)d * (n + 1));
  double* R = cc.take<double>((size_t)n * n);
  FxScratch pre{};
  if (prefx) pre = carve_fx(cc, ctx, m, n);
  const size_t mark2 = cc.off;
  if ((st = reset_status(ctx))) return st;

  const long long l0 = ctx->launches;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
  if ((st = sketch_impl(ctx, Ad, m, n, lda, bd, d, zeta, seed, B, d, cc, wait_A, dA ? nullptr : &pieces)))
    return st;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
  if (prefx) {
    // A to fixed point on a second stream, overlapping the QR of the sketch
    // (the QR is bound by the FP64 unit, the conversion by memory and the
    // integer units); the iteration waits for it
    if (!ctx->fx_stream) {
      CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->fx_stream, cudaStreamNonBlocking));
      CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->fx_done, cudaEventDisableTiming));
    }
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->fx_stream, ctx->ev[1], 0));
    if (wait_A) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->fx_stream, wait_A, 0));
    cudaStream_t main = ctx->stream;
    ctx->stream = ctx->fx_stream;
    const cudaError_t ce = launch_to_fixed(ctx, Ad, m, n, lda, pre.Af, pre.ldf, pre.rexp);
    ctx->stream = main;
    CUDA_TRY(ctx, ce);
    CUDA_TRY(ctx, cudaEventRecord(ctx->fx_done, ctx->fx_stream));
  }
  cc.off = mark2;
  double est[2];
  if ((st = factor_impl(ctx, B, d, n, d, R, n, xd, seed, cc, est))) return st;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], ctx->stream));
  cc.off = mark2;
  ls_info local{};
  if (prefx) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->fx_done, 0));
  ls_status it = iterate_impl(ctx, Ad, m, n, lda, bd, R, n, xd, q, opts, est[0], est[1], cc, &local,
                              prefx ? &pre : nullptr);
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[3], ctx->stream));
  if (it != LS_OK && it != LS_ENOTCONV) return it;
  if (!dx) CUDA_TRY(ctx, cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (info) {
    *info = local;
    cudaEventElapsedTime(&info->ms_sketch, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&info->ms_factor, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&info->ms_iterate, ctx->ev[2], ctx->ev[3]);
    info->launches = (int)(ctx->launches - l0);
  }
  return it;
}

}  // extern "C"
