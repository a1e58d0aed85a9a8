// server.cu -- continuous batching: least-squares requests arrive at any time,
// are admitted while they fit an HBM budget, and every in-flight request
// advances by one iteration of Algorithm 2 per server step.
//
// The server reuses the batched kernels (batched.cu) on a fixed table of slots:
//  * admission, on a stream of its own so that it overlaps the iteration of
//    the requests already in flight: the admitted requests are sketched as
//    one batch (sparse-sign indices, per-problem CSR, gather-add into their
//    slots' B), factored (one CTA per request, blocked Householder QR) and
//    started (x0, normest, condest, iteration state), all addressed through
//    the slot table; a request joins the iteration once its state is
//    published (one admission batch in flight at a time);
//  * step: one captured CUDA graph -- list the iterating slots, the fused
//    residual/gradient pass over their row tiles, the per-slot solves, update
//    and stopping rule -- replayed every step; finished slots append a record
//    to a device completion queue that the host drains after the step;
//  * memory: each request's workspace (sketch, R and R^T, eight n-vectors,
//    pass partials, r_prev) is one region of a device arena handed out by a
//    first-fit allocator with coalescing; admission also counts the request's
//    own A, b and x against the budget, since they stay resident while the
//    request is in flight.
// Requests never interact: each one's sketch, factor and iteration use only
// its own data in a fixed order, so a result is bit-identical whether the
// request ran alone or among others.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "ls_internal.cuh"

using namespace lsk;

namespace lsk {
int64_t b_csr_max_d();
}  // namespace lsk

namespace {

// First-fit allocator over [0, size) in bytes, blocks aligned to 256 bytes.
class FirstFit {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }


struct Layout {   // byte offsets within a request's workspace region
  size_t B, R, V, part, rprev, total;
};

Layout request_layout(int64_t m, int64_t n, int64_t d, int items) {
  Layout L;
  L.B = 0;
  L.R = L.B + al256(sizeof(double) * (size_t)d * (n + 1));
  L.V = L.R + al256(sizeof(double) * 2 * (size_t)n * n);
  L.part = L.V + al256(sizeof(double) * 8 * (size_t)n);
  L.rprev = L.part + al256(sizeof(double) * (size_t)items * (n + 2));
  L.total = L.rprev + al256(sizeof(double) * (size_t)m);
  return L;
}

size_t resident_bytes(const ls_problem& p) {
  return al256(sizeof(double) * (size_t)p.m * p.lda) + al256(sizeof(double) * (size_t)p.m) +
         al256(sizeof(double) * (size_t)p.n);
}

__global__ void k_srv_init_states(IterState* st, unsigned int* pstatus, int cap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    IterState s{};
    s.done = 1;
    st[i] = s;
    pstatus[i] = 0;
  }
}

__global__ void k_srv_admit(const int* list, int k, unsigned int* pstatus) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) pstatus[list[i]] = 0;
}

}  // namespace

struct ls_server {
  ls_ctx* user = nullptr;       // the creating context (device, errors)
  ls_ctx* ctx = nullptr;        // own context: iteration stream, used for capture
  ls_ctx* adm = nullptr;        // own context: admission stream
  cudaEvent_t adm_done = nullptr;
  bool adm_pending = false;
  int adm_k = 0;                // requests in the pending admission batch
  int cap = 0, max_n = 0, zeta = 8, q = 100;
  ls_opts opts;
  size_t admit_budget = 0, admit_used = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  FirstFit alloc;
  // device tables
  BProb* dslots = nullptr;
  BPools pools{};
  int* alist = nullptr;
  int64_t* aoff = nullptr;
  int64_t* cnt = nullptr;
  BDone* done_rec = nullptr;
  unsigned int* done_count = nullptr;
  // admission buffers (cap entries)
  BProb* dadm = nullptr;
  int64_t* dadm_offs = nullptr;   // moffs | doffs | woffs
  int* dlist = nullptr;
  int* dorder = nullptr;
  // sketch scratch for one admission batch (grown on demand)
  int32_t* rows = nullptr;
  uint32_t* signs = nullptr;
  int64_t* row_ptr = nullptr;
  uint32_t* ent = nullptr;
  uint32_t* sort_scratch = nullptr;
  unsigned long long* fill = nullptr;
  size_t cap_entries = 0, cap_ent = 0, cap_cols = 0, cap_buckets = 0, cap_scratch = 0, cap_fill = 0;
  // host state

  struct Live {
    int64_t ticket = -1;
    size_t off = 0, bytes = 0, admit = 0;
  };
  std::vector<Live> live;
  std::vector<int> free_slots;
  struct Req {
    ls_problem p;
    int64_t ticket;
  };
  std::deque<Req> queue;
  std::vector<std::pair<int64_t, ls_info>> done;
  int64_t next_ticket = 0, steps = 0, completed = 0;
  int inflight = 0;
  cudaGraphExec_t graph = nullptr;
  int pass_grid = 0;
  int pass_cap = 0;             // doubles per pass buffer
  int qr_csize = 0;             // CTAs per cluster of the large-problem QR (0: not used)
  PassTune tune = default_tune();  // pass geometry, copied from the creating context
  BDone* h_rec = nullptr;      // pinned
  unsigned int* h_count = nullptr;
  // pinned staging of one admission batch (read by its async copies)
  BProb* h_adm = nullptr;
  int64_t* h_offs = nullptr;
  int* h_list = nullptr;
  int* h_order = nullptr;
  BProb* h_slots = nullptr;     // pinned mirror of the slot table
};

namespace {

ls_status srv_fail(ls_server* s, ls_status st, const char* msg) {
  if (s && s->user) s->user->err = msg;
  return st;
}

#define SRV_CUDA(s, call)                                                  \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      if (s->user) s->user->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? LS_ENOMEM : LS_ECUDA;       \
    }                                                                      \
  } while (0)

template <class T>
cudaError_t grow(T** p, size_t* have, size_t want) {
  if (want <= *have) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  size_t n = want + want / 4 + 1024;
  cudaError_t e = cudaMalloc(p, sizeof(T) * n);
  if (e == cudaSuccess) *have = n;
  return e;
}

// Capture the per-step graph: list iterating slots, pass, per-slot step.
ls_status capture_step(ls_server* s) {
  ls_ctx* ctx = s->ctx;
  SRV_CUDA(s, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_b_compact(ctx, s->dslots, s->cap, s->pools, s->alist, s->aoff, s->cnt);
  if (e == cudaSuccess)
    e = launch_b_pass(ctx, s->dslots, s->alist, s->aoff, s->cnt, s->max_n, s->pass_cap, (int64_t)1 << 40, s->pools);
  if (e == cudaSuccess)
    e = launch_b_step(ctx, s->dslots, s->alist, s->cnt, s->cap, s->pools, s->opts.use_stop, s->opts.extra_iters, s->q);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return srv_fail(s, LS_ECUDA, "capturing the server step failed");
  }
  e = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return srv_fail(s, LS_ECUDA, "instantiating the server step graph failed");
  return LS_OK;
}

// Admit queued requests (FIFO) while a slot, arena space and budget allow,
// and launch their sketch, factor and start on the admission stream (not
// waited for).  Returns the number admitted in *k.
ls_status admit(ls_server* s, int* kout) {
  ls_ctx* ctx = s->adm;
  std::vector<ls_problem> ps;
  std::vector<int> slots;
  while (!s->queue.empty() && !s->free_slots.empty() && (int)ps.size() < s->cap) {
    const ls_server::Req& r = s->queue.front();
    BProb tmp;
    BatchPlan one;
    batch_plan(&r.p, 1, &tmp, one, s->tune);
    const Layout L = request_layout(r.p.m, r.p.n, r.p.d, tmp.items);
    const size_t admit = L.total + resident_bytes(r.p);
    if (s->admit_used + admit > s->admit_budget) break;
    size_t off = 0;
    if (!s->alloc.alloc(L.total, &off)) break;
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->admit_used += admit;
    ls_server::Live& lv = s->live[slot];
    lv.ticket = r.ticket;
    lv.off = off;
    lv.bytes = L.total;
    lv.admit = admit;
    BProb b = tmp;
    b.boff = (int64_t)((off + L.B) / sizeof(double));
    b.roff = (int64_t)((off + L.R) / sizeof(double));
    b.voff = (int64_t)((off + L.V) / sizeof(double));
    b.poff = (int64_t)((off + L.part) / sizeof(double));
    b.rpoff = (int64_t)((off + L.rprev) / sizeof(double));
    b.moff = 0; b.doff = 0; b.toff = 0;
    s->h_slots[slot] = b;
    ps.push_back(r.p);
    slots.push_back(slot);
    s->queue.pop_front();
  }
  const int k = (int)ps.size();
  *kout = k;
  if (k == 0) return LS_OK;
  // admission batch: sketch offsets local to the batch, B in the slots' regions
  BatchPlan pl;
  batch_plan(ps.data(), k, s->h_adm, pl, s->tune);
  for (int i = 0; i < k; ++i) s->h_adm[i].boff = s->h_slots[slots[i]].boff;
  batch_offsets(s->h_adm, k, s->h_offs, s->h_offs + k, s->h_offs + 2 * k);
  std::vector<int> order(k);
  const int nsmall = batch_order(s->h_adm, k, order.data(), s->qr_csize > 0);
  for (int i = 0; i < k; ++i) {
    s->h_list[i] = slots[i];
    s->h_order[i] = slots[order[i]];
  }
  // scratch (no admission is in flight here, so it may be reallocated)
  const size_t entries = (size_t)pl.mtotal * s->zeta;
  SRV_CUDA(s, grow(&s->rows, &s->cap_entries, entries));
  SRV_CUDA(s, grow(&s->ent, &s->cap_ent, entries));
  SRV_CUDA(s, grow(&s->signs, &s->cap_cols, (size_t)pl.mtotal));
  SRV_CUDA(s, grow(&s->row_ptr, &s->cap_buckets, (size_t)pl.dtotal + 1));
  // one CTA per problem builds small problems' CSR fastest; a problem with
  // millions of entries would keep its CTA busy for tens of milliseconds, so
  // batches holding one go through the device-wide counting sort instead
  const bool global_csr = (int64_t)pl.max_m * s->zeta > b_csr_global_entries();
  uint32_t* scratch = nullptr;
  if (global_csr || pl.max_fill * s->zeta > 600.0) {
    SRV_CUDA(s, grow(&s->sort_scratch, &s->cap_scratch, 2 * entries));
    scratch = s->sort_scratch;
  }
  if (global_csr) SRV_CUDA(s, grow(&s->fill, &s->cap_fill, (size_t)pl.dtotal));
  // tables
  for (int i = 0; i < k; ++i)
    SRV_CUDA(s, cudaMemcpyAsync(s->dslots + slots[i], s->h_slots + slots[i], bprob_bytes(), cudaMemcpyHostToDevice,
                                ctx->stream));
  SRV_CUDA(s, cudaMemcpyAsync(s->dadm, s->h_adm, bprob_bytes() * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
  SRV_CUDA(s, cudaMemcpyAsync(s->dadm_offs, s->h_offs, sizeof(int64_t) * 3 * k, cudaMemcpyHostToDevice, ctx->stream));
  SRV_CUDA(s, cudaMemcpyAsync(s->dlist, s->h_list, sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
  SRV_CUDA(s, cudaMemcpyAsync(s->dorder, s->h_order, sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
  k_srv_admit<<<1, 256, 0, ctx->stream>>>(s->dlist, k, s->pools.pstatus);
  ++ctx->launches;
  SRV_CUDA(s, cudaGetLastError());
  SRV_CUDA(s, launch_b_sketch_indices(ctx, s->dadm, s->dadm_offs, pl, s->zeta, s->rows, s->signs));
  if (global_csr)
    SRV_CUDA(s, launch_sketch_csr(ctx, pl.mtotal, pl.dtotal, s->zeta, s->rows, s->signs, s->row_ptr, s->ent, s->fill,
                                  scratch, nullptr));
  else
    SRV_CUDA(s, launch_b_csr(ctx, s->dadm, pl, s->zeta, s->rows, s->signs, s->row_ptr, s->ent, scratch));
  SRV_CUDA(s, launch_b_gather(ctx, s->dadm, s->dadm_offs + 2 * k, pl, s->row_ptr, s->ent,
                              1.0 / std::sqrt((double)s->zeta), s->pools.B));
  SRV_CUDA(s, launch_b_factor2(ctx, s->dslots, s->dorder, nsmall, s->dorder + nsmall, k - nsmall, s->qr_csize, k,
                               s->dlist, s->pools));
  SRV_CUDA(s, launch_b_iter_init(ctx, s->dslots, k, s->dlist, s->pools, s->opts.gamma, s->opts.rho, s->opts.alpha,
                                 s->opts.beta));
  SRV_CUDA(s, cudaEventRecord(s->adm_done, ctx->stream));
  s->adm_pending = true;
  s->adm_k = k;
  s->inflight += k;
  return LS_OK;
}

// Drain the completion queue: free the finished requests' slots and regions.
ls_status drain(ls_server* s, int* n_done) {
  ls_ctx* ctx = s->ctx;
  SRV_CUDA(s, cudaMemcpyAsync(s->h_count, s->done_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  SRV_CUDA(s, cudaStreamSynchronize(ctx->stream));
  const unsigned int c = *s->h_count;
  *n_done = (int)c;
  if (c == 0) return LS_OK;
  SRV_CUDA(s, cudaMemcpyAsync(s->h_rec, s->done_rec, sizeof(BDone) * c, cudaMemcpyDeviceToHost, ctx->stream));
  SRV_CUDA(s, cudaMemsetAsync(s->done_count, 0, sizeof(unsigned int), ctx->stream));
  SRV_CUDA(s, cudaStreamSynchronize(ctx->stream));
  for (unsigned int i = 0; i < c; ++i) {
    const BDone& r = s->h_rec[i];
    ls_server::Live& lv = s->live[r.slot];
    ls_info in;
    std::memset(&in, 0, sizeof in);
    in.iters = r.iters;
    in.stop_reason = r.stop_reason;
    in.res_norm = r.res_norm;
    in.step_norm = r.step_norm;
    in.normest = r.normest;
    in.condest = r.condest;
    s->done.emplace_back(lv.ticket, in);
    s->alloc.release(lv.off, lv.bytes);
    s->admit_used -= lv.admit;
    lv = ls_server::Live();
    s->free_slots.push_back(r.slot);
    --s->inflight;
    ++s->completed;
  }
  return LS_OK;
}

}  // namespace

extern "C" {

size_t ls_server_request_bytes(int64_t m, int64_t n, int64_t lda, int64_t d) {
  if (m < 1 || n < 1 || d < 1 || lda < n) return 0;
  ls_problem p{};
  p.m = m; p.n = n; p.lda = lda; p.d = d;
  BProb tmp;
  BatchPlan one;
  batch_plan(&p, 1, &tmp, one, default_tune());
  return request_layout(m, n, d, tmp.items).total + resident_bytes(p);
}

ls_status ls_server_create(ls_ctx* user, int max_inflight, int64_t max_n, size_t workspace_bytes,
                           size_t admit_bytes, int zeta, int q, const ls_opts* opts, ls_server** out) {
  if (!user || !out) return LS_EINVAL;
  *out = nullptr;
  user->err.clear();
  if (max_inflight < 1 || max_n < 1 || max_n > 1024 || zeta < 1 || zeta > 32 || workspace_bytes < 4096) {
    user->err = "ls_server_create: need max_inflight >= 1, 1 <= max_n <= 1024, 1 <= zeta <= 32";
    return LS_EINVAL;
  }
  ls_server* s = new ls_server();
  s->user = user;
  s->cap = max_inflight;
  s->max_n = (int)max_n;
  s->zeta = zeta;
  s->q = q > 0 ? q : 100;
  ls_default_opts(&s->opts);
  if (opts) s->opts = *opts;
  s->admit_budget = admit_bytes ? admit_bytes : workspace_bytes;
  ls_status st = ls_create(&s->ctx, user->device, nullptr);
  if (st == LS_OK) st = ls_create(&s->adm, user->device, nullptr);
  if (st != LS_OK) {
    if (s->ctx) ls_destroy(s->ctx);
    delete s;
    return st;
  }
  if (cudaEventCreateWithFlags(&s->adm_done, cudaEventDisableTiming) != cudaSuccess) {
    ls_destroy(s->ctx);
    ls_destroy(s->adm);
    delete s;
    return LS_ECUDA;
  }
  auto bad = [&](const char* why) {
    user->err = why;
    ls_server_destroy(s);
    return LS_ENOMEM;
  };
  cudaSetDevice(user->device);
  const int cap = s->cap;
  if (cudaMalloc(&s->arena, workspace_bytes) != cudaSuccess) return bad("server workspace arena");
  s->arena_bytes = workspace_bytes;
  s->alloc.reset(workspace_bytes);
  double* base = reinterpret_cast<double*>(s->arena);
  s->pools.B = s->pools.R = s->pools.V = s->pools.part = s->pools.r_prev = base;
  if (cudaMalloc(&s->dslots, bprob_bytes() * cap) != cudaSuccess ||
      cudaMalloc(&s->pools.slots, sizeof(double) * 64 * cap) != cudaSuccess ||
      cudaMalloc(&s->pools.est, sizeof(double) * 2 * cap) != cudaSuccess ||
      cudaMalloc(&s->pools.st, sizeof(IterState) * cap) != cudaSuccess ||
      cudaMalloc(&s->pools.pstatus, sizeof(unsigned int) * cap) != cudaSuccess ||
      cudaMalloc(&s->done_rec, sizeof(BDone) * cap) != cudaSuccess ||
      cudaMalloc(&s->done_count, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&s->alist, sizeof(int) * cap) != cudaSuccess ||
      cudaMalloc(&s->aoff, sizeof(int64_t) * cap) != cudaSuccess ||
      cudaMalloc(&s->cnt, sizeof(int64_t) * 4) != cudaSuccess ||
      cudaMalloc(&s->dadm, bprob_bytes() * cap) != cudaSuccess ||
      cudaMalloc(&s->dadm_offs, sizeof(int64_t) * 3 * cap) != cudaSuccess ||
      cudaMalloc(&s->dlist, sizeof(int) * cap) != cudaSuccess ||
      cudaMalloc(&s->dorder, sizeof(int) * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_rec, sizeof(BDone) * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_count, sizeof(unsigned int) * 4) != cudaSuccess ||
      cudaMallocHost(&s->h_adm, bprob_bytes() * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_offs, sizeof(int64_t) * 3 * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_list, sizeof(int) * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_order, sizeof(int) * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_slots, bprob_bytes() * cap) != cudaSuccess)
    return bad("server tables");
  std::memset(s->h_slots, 0, bprob_bytes() * cap);
  s->pools.done_rec = s->done_rec;
  s->pools.done_count = s->done_count;
  cudaMemset(s->dslots, 0, bprob_bytes() * cap);
  cudaMemset(s->done_count, 0, sizeof(unsigned int));
  k_srv_init_states<<<(cap + 255) / 256, 256, 0, s->ctx->stream>>>(s->pools.st, s->pools.pstatus, cap);
  s->live.assign(cap, ls_server::Live());
  for (int i = cap - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->tune = user->tune;
  s->pass_cap = std::max(tune_cap(s->tune), s->max_n + 4);   // every slot's tile fits
  s->pass_grid = b_pass_grid(s->ctx, s->max_n, s->pass_cap);
  s->qr_csize = b_qr_cluster_size(s->ctx);
  if (s->pass_grid == 0) return bad("pass configuration");
  if (cudaStreamSynchronize(s->ctx->stream) != cudaSuccess) return bad("server set-up");
  if ((st = capture_step(s)) != LS_OK) {
    ls_server_destroy(s);
    return st;
  }
  *out = s;
  return LS_OK;
}

ls_status ls_server_destroy(ls_server* s) {
  if (!s) return LS_EINVAL;
  if (s->ctx) cudaStreamSynchronize(s->ctx->stream);
  if (s->adm) cudaStreamSynchronize(s->adm->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->adm_done) cudaEventDestroy(s->adm_done);
  void* ptrs[] = {s->arena, s->dslots, s->pools.slots, s->pools.est, s->pools.st, s->pools.pstatus, s->done_rec,
                  s->done_count, s->alist, s->aoff, s->cnt, s->dadm, s->dadm_offs, s->dlist, s->dorder, s->rows,
                  s->signs, s->row_ptr, s->ent, s->sort_scratch, s->fill};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* hptrs[] = {s->h_rec, s->h_count, s->h_adm, s->h_offs, s->h_list, s->h_order, s->h_slots};
  for (void* p : hptrs)
    if (p) cudaFreeHost(p);
  if (s->ctx) ls_destroy(s->ctx);
  if (s->adm) ls_destroy(s->adm);
  delete s;
  return LS_OK;
}

ls_status ls_server_submit(ls_server* s, const ls_problem* p, int64_t* ticket) {
  if (!s || !p) return LS_EINVAL;
  s->user->err.clear();
  if (!p->A || !p->b || !p->x) return srv_fail(s, LS_EINVAL, "null A, b or x");
  if (p->n < 1 || p->n > p->m) return srv_fail(s, LS_EINVAL, "need 1 <= n <= m");
  if (p->n > s->max_n) return srv_fail(s, LS_EINVAL, "n above the server's max_n");
  if (p->lda < p->n || (p->lda & 1) || (reinterpret_cast<uintptr_t>(p->A) & 15))
    return srv_fail(s, LS_EINVAL, "lda must be even and >= n, A 16-byte aligned");
  if (p->d < p->n || p->d > b_csr_max_d() || s->zeta > p->d)
    return srv_fail(s, LS_EINVAL, "need n <= d <= 12288 and zeta <= d");
  if (p->m * s->zeta > INT32_MAX) return srv_fail(s, LS_EINVAL, "m zeta reaches 2^31");
  const size_t need = ls_server_request_bytes(p->m, p->n, p->lda, p->d);
  BProb tmp;
  BatchPlan one;
  batch_plan(p, 1, &tmp, one, s->tune);
  if (need > s->admit_budget || request_layout(p->m, p->n, p->d, tmp.items).total > s->arena_bytes)
    return srv_fail(s, LS_ENOMEM, "request larger than the server's budget");
  ls_server::Req r;
  r.p = *p;
  r.ticket = s->next_ticket++;
  s->queue.push_back(r);
  if (ticket) *ticket = r.ticket;
  return LS_OK;
}

ls_status ls_server_step(ls_server* s, int* n_done) {
  if (!s) return LS_EINVAL;
  s->user->err.clear();
  cudaSetDevice(s->user->device);
  ls_status st;
  if (s->adm_pending) {
    const cudaError_t q = cudaEventQuery(s->adm_done);
    if (q == cudaSuccess) s->adm_pending = false;
    else if (q != cudaErrorNotReady) SRV_CUDA(s, q);
  }
  if (!s->adm_pending) {
    int k = 0;
    if ((st = admit(s, &k)) != LS_OK) return st;
  }
  // nothing else to iterate: wait for the admission batch instead of spinning
  if (s->adm_pending && s->inflight == s->adm_k) {
    SRV_CUDA(s, cudaEventSynchronize(s->adm_done));
    s->adm_pending = false;
  }
  int nd = 0;
  if (s->inflight - (s->adm_pending ? s->adm_k : 0) > 0) {
    SRV_CUDA(s, cudaMemsetAsync(s->ctx->d_status, 0, sizeof(unsigned int), s->ctx->stream));
    SRV_CUDA(s, cudaGraphLaunch(s->graph, s->ctx->stream));
    s->ctx->launches += 3;
    ++s->steps;
    if ((st = drain(s, &nd)) != LS_OK) return st;
    SRV_CUDA(s, cudaMemcpyAsync(s->ctx->h_pinned, s->ctx->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                s->ctx->stream));
    SRV_CUDA(s, cudaStreamSynchronize(s->ctx->stream));
    if (*reinterpret_cast<unsigned int*>(s->ctx->h_pinned) & LS_DEV_TIMEOUT)
      return srv_fail(s, LS_ETIMEOUT, "a bounded device wait gave up");
  }
  if (n_done) *n_done = nd;
  return LS_OK;
}

ls_status ls_server_poll(ls_server* s, int64_t* tickets, ls_info* infos, int cap, int* n_out) {
  if (!s || !n_out || cap < 0) return LS_EINVAL;
  const int n = std::min<int>(cap, (int)s->done.size());
  for (int i = 0; i < n; ++i) {
    if (tickets) tickets[i] = s->done[i].first;
    if (infos) infos[i] = s->done[i].second;
  }
  s->done.erase(s->done.begin(), s->done.begin() + n);
  *n_out = n;
  return LS_OK;
}

ls_status ls_server_get_stats(ls_server* s, ls_server_stats* out) {
  if (!s || !out) return LS_EINVAL;
  out->inflight = s->inflight;
  out->queued = (int64_t)s->queue.size();
  out->completed = s->completed;
  out->steps = s->steps;
  out->admitted_bytes = s->admit_used;
  out->workspace_bytes_used = s->alloc.used();
  return LS_OK;
}

}  // extern "C"
