/*
 * ls.h -- C ABI of libls, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of iterative sketching for overdetermined linear
 * least squares (E. N. Epperly, "Fast and forward stable randomized algorithms
 * for linear least-squares problems", arXiv:2311.04362).
 *
 * Problem (Sec. 1, Eq. (1.1)): x = argmin_y ||b - A y||, A m x n, m >= n,
 * full rank.  Method (Algorithm 2, "Iterative sketching"):
 *     S   d x m sparse sign embedding                 (Sec. 2.2, Eq. (2.4))
 *     B = S A, Sb = S b                                (sketch)
 *     (Q, R) = QR(B, 'econ')                          (Sec. 3.2, Eq. (3.4))
 *     x0 = R^{-1} (Q^T (S b))                         (Sec. 2.3, Eq. (2.5))
 *     repeat: r = b - A x; c = A^T r; d = R^{-1}(R^{-T} c); x = x + d
 * with the stopping rule of Sec. 3.3.
 *
 * Conventions for every call below
 *  - Every array argument is a pointer the caller owns.  Unless a call says
 *    otherwise it must be DEVICE memory of the context's device.  No call keeps
 *    a pointer after it returns.
 *  - A is row-major: A[j*lda + k] is entry (j, k); lda >= n, lda even, and A
 *    16-byte aligned (rows are streamed with 16-byte bulk copies).
 *  - B (the sketch) and R are column-major: B[t + c*ldb], R[i + j*ldr].
 *  - All calls run on the context's CUDA stream and RETURN AFTER THE WORK HAS
 *    FINISHED (each call synchronises that stream), so output arrays and the
 *    host-side ls_info are valid on return.
 *  - Calls never throw; they return an ls_status.  On any status other than
 *    LS_OK the outputs are unspecified and ls_last_error() gives a message.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LS_API __attribute__((visibility("default")))
#else
#define LS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LS_OK = 0,
    LS_EINVAL = 1,      /* invalid argument (sizes, leading dims, alignment, null) */
    LS_ENOMEM = 2,      /* device or pinned-host allocation failed */
    LS_ECUDA = 3,       /* a CUDA runtime call failed */
    LS_ERANK = 4,       /* R[k,k] of the sketch is zero or not finite (rank deficient) */
    LS_ENONFINITE = 5,  /* a non-finite value appeared in the iterate */
    LS_ETIMEOUT = 6,    /* a bounded device-side wait gave up (pipeline stalled) */
    LS_ENOTCONV = 7     /* q updates done and the stopping rule never held; x is still the q-th iterate */
} ls_status;

typedef struct ls_ctx ls_ctx;   /* opaque: device, stream, device scratch arena */

typedef struct {
    int   iters;        /* updates x <- x + d applied by this call */
    int   stop_reason;  /* 0: stopping rule held, 1: q reached, 2: stop rule off */
    double res_norm;    /* ||r(x_i)|| of the last residual formed */
    double step_norm;   /* ||r(x_i) - r(x_{i-1})|| of the last step tested */
    double normest;     /* estimate of ||R||_2 (Sec. 3.3) */
    double condest;     /* estimate of kappa_1(R) (Sec. 3.3) */
    float ms_sketch, ms_factor, ms_iterate;   /* device time of each phase (ls_solve) */
    float ms_pass;      /* device time of the fused passes that did work (CUDA events) */
    int   n_pass;       /* number of those passes */
    int   launches;     /* kernels this call launched */
} ls_info;

typedef struct {
    double gamma;       /* Sec. 3.3 stopping rule, default 1.0 */
    double rho;         /* Sec. 3.3 stopping rule, default 0.04 */
    int extra_iters;    /* updates to run after the rule first holds, default 3: the
                           residual is formed exactly, so further updates still lower
                           the forward error after the rule's first hold */
    int use_stop;       /* 1: apply the stopping rule (default), 0: run exactly q updates */
    double alpha;       /* App. B, Eq. (B.1) step weight; 1.0 = Algorithm 2 */
    double beta;        /* App. B, Eq. (B.1) momentum weight; 0.0 = Algorithm 2 */
} ls_opts;

/* Default options: gamma 1, rho 0.04, extra 3, stop on, alpha 1, beta 0. */
LS_API void ls_default_opts(ls_opts* opts);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * the calls run on (0: a new non-blocking stream owned by the context).
 * LS_ECUDA if the device is not an sm_103 GPU or the kernels fail to load. */
LS_API ls_status ls_create(ls_ctx** ctx, int device, void* cuda_stream);

/* Free the context and its device scratch.  NULL is accepted. */
LS_API ls_status ls_destroy(ls_ctx* ctx);

/* Text of the last error on this context ("" after a successful call). */
LS_API const char* ls_last_error(const ls_ctx* ctx);

/* Device scratch bytes the context needs for a solve of this shape (for
 * admission against an HBM budget).  Excludes the caller's A, b, x. */
LS_API size_t ls_workspace_bytes(int64_t m, int64_t n, int64_t d, int zeta);

/* (a1) Sparse sign embedding indices, Sec. 2.2, Eq. (2.4): for each column
 * j < m of S, zeta distinct rows in [0, d), ascending, written to
 * rows[j*zeta .. j*zeta+zeta-1]; signs[j] bit k is the sign of the k-th
 * smallest row (1 means -1).  Generated from Philox4x32-10 keyed by `seed`
 * (counter (j lo, j hi, block, 0)); bit-identical for a given (m, d, zeta,
 * seed).  rows: m*zeta int32, signs: m uint32 (device).
 * LS_EINVAL unless 1 <= zeta <= min(d, 32), d <= 2^31-1, m <= 2^31-1. */
LS_API ls_status ls_sketch_indices(ls_ctx* ctx, int64_t m, int64_t d, int zeta, uint64_t seed,
                            int32_t* rows, uint32_t* signs);

/* (a2) Counting sort of the m*zeta nonzeros of S by sketch row, stable in the
 * column index: row_ptr (d+1 int64) and ent (m*zeta uint32) with
 * ent[e] = (j << 1) | (sign < 0) for the e-th nonzero, ascending j inside
 * each sketch row.  Inputs are ls_sketch_indices outputs (device). */
LS_API ls_status ls_sketch_csr(ls_ctx* ctx, int64_t m, int64_t d, int zeta,
                        const int32_t* rows, const uint32_t* signs,
                        int64_t* row_ptr, uint32_t* ent);

/* (a1-a3) B_aug = S [A b] (Algorithm 2, sketch step): B column-major
 * d x (n+1), ldb >= d; column n holds S b.  Entry (t, c) is
 * (1/sqrt(zeta)) * (sum over column indices j of sketch row t, ascending, of
 * +-A[j, c]) with the sum taken left to right from +0.0; no floating-point
 * atomics, so the result is bit-identical run to run. */
LS_API ls_status ls_sketch(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                    const double* b, int64_t d, int zeta, uint64_t seed,
                    double* B, int64_t ldb);

/* (a4-a5) Householder QR of B_aug in place (Sec. 3.2, Eq. (3.4)); writes the
 * upper-triangular R (n x n, column-major, ldr >= n; strictly-lower part set
 * to zero), the sketch-and-solve start x0 = R^{-1} (Q^T S b)[0:n]
 * (Sec. 2.3, Eq. (2.5)), and in info (may be NULL) normest (ceil(ln n) power
 * steps on R, start vector from Philox keyed by `seed`) and condest
 * (||R||_1 times Hager's estimate of ||R^{-1}||_1), the estimates of Sec. 3.3.
 * The diagonal of R may be negative.  LS_ERANK if some R[k,k] is zero or
 * not finite.  B is overwritten with the Householder vectors. */
LS_API ls_status ls_factor(ls_ctx* ctx, double* B, int64_t d, int64_t n, int64_t ldb,
                    double* R, int64_t ldr, double* x0, uint64_t seed, ls_info* info);

/* (a6) One fused residual/gradient pass over A (Algorithm 2 loop body):
 * r = b - A x and c = A^T r, reading A from HBM once.  c: n doubles;
 * norms[0] = ||r||^2, norms[1] = ||r - r_prev||^2 (0 if r_prev is NULL).
 * r_out (m doubles) may be NULL; r_prev (m doubles) may be NULL and may equal
 * r_out (then it is read before being overwritten).  Sums are taken in a
 * fixed order, so the results are bit-identical run to run. */
LS_API ls_status ls_residual_gradient(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                               const double* b, const double* x, const double* r_prev,
                               double* r_out, double* c, double* norms);

/* (a6 as ls_iterate runs it for n <= 1024) A in fixed point, so that the
 * fused pass runs on the integer multiply-add units (no counterpart in the
 * paper's pseudocode: it is how this library forms the Algorithm 2 residual
 * and gradient to the accuracy Sec. 4.3, Eqs. (4.8)-(4.9), asks of them).
 * Row j is written as A_fx[2 (j ldf + k)] = lo, A_fx[2 (j ldf + k) + 1] = hi
 * with A[j, k] ~= (hi 2^28 + lo) 2^(row_exp[j] - 1077), 0 <= lo < 2^28, where
 * row_exp[j] is the largest biased FP64 exponent field in the row (at least
 * 1): entries within two binades of the row's largest are exact, smaller ones
 * are rounded to nearest, an error below 2^-55 of the row's largest
 * magnitude.  A_fx: m x ldf pairs of int32 (device, 16-byte aligned, ldf even,
 * ldf >= n); row_exp: m int32 (device).  A as for ls_residual_gradient.
 * LS_ENONFINITE if A holds an Inf or NaN (those rows are written as zero). */
LS_API ls_status ls_fixed_point(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                                int32_t* A_fx, int64_t ldf, int32_t* row_exp);

/* (a6) The fused residual/gradient pass of ls_residual_gradient on the fixed-
 * point A of ls_fixed_point (n <= 1024): r = b - A x and c = A^T r.  The row
 * dots and the column sums are exact integer sums of the 55-bit fixed-point
 * products (x is put in fixed point with one exponent; r_j with one exponent
 * per CTA), each result rounded once to FP64, so r and c differ from the
 * exact values for the fixed-point A by about one rounding.  Bit-identical run
 * to run.  Outputs and r_prev / r_out rules as ls_residual_gradient; a
 * non-finite x or r makes c and norms NaN. */
LS_API ls_status ls_residual_gradient_fx(ls_ctx* ctx, const int32_t* A_fx, const int32_t* row_exp, int64_t m,
                                         int64_t n, int64_t ldf, const double* b, const double* x,
                                         const double* r_prev, double* r_out, double* c, double* norms);

/* Bounded device waits of the fixed-point pass give up after `ns`
 * nanoseconds (0: the default, 2 s), set LS_ETIMEOUT and let the kernel
 * return; the context stays usable.  No counterpart in the paper. */
LS_API ls_status ls_set_wait_limit(ls_ctx* ctx, uint64_t ns);

/* Failure injection for tests (no counterpart in the paper).  The fault is
 * made on the host side of the library and consumed by the next call it
 * applies to:
 *   LS_FAULT_SKIP_TILE: in the next fixed-point pass, CTA 0's producer does
 *     not issue its tile number `arg`, so the consumers' bounded waits run
 *     out (with the wait limit above) and the call returns LS_ETIMEOUT;
 *   LS_FAULT_ALLOC: the next device scratch allocation fails (LS_ENOMEM);
 *   LS_FAULT_NONE: clear both. */
enum { LS_FAULT_NONE = 0, LS_FAULT_SKIP_TILE = 1, LS_FAULT_ALLOC = 2 };
LS_API ls_status ls_inject_fault(ls_ctx* ctx, int kind, int64_t arg);

/* (a7) The correction of Algorithm 2: y = R^{-T} c, d = R^{-1} y (two
 * triangular solves), x <- x + d.  y_out, d_out (n doubles) may be NULL. */
LS_API ls_status ls_correct(ls_ctx* ctx, const double* R, int64_t ldr, int64_t n, const double* c,
                     double* x, double* y_out, double* d_out);

/* (a6-a7) Iterate from x (in: start, out: final iterate), at most q updates,
 * with the Sec. 3.3 stopping rule (opts may be NULL for defaults).  For
 * n <= 1024 each call first puts A in fixed point (ls_fixed_point, in the
 * context's scratch: 8 m (n rounded up to even) + 4 m bytes) and runs the
 * fixed-point pass; above that the FP64 pass of ls_residual_gradient.
 * normest/condest come from ls_factor (pass info from ls_factor, or set
 * info->normest/condest); info must not be NULL.  Resumable: calling twice
 * with q1 then q2 and use_stop = 0 equals one call with q1 + q2.
 * Returns LS_OK when the rule held, LS_ENOTCONV when q updates ran without
 * it (x valid), LS_ENONFINITE if x became non-finite. */
LS_API ls_status ls_iterate(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda,
                     const double* b, const double* R, int64_t ldr, double* x, int q,
                     const ls_opts* opts, ls_info* info);

/* (a6-a7, row-sharded) ls_iterate with the rows of A and b split into
 * `nparts` parts: part p is A_parts[p] (m_parts[p] x n, row-major, leading
 * dimension lda, device) and b_parts[p] (m_parts[p]).  This is the
 * data-parallel form of the Algorithm 2 loop: every part forms its own
 * partial A^T r, ||r||^2 and ||r - r_prev||^2 (the fixed-point pass), the
 * partials are reduced in part order (exact integer sums of the column
 * partials, FP64 norm sums in part order), and R, x and the two substitutions
 * are shared.  On several GPUs each part would live on its own device with
 * one exchange of the partials per iteration; here all parts run on the
 * context's device.  n <= 1024, 1 <= nparts <= 64.  Results are bit-identical
 * run to run for a given split (the fixed-point exponents are per CTA, so a
 * different split rounds r differently, within the same bounds).  Other
 * arguments and status as ls_iterate. */
LS_API ls_status ls_iterate_rows(ls_ctx* ctx, int nparts, const double* const* A_parts, const int64_t* m_parts,
                                 int64_t n, int64_t lda, const double* const* b_parts, const double* R, int64_t ldr,
                                 double* x, int q, const ls_opts* opts, ls_info* info);

/* One problem of a batch (ls_solve_batched).  All pointers are device
 * pointers: row-major A (m x n, lda even >= n, 16-byte aligned), b (m), x (n,
 * output: the final iterate; left unwritten when the sketch is rank
 * deficient).  d is the embedding dimension and seed keys the problem's
 * sparse sign embedding (ls_sketch_indices with this seed).  Optional outputs
 * (NULL to skip): B_out receives [S A, S b] before factorisation (d x (n+1),
 * column-major, leading dimension d), R_out the triangular factor (n x n,
 * column-major, leading dimension n, zero below the diagonal). */
typedef struct {
    const double* A;
    const double* b;
    double* x;
    int64_t m, n, lda, d;
    uint64_t seed;
    double* B_out;
    double* R_out;
} ls_problem;

/* App. B, Eqs. (B.2) and (B.3): set opts->alpha / opts->beta for iterative
 * sketching with damping (alpha = (1-e^2)^2/(1+e^2), beta = 0) or with
 * momentum (alpha = (1-e^2)^2, beta = e^2), with the paper's recommended
 * distortion estimate e = sqrt(n/d).  Other fields are left as they are. */
LS_API void ls_opts_damping(ls_opts* opts, int64_t n, int64_t d);
LS_API void ls_opts_momentum(ls_opts* opts, int64_t n, int64_t d);

/* The whole method: sketch, factor, start, iterate (q <= 0 means 100).
 * A, b and x may be HOST or DEVICE pointers (detected per pointer); host
 * arrays are copied to context-owned device memory and x is copied back.
 * info may be NULL.  Status as ls_iterate. */
LS_API ls_status ls_solve(ls_ctx* ctx, const double* A, const double* b, int64_t m, int64_t n,
                   int64_t lda, int64_t d, int zeta, int q, uint64_t seed, double* x,
                   ls_info* info);

/* Solve `nprob` independent problems of different shapes together (each one
 * exactly as ls_solve_ex would: sketch, Householder QR, sketch-and-solve
 * start, refinement with the stopping rule), with one kernel launch per
 * phase for the whole batch.  Each problem's sketch is bit-identical to
 * ls_sketch of that problem.  probs: host array; infos: host array of nprob
 * (may be NULL), per problem iterations / stop reason (0 rule held, 1 q
 * reached, 2 stop rule off, 3 non-finite, 4 rank deficient) and estimates.
 * Limits: n <= 1024 per problem, sum of m and sum of d below 2^31.
 * Returns LS_OK when the batch ran (per-problem outcomes are in infos). */
LS_API ls_status ls_solve_batched(ls_ctx* ctx, const ls_problem* probs, int nprob, int zeta, int q,
                                  const ls_opts* opts, ls_info* infos);

/* Sparse A (Sec. 3.5: a few nonzeros per row): Algorithm 2 with the Sec. 3.3
 * stopping rule for A in CSR form -- row_ptr (m+1, int64), col (nnz, int32,
 * distinct within a row), val (nnz) -- and b (m); all device pointers.  The
 * sketch [S A, S b] is bit-identical to ls_sketch of the dense matrix; the QR
 * is the dense one; the residual/gradient pass reads A row-wise for A x and a
 * deterministic CSC copy (built here, nnz * 12 bytes of scratch) for A^T r.
 * x: n (device, output).  n <= 2048, nnz < 2^31.  Errors as ls_solve_ex
 * (LS_ERANK for a zero column, LS_ENOTCONV when q is reached).
 * ls_sketch_sparse: the sketch step alone, B (d x (n+1), column-major, ldb). */
LS_API ls_status ls_sketch_sparse(ls_ctx* ctx, const int64_t* row_ptr, const int32_t* col, const double* val,
                                  int64_t m, int64_t n, const double* b, int64_t d, int zeta, uint64_t seed, double* B,
                                  int64_t ldb);
LS_API ls_status ls_solve_sparse(ls_ctx* ctx, const int64_t* row_ptr, const int32_t* col, const double* val,
                                 int64_t m, int64_t n, int64_t nnz, const double* b, int64_t d, int zeta, int q,
                                 uint64_t seed, const ls_opts* opts, double* x, ls_info* info);

/* Autotuner of the batched pass (no counterpart in the paper; Sec. 3.3
 * mentions tuning the implementation to the machine): for each class of n
 * present in probs (n < 32, < 64, < 128, < 256, < 512, <= 1024), in turn,
 * it times the fused pass on a sample of up to 64 problems of every class
 * (x = 0, `reps` repetitions) for tile sizes {1536, 2560, 3840, 6144}
 * doubles and {64, 128, 256} rows per work item, the other classes held
 * fixed (the largest tile sets the launch's shared memory, so the classes
 * interact), and keeps a choice that is at least 1% faster.  Later ls_solve_batched*
 * calls and servers created from ctx use the table; the default is 3840 /
 * 128 everywhere.  Reads A and b only.  A different table changes the order
 * of the pass's sums, so results differ (within the same bounds) from an
 * untuned run; with one table they are deterministic.  report (may be NULL)
 * receives one line per class and the sample's pass time before and after.
 * ls_reset_tuning restores the defaults. */
LS_API ls_status ls_tune_batched(ls_ctx* ctx, const ls_problem* probs, int nprob, int reps, char* report,
                                 size_t report_len);
LS_API ls_status ls_reset_tuning(ls_ctx* ctx);

/* Mixed precision (no counterpart in the paper's experiments; Sec. 3.2 reads
 * the iteration as iterative refinement, which tolerates a preconditioner R
 * perturbed by c kappa u32): as ls_solve_batched, but the sketch is summed in
 * FP32 (each A entry rounded to FP32, FP32 accumulation in the same order,
 * the scale applied once) and the Householder QR runs in FP32 on one CTA per
 * problem; R, Q^T S b and everything after them are FP64 (R is the FP32
 * factor widened).  The FP64 residual and gradient make x as accurate as the
 * FP64 path; the FP32 R costs iterations (the contraction rate grows with
 * kappa u32), and beyond kappa(A) ~ 1e6 the iteration may not contract.
 * B_out receives the FP32 sketch widened to FP64, R_out the widened R. */
LS_API ls_status ls_solve_batched_mixed(ls_ctx* ctx, const ls_problem* probs, int nprob, int zeta, int q,
                                        const ls_opts* opts, ls_info* infos);

/* ---------------------------------------------------------------- serving
 * Continuous batching (no counterpart in the paper, which solves one problem
 * at a time): requests are queued by ls_server_submit, admitted in arrival
 * order while the admission budget allows, and every in-flight request
 * advances by one iteration of Algorithm 2 per ls_server_step.  Each admitted
 * request is sketched, factored and started exactly as ls_solve_batched does
 * it, so its result is bit-identical to solving it alone.  The server runs on
 * its own CUDA stream: the caller must have finished writing A and b before
 * ls_server_submit, and must not touch x until the request is returned by
 * ls_server_poll.  One thread at a time per server. */
typedef struct ls_server ls_server;
typedef struct {
    int64_t inflight;               /* admitted, not finished */
    int64_t queued;                 /* submitted, not admitted */
    int64_t completed;
    int64_t steps;                  /* iteration steps run */
    size_t admitted_bytes;          /* budget in use (resident A, b, x + workspace) */
    size_t workspace_bytes_used;    /* arena bytes in use */
} ls_server_stats;

/* Bytes a request counts against the admission budget: its A (m x lda), b,
 * x and the server workspace (sketch d x (n+1), R and R^T, eight n-vectors,
 * pass partials, previous residual).  0 for invalid sizes. */
LS_API size_t ls_server_request_bytes(int64_t m, int64_t n, int64_t lda, int64_t d);

/* Create a server on ctx's device.  max_inflight: slots; max_n (<= 1024):
 * largest n accepted; workspace_bytes: device arena for the workspaces
 * (allocated here); admit_bytes: admission budget (0: workspace_bytes);
 * zeta, q, opts: as for ls_solve_ex (opts may be NULL).  Errors: LS_EINVAL,
 * LS_ENOMEM, LS_ECUDA (text in ls_last_error(ctx)). */
LS_API ls_status ls_server_create(ls_ctx* ctx, int max_inflight, int64_t max_n, size_t workspace_bytes,
                                  size_t admit_bytes, int zeta, int q, const ls_opts* opts, ls_server** out);
LS_API ls_status ls_server_destroy(ls_server* srv);
/* Queue a request (device pointers as in ls_problem; B_out and R_out are
 * ignored; d <= 12288).  *ticket identifies it in ls_server_poll.  LS_ENOMEM
 * when the request alone exceeds the budget or the arena. */
LS_API ls_status ls_server_submit(ls_server* srv, const ls_problem* prob, int64_t* ticket);
/* Admit what fits, then one iteration of every in-flight request; returns
 * after the step has finished on the device.  *n_done (may be NULL): requests
 * finished in this call. */
LS_API ls_status ls_server_step(ls_server* srv, int* n_done);
/* Move up to cap finished requests out: tickets[i] and infos[i] (either may
 * be NULL); *n_out set to the number returned. */
LS_API ls_status ls_server_poll(ls_server* srv, int64_t* tickets, ls_info* infos, int cap, int* n_out);
LS_API ls_status ls_server_get_stats(ls_server* srv, ls_server_stats* out);

/* ls_solve with iteration options (stopping rule constants, extra updates,
 * damping / momentum of App. B); opts may be NULL for the defaults. */
LS_API ls_status ls_solve_ex(ls_ctx* ctx, const double* A, const double* b, int64_t m, int64_t n,
                             int64_t lda, int64_t d, int zeta, int q, uint64_t seed,
                             const ls_opts* opts, double* x, ls_info* info);

/* Fused residual/gradient pass that allocates nothing (no counterpart in the
 * paper: this is an interface for callers, not a step of the method).
 *
 * Some callers cannot call cudaMalloc: code that runs inside a memory pool or
 * arena it does not own, code under a framework that forbids device
 * allocation on its hot path, or code that must not trigger the implicit
 * synchronisation an allocation can cause.  An ls_ctx allocates its scratch,
 * so those callers use this entry point instead; it needs no context.
 *
 * Computes exactly what ls_residual_gradient computes (same kernels, same
 * fixed summation order, so the same bits on a device with at most 160 SMs,
 * such as GB300's 152; a larger device runs the pass on 160 CTAs, which
 * changes the order of the per-CTA sums but not their bounds), on
 * `cuda_stream` (a cudaStream_t, 0 = the legacy default stream) of the
 * CURRENT device.  The caller still
 * passes every input and output (device memory).  The per-CTA partial sums
 * live in a fixed array inside the library, about 1.3 MB, which every GPU
 * that loads the library holds until the process exits.
 *
 * Limits: n <= 1024 (the array's size); beyond that the call returns
 * LS_EINVAL.  Also LS_EINVAL for the argument rules of ls_residual_gradient,
 * LS_ECUDA on a non-sm_103 device or a CUDA error, LS_ETIMEOUT if a bounded
 * device wait gave up.  The first call on a device looks up the array's
 * device address (set-up, once per device); make that first call before any
 * stream capture.  All calls share the one array: calls that overlap on the
 * GPU (concurrent streams, or several host threads) race on it and must be
 * serialised by the caller.  Returns after the work finished (synchronises
 * the stream). */
LS_API ls_status ls_residual_gradient_noalloc(void* cuda_stream, const double* A, int64_t m, int64_t n,
                                              int64_t lda, const double* b, const double* x,
                                              const double* r_prev, double* r_out, double* c,
                                              double* norms);

#ifdef __cplusplus
}
#endif
#endif /* LS_H */
