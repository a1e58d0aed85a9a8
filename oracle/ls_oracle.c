/*
 * ls_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * iterative-sketching least-squares method of Epperly, "Fast and forward
 * stable randomized algorithms for linear least-squares problems"
 * (arXiv:2311.04362).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product (CUDA) path may include,
 * link, import or call this file.  It shares no code, header, table or
 * constant generator with the CUDA library; the two meet only through the
 * seeded input generators and the tests that compare them.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math, no
 * FMA contraction) so that every arithmetic operation below rounds exactly as
 * written, identically on x86-64 and aarch64.
 *
 * Contents, each following the passage it cites:
 *   philox4x32_10      Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *                      as easy as 1, 2, 3" (SC'11), the Philox-4x32 bijection
 *                      with 10 rounds.  (Random source; the paper used MATLAB's
 *                      generator, Sec. 1.1.1, so the stream layout below is
 *                      this library's own definition.)
 *   sparse-sign column Sec. 2.2, Eq. (2.4) (sparse sign embedding): column j of
 *                      S has exactly zeta nonzeros +-1/sqrt(zeta) at distinct,
 *                      uniformly random rows.  Rows are drawn by Floyd's
 *                      subset sampling (Bentley & Floyd, CACM 1987) with
 *                      Lemire's bounded-integer rejection (Lemire, ACM TOMACS
 *                      2019), then sorted ascending; bit k of one 32-bit word
 *                      gives the sign of the k-th smallest row (1 -> -1).
 *   counting sort      CSR of S grouped by sketch row t, stable in column j.
 *   sketch apply       Algorithm 2, sketch step: B = S A, and S b for the start.
 *   Householder QR     Algorithm 2, QR step; Sec. 3.2, Eq. (3.4); Householder reflectors
 *                      in the LAPACK geqr2 convention (Golub & Van Loan Sec. 5.1-5.2).
 *   sketch-and-solve   Sec. 2.3, Eq. (2.5), Algorithm 2 start: x0 = R^{-1} (Q^T S b).
 *   normest / condest  Sec. 3.3 (implementation guidance): ceil(log n) steps
 *                      of the power method on R; the 1-norm condition
 *                      estimator of Higham Ch. 15 (Hager's method).
 *   iteration          Algorithm 2 loop, with the Sec. 3.3 stopping rule,
 *                      and the damping/momentum update of App. B,
 *                      Eqs. (B.1)-(B.3).
 *   direct QR solve    Householder QR least squares (Sec. 1, Eq. (1.1)): the
 *                      yardstick for the forward-error acceptance rule.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 3-4).                                     */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 32-bit word stream of one sketch column j under a 64-bit seed:
 * block t = Philox(ctr = (lo32 j, hi32 j, t, 0), key = (lo32 seed, hi32 seed)),
 * words consumed block by block, lane 0..3 within a block. */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;            /* next lane of buf to hand out; 4 = exhausted */
} or_stream;

static void stream_init(or_stream* s, uint64_t seed, uint64_t j, uint32_t domain)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = (uint32_t)j;
    s->ctr[1] = (uint32_t)(j >> 32);
    s->ctr[2] = 0;          /* block index t */
    s->ctr[3] = domain;     /* 0: sketch columns, 1/2: power-method start vectors */
    s->pos = 4;
}

static uint32_t stream_next(or_stream* s)
{
    if (s->pos == 4) {
        or_philox4x32_10(s->ctr, s->key, s->buf);
        s->ctr[2] += 1;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform integer in [0, range), range >= 1 (Lemire 2019, nearly divisionless
 * multiply-shift with rejection of the biased low products). */
static uint32_t bounded_draw(or_stream* s, uint32_t range)
{
    uint64_t prod = (uint64_t)stream_next(s) * (uint64_t)range;
    uint32_t low = (uint32_t)prod;
    if (low < range) {
        uint32_t threshold = (uint32_t)(-range) % range;   /* 2^32 mod range */
        while (low < threshold) {
            prod = (uint64_t)stream_next(s) * (uint64_t)range;
            low = (uint32_t)prod;
        }
    }
    return (uint32_t)(prod >> 32);
}

uint32_t or_bounded_draw_test(uint64_t seed, uint64_t j, uint32_t range, int ndraws, uint32_t* out)
{
    or_stream s; stream_init(&s, seed, j, 0);
    for (int i = 0; i < ndraws; ++i) out[i] = bounded_draw(&s, range);
    return 0;
}

/* Column j of the sparse sign embedding (Sec. 2.2, Eq. (2.4)): zeta distinct rows in
 * [0, d), ascending, and the sign mask. */
int or_sparse_sign_column(uint64_t seed, int64_t j, int64_t d, int zeta,
                          int32_t* rows, uint32_t* signmask)
{
    if (zeta < 1 || zeta > 32 || d < zeta) return -1;
    or_stream s; stream_init(&s, seed, (uint64_t)j, 0);
    *signmask = stream_next(&s);
    int cnt = 0;
    /* Floyd: for t = d-zeta .. d-1 draw v uniform in [0, t]; take v unless it
     * is already chosen, in which case take t. */
    for (int64_t t = d - zeta; t < d; ++t) {
        uint32_t v = bounded_draw(&s, (uint32_t)(t + 1));
        int seen = 0;
        for (int i = 0; i < cnt; ++i) if (rows[i] == (int32_t)v) { seen = 1; break; }
        rows[cnt++] = seen ? (int32_t)t : (int32_t)v;
    }
    /* ascending order (insertion sort) */
    for (int i = 1; i < cnt; ++i) {
        int32_t key = rows[i]; int k = i - 1;
        while (k >= 0 && rows[k] > key) { rows[k + 1] = rows[k]; --k; }
        rows[k + 1] = key;
    }
    return 0;
}

/* rows: m*zeta int32 (column j's rows at j*zeta..), signs: m uint32 masks */
int or_sketch_indices(int64_t m, int64_t d, int zeta, uint64_t seed, int32_t* rows, uint32_t* signs)
{
    for (int64_t j = 0; j < m; ++j)
        if (or_sparse_sign_column(seed, j, d, zeta, rows + j * zeta, signs + j) != 0) return -1;
    return 0;
}

/* Counting sort of the m*zeta nonzeros of S by sketch row t, stable in j.
 * row_ptr: d+1 int64; ent: m*zeta uint32 with ent = (j << 1) | (sign < 0). */
int or_sketch_csr(int64_t m, int64_t d, int zeta, const int32_t* rows, const uint32_t* signs,
                  int64_t* row_ptr, uint32_t* ent)
{
    for (int64_t t = 0; t <= d; ++t) row_ptr[t] = 0;
    for (int64_t j = 0; j < m; ++j)
        for (int k = 0; k < zeta; ++k) row_ptr[rows[j * zeta + k] + 1] += 1;
    for (int64_t t = 0; t < d; ++t) row_ptr[t + 1] += row_ptr[t];
    int64_t* fill = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    if (!fill) return -2;
    for (int64_t t = 0; t < d; ++t) fill[t] = row_ptr[t];
    for (int64_t j = 0; j < m; ++j)
        for (int k = 0; k < zeta; ++k) {
            int32_t t = rows[j * zeta + k];
            uint32_t neg = (signs[j] >> k) & 1u;
            ent[fill[t]++] = ((uint32_t)j << 1) | neg;
        }
    free(fill);
    return 0;
}

/* B_aug = s * S [A b]  (Algorithm 2, sketch step), B column-major d x (n+1).
 * Each entry is the left-to-right sum, in ascending j, of +-A[j, c] over
 * sketch row t's bucket, started from +0.0, then one multiplication by
 * s = 1/sqrt(zeta).  Column n takes b in place of A. */
int or_sketch_apply(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                    int64_t d, const int64_t* row_ptr, const uint32_t* ent, double s,
                    double* B, int64_t ldb)
{
    (void)m;
    for (int64_t t = 0; t < d; ++t) {
        for (int64_t c = 0; c <= n; ++c) {
            double acc = 0.0;
            for (int64_t e = row_ptr[t]; e < row_ptr[t + 1]; ++e) {
                int64_t j = (int64_t)(ent[e] >> 1);
                double a = (c < n) ? A[j * lda + c] : b[j];
                if (ent[e] & 1u) acc = acc - a; else acc = acc + a;
            }
            B[t + c * ldb] = s * acc;
        }
    }
    return 0;
}

/* Euclidean norm of x[0..len) with scaling by the largest magnitude. */
static double scaled_norm(const double* x, int64_t len, int64_t inc)
{
    double mx = 0.0;
    for (int64_t i = 0; i < len; ++i) { double a = fabs(x[i * inc]); if (a > mx) mx = a; }
    if (mx == 0.0 || !isfinite(mx)) return mx;
    double ss = 0.0;
    for (int64_t i = 0; i < len; ++i) { double y = x[i * inc] / mx; ss = ss + y * y; }
    return mx * sqrt(ss);
}

/* Householder QR (LAPACK geqr2 convention) of the first nref columns of the
 * column-major rows x ncols matrix B; every reflector is also applied to the
 * remaining columns nref..ncols-1.  On exit R is in the upper triangle,
 * the essential parts of the Householder vectors below it, tau[k] the
 * reflector scalars.  Returns k+1 (> 0) if R[k,k] is zero or not finite. */
int or_householder_qr(double* B, int64_t rows, int64_t ncols, int64_t nref, int64_t ldb, double* tau)
{
    for (int64_t k = 0; k < nref; ++k) {
        double* col = B + k + k * ldb;          /* B[k:rows, k] */
        int64_t len = rows - k;
        double alpha = col[0];
        double xnorm = scaled_norm(col + 1, len - 1, 1);
        double beta, tk;
        if (xnorm == 0.0) {
            tk = 0.0; beta = alpha;             /* H = I */
        } else {
            double h = hypot(alpha, xnorm);
            beta = (alpha >= 0.0) ? -h : h;     /* beta = -sign(alpha) ||x||, sign(0) = + */
            tk = (beta - alpha) / beta;
            double scal = 1.0 / (alpha - beta);
            for (int64_t i = 1; i < len; ++i) col[i] = col[i] * scal;
        }
        col[0] = beta;
        tau[k] = tk;
        if (beta == 0.0 || !isfinite(beta)) return (int)(k + 1);
        /* apply H = I - tau v v^T, v = [1; col[1:]] to columns k+1..ncols-1 */
        for (int64_t j = k + 1; j < ncols; ++j) {
            double* cj = B + k + j * ldb;
            double w = cj[0];
            for (int64_t i = 1; i < len; ++i) w = w + col[i] * cj[i];
            double tw = tk * w;
            cj[0] = cj[0] - tw;
            for (int64_t i = 1; i < len; ++i) cj[i] = cj[i] - tw * col[i];
        }
    }
    return 0;
}

/* Solve R x = z by back substitution; R upper n x n column-major (ldr). */
static void back_subst(const double* R, int64_t n, int64_t ldr, const double* z, double* x)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int64_t k = i + 1; k < n; ++k) s = s - R[i + k * ldr] * x[k];
        x[i] = s / R[i + i * ldr];
    }
}

/* Solve R^T y = c by forward substitution. */
static void fwd_subst_T(const double* R, int64_t n, int64_t ldr, const double* c, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = c[i];
        for (int64_t k = 0; k < i; ++k) s = s - R[k + i * ldr] * y[k];
        y[i] = s / R[i + i * ldr];
    }
}

void or_trsv_upper(const double* R, int64_t n, int64_t ldr, const double* z, double* x) { back_subst(R, n, ldr, z, x); }
void or_trsv_upper_T(const double* R, int64_t n, int64_t ldr, const double* c, double* y) { fwd_subst_T(R, n, ldr, c, y); }

static double vnorm(const double* v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + v[i] * v[i];
    return sqrt(s);
}

/* Start vector of the power method: entry i = 2u - 1 with u the top 53 bits
 * of words 0,1 of Philox(ctr = (lo32 i, hi32 i, 0, domain), key = seed). */
static void power_start(uint64_t seed, uint32_t domain, int64_t n, double* v)
{
    for (int64_t i = 0; i < n; ++i) {
        or_stream s; stream_init(&s, seed, (uint64_t)i, domain);
        uint32_t w0 = stream_next(&s), w1 = stream_next(&s);
        uint64_t bits = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
        double u = (double)bits * 0x1.0p-53;
        v[i] = 2.0 * u - 1.0;
    }
}

int64_t or_power_steps(int64_t n)
{
    /* ceil(log n), natural logarithm, at least one step (Sec. 3.3) */
    int64_t k = 0;
    while (k < 64 && exp((double)k) < (double)n) ++k;
    return k < 1 ? 1 : k;
}

/* normest: power method on R^T R; returns ||R v|| for the final unit v. */
double or_normest(const double* R, int64_t n, int64_t ldr, uint64_t seed)
{
    double* v = (double*)malloc((size_t)n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    power_start(seed, 1u, n, v);
    double nv = vnorm(v, n);
    for (int64_t i = 0; i < n; ++i) v[i] = v[i] / nv;
    int64_t steps = or_power_steps(n);
    for (int64_t st = 0; st < steps; ++st) {
        for (int64_t i = 0; i < n; ++i) {         /* w = R v */
            double s = 0.0;
            for (int64_t k = i; k < n; ++k) s = s + R[i + k * ldr] * v[k];
            w[i] = s;
        }
        for (int64_t i = 0; i < n; ++i) {         /* v = R^T w */
            double s = 0.0;
            for (int64_t k = 0; k <= i; ++k) s = s + R[k + i * ldr] * w[k];
            v[i] = s;
        }
        nv = vnorm(v, n);
        for (int64_t i = 0; i < n; ++i) v[i] = v[i] / nv;
    }
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = i; k < n; ++k) s = s + R[i + k * ldr] * v[k];
        w[i] = s;
    }
    double est = vnorm(w, n);
    free(v); free(w);
    return est;
}

/* condest (Sec. 3.3, citing Higham, "Accuracy and Stability of Numerical
 * Algorithms", Ch. 15): kappa_1(R) estimated as ||R||_1 times Hager's 1-norm
 * estimate of ||R^{-1}||_1 with Higham's refinements (at most 5 sign-vector
 * steps, stop on a repeated sign vector or no increase, and the final
 * alternating-sign test vector).  R^{-1} and R^{-T} are applied by the two
 * substitutions.  The seed is unused: the estimator is deterministic. */
static double sgn1(double v) { return v >= 0.0 ? 1.0 : -1.0; }

double or_inv_norm1_est(const double* R, int64_t n, int64_t ldr)
{
    double* x = (double*)malloc((size_t)n * sizeof(double));
    double* y = (double*)malloc((size_t)n * sizeof(double));
    double* xi = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0 / (double)n;
    back_subst(R, n, ldr, x, y);                       /* y = R^{-1} x */
    double est = 0.0;
    if (n == 1) { est = fabs(y[0]); free(x); free(y); free(xi); return est; }
    for (int64_t i = 0; i < n; ++i) est = est + fabs(y[i]);
    for (int64_t i = 0; i < n; ++i) xi[i] = sgn1(y[i]);
    fwd_subst_T(R, n, ldr, xi, x);                     /* x = R^{-T} xi */
    int64_t j = 0;
    for (int64_t i = 1; i < n; ++i) if (fabs(x[i]) > fabs(x[j])) j = i;
    int iter = 2;
    for (;;) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        x[j] = 1.0;
        back_subst(R, n, ldr, x, y);                   /* y = R^{-1} e_j */
        double est_old = est;
        est = 0.0;
        for (int64_t i = 0; i < n; ++i) est = est + fabs(y[i]);
        int same = 1;
        for (int64_t i = 0; i < n; ++i) if (sgn1(y[i]) != xi[i]) { same = 0; break; }
        if (same || est <= est_old) break;
        for (int64_t i = 0; i < n; ++i) xi[i] = sgn1(y[i]);
        fwd_subst_T(R, n, ldr, xi, x);                 /* x = R^{-T} xi */
        int64_t jlast = j;
        j = 0;
        for (int64_t i = 1; i < n; ++i) if (fabs(x[i]) > fabs(x[j])) j = i;
        if (x[jlast] != fabs(x[j]) && iter < 5) { iter += 1; continue; }
        break;
    }
    /* alternating-sign test vector x_i = (-1)^i (1 + i/(n-1)) */
    for (int64_t i = 0; i < n; ++i) {
        double v = 1.0 + (double)i / (double)(n - 1);
        x[i] = (i % 2 == 0) ? v : -v;
    }
    back_subst(R, n, ldr, x, y);
    double alt = 0.0;
    for (int64_t i = 0; i < n; ++i) alt = alt + fabs(y[i]);
    alt = 2.0 * alt / (3.0 * (double)n);
    if (alt > est) est = alt;
    free(x); free(y); free(xi);
    return est;
}

double or_norm1_upper(const double* R, int64_t n, int64_t ldr)
{
    double mx = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i <= j; ++i) s = s + fabs(R[i + j * ldr]);
        if (s > mx) mx = s;
    }
    return mx;
}

double or_condest(const double* R, int64_t n, int64_t ldr, uint64_t seed, double normest)
{
    (void)seed; (void)normest;
    return or_norm1_upper(R, n, ldr) * or_inv_norm1_est(R, n, ldr);
}

/* Factor step: in-place QR of B_aug (d x (n+1), column-major), R copied out
 * to R (n x n column-major, ldr), x0 = R^{-1} z with z = (Q^T S b)[0:n]
 * (Sec. 2.3, Eq. (2.5)), and the two estimates.  Returns 0 or k+1 for a bad R[k,k]. */
int or_factor(double* B, int64_t d, int64_t n, int64_t ldb, double* R, int64_t ldr,
              double* x0, uint64_t seed, double* normest, double* condest)
{
    double* tau = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int rc = or_householder_qr(B, d, n + 1, n, ldb, tau);
    free(tau);
    if (rc != 0) return rc;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? B[i + j * ldb] : 0.0;
    back_subst(R, n, ldr, B + n * ldb, x0);
    *normest = or_normest(R, n, ldr, seed);
    *condest = or_condest(R, n, ldr, seed, *normest);
    return 0;
}

/* One residual/gradient pass (Algorithm 2 loop body, first two statements):
 * r_j = b_j - sum_k A_jk x_k ;  c_k = sum_j A_jk r_j  (plain ascending loops). */
void or_residual_gradient(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                          const double* x, double* r, double* c)
{
    for (int64_t j = 0; j < m; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s = s + A[j * lda + k] * x[k];
        r[j] = b[j] - s;
    }
    for (int64_t k = 0; k < n; ++k) c[k] = 0.0;
    for (int64_t j = 0; j < m; ++j)
        for (int64_t k = 0; k < n; ++k) c[k] = c[k] + A[j * lda + k] * r[j];
}

/* Iteration (Algorithm 2 loop) from x (in: x0, out: final iterate).
 * variant 0: stable residual  c = A^T (b - A x)
 * variant 1: "bad residual" control of Sec. 3.2, c = A^T b - A^T (A x)
 * alpha, beta: App. B, Eq. (B.1) update x+ = x + alpha d + beta (x - x_prev);
 * (1, 0) is Algorithm 2.
 * Stopping rule (Sec. 3.3): at the start of step i >= 1, with r_i = r(x_i),
 * stop if ||r_i - r_{i-1}|| <= u (gamma normest ||x_i|| + rho condest ||r_i||)
 * and return x_i, after `extra` further updates if extra > 0.
 * out[0] = updates applied, out[1] = 1 if the rule fired, out[2] = ||r||
 * of the last residual formed, out[3] = the last ||r_i - r_{i-1}||. */
int or_iterate(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
               const double* R, int64_t ldr, double* x, int q, int use_stop, int extra,
               double gamma, double rho, double normest, double condest,
               int variant, double alpha, double beta, double* out)
{
    const double u = 0x1.0p-53;
    double* r = (double*)malloc((size_t)m * sizeof(double));
    double* rp = (double*)malloc((size_t)m * sizeof(double));
    double* c = (double*)malloc((size_t)n * sizeof(double));
    double* y = (double*)malloc((size_t)n * sizeof(double));
    double* dd = (double*)malloc((size_t)n * sizeof(double));
    double* xp = (double*)malloc((size_t)n * sizeof(double));
    double* Atb = NULL;
    if (!r || !rp || !c || !y || !dd || !xp) return -2;
    for (int64_t k = 0; k < n; ++k) xp[k] = x[k];
    if (variant == 1) {
        Atb = (double*)malloc((size_t)n * sizeof(double));
        for (int64_t k = 0; k < n; ++k) Atb[k] = 0.0;
        for (int64_t j = 0; j < m; ++j)
            for (int64_t k = 0; k < n; ++k) Atb[k] = Atb[k] + A[j * lda + k] * b[j];
    }
    int updates = 0, fired = 0, remaining_extra = -1;
    double last_rn = 0.0, last_dn = 0.0;
    for (int i = 0; i < q; ++i) {
        /* r_i = b - A x_i */
        for (int64_t j = 0; j < m; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k) s = s + A[j * lda + k] * x[k];
            r[j] = b[j] - s;
        }
        double rn = vnorm(r, m);
        last_rn = rn;
        if (i >= 1) {
            double dn2 = 0.0;
            for (int64_t j = 0; j < m; ++j) { double t = r[j] - rp[j]; dn2 = dn2 + t * t; }
            double dn = sqrt(dn2);
            last_dn = dn;
            if (use_stop && remaining_extra < 0) {
                double xn = vnorm(x, n);
                if (dn <= u * (gamma * normest * xn + rho * condest * rn)) {
                    fired = 1;
                    remaining_extra = extra;
                }
            }
            if (remaining_extra == 0) break;
            if (remaining_extra > 0) remaining_extra -= 1;
        }
        if (variant == 1) {
            /* c = A^T b - A^T (A x) */
            double* ax = rp;   /* scratch; r_prev rebuilt below */
            for (int64_t j = 0; j < m; ++j) {
                double s = 0.0;
                for (int64_t k = 0; k < n; ++k) s = s + A[j * lda + k] * x[k];
                ax[j] = s;
            }
            for (int64_t k = 0; k < n; ++k) {
                double s = 0.0;
                for (int64_t j = 0; j < m; ++j) s = s + A[j * lda + k] * ax[j];
                c[k] = Atb[k] - s;
            }
        } else {
            for (int64_t k = 0; k < n; ++k) c[k] = 0.0;
            for (int64_t j = 0; j < m; ++j)
                for (int64_t k = 0; k < n; ++k) c[k] = c[k] + A[j * lda + k] * r[j];
        }
        fwd_subst_T(R, n, ldr, c, y);   /* y = R^{-T} c */
        back_subst(R, n, ldr, y, dd);   /* d = R^{-1} y */
        for (int64_t k = 0; k < n; ++k) {
            double xn = x[k] + alpha * dd[k] + beta * (x[k] - xp[k]);
            xp[k] = x[k];
            x[k] = xn;
        }
        for (int64_t j = 0; j < m; ++j) rp[j] = r[j];
        updates += 1;
    }
    out[0] = (double)updates; out[1] = (double)fired; out[2] = last_rn; out[3] = last_dn;
    free(r); free(rp); free(c); free(y); free(dd); free(xp); free(Atb);
    return 0;
}

/* Direct Householder QR least-squares solve of min ||b - A x|| (Eq. (1.1)),
 * A row-major m x n: QR of [A b] (b as an extra column receiving the
 * reflectors), then back substitution. */
int or_qr_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double* x)
{
    double* W = (double*)malloc((size_t)m * (size_t)(n + 1) * sizeof(double));
    double* tau = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!W || !tau) return -2;
    for (int64_t j = 0; j < m; ++j) {
        for (int64_t k = 0; k < n; ++k) W[j + k * m] = A[j * lda + k];
        W[j + n * m] = b[j];
    }
    int rc = or_householder_qr(W, m, n + 1, n, m, tau);
    if (rc == 0) back_subst(W, n, m, W + n * m, x);
    free(W); free(tau);
    return rc;
}

/* Whole method (Algorithm 2 with the Sec. 3.3 stopping rule). */
int or_solve(const double* A, const double* b, int64_t m, int64_t n, int64_t lda,
             int64_t d, int zeta, int q, uint64_t seed, int use_stop, int extra,
             double* x, double* info)
{
    int32_t* rows = (int32_t*)malloc((size_t)m * (size_t)zeta * sizeof(int32_t));
    uint32_t* signs = (uint32_t*)malloc((size_t)m * sizeof(uint32_t));
    int64_t* row_ptr = (int64_t*)malloc((size_t)(d + 1) * sizeof(int64_t));
    uint32_t* ent = (uint32_t*)malloc((size_t)m * (size_t)zeta * sizeof(uint32_t));
    double* B = (double*)malloc((size_t)d * (size_t)(n + 1) * sizeof(double));
    double* R = (double*)malloc((size_t)n * (size_t)n * sizeof(double));
    if (!rows || !signs || !row_ptr || !ent || !B || !R) return -2;
    int rc = or_sketch_indices(m, d, zeta, seed, rows, signs);
    if (rc == 0) rc = or_sketch_csr(m, d, zeta, rows, signs, row_ptr, ent);
    double s = 1.0 / sqrt((double)zeta);
    if (rc == 0) rc = or_sketch_apply(A, m, n, lda, b, d, row_ptr, ent, s, B, d);
    double ne = 0.0, ce = 0.0;
    if (rc == 0) rc = or_factor(B, d, n, d, R, n, x, seed, &ne, &ce);
    double out[4] = {0, 0, 0, 0};
    if (rc == 0) rc = or_iterate(A, m, n, lda, b, R, n, x, q, use_stop, extra, 1.0, 0.04, ne, ce, 0, 1.0, 0.0, out);
    if (info) { info[0] = out[0]; info[1] = out[1]; info[2] = out[2]; info[3] = out[3]; info[4] = ne; info[5] = ce; }
    free(rows); free(signs); free(row_ptr); free(ent); free(B); free(R);
    return rc;
}
