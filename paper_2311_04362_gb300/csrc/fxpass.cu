// fxpass.cu -- the fused residual/gradient pass of Algorithm 2 (a6) in exact
// fixed-point integer arithmetic, so that it runs on the integer multiply-add
// units instead of the FP64 pipe.
//
// Why: on GB300 an FP64 FMA issues at about 1.7 per SM clock while a 32x32 ->
// 64-bit integer multiply-add (IMAD.WIDE) issues at about 60 (measured by
// rates.cu).  The FP64 pass needs two FMAs per element of A and is bound by
// that pipe at ~37% of HBM bandwidth.  Three IMAD.WIDE per element and
// direction (Karatsuba's split of the 55 x 55-bit product) fit the integer
// units several times over, and the pass runs at about 0.85 of the HBM
// bandwidth its one read of A needs.
//
// Representation (exact, reversible up to the stated rounding):
//  * A row j is held in 55-bit fixed point relative to its own binade bound:
//    A_jk ~= a_jk 2^(e_j - 1077), |a_jk| < 2^55, where e_j is the largest
//    biased FP64 exponent field of the row (subnormals count as 1).  Entries
//    within 2 binades of the row's largest are exact; smaller ones are rounded
//    to nearest (ties to even), an error below 2^-55 of the row's largest
//    magnitude.  a = hi 2^28 + lo with 0 <= lo < 2^28, stored as int2 {lo, hi}.
//  * x is held the same way with one exponent for the whole vector (per pass).
//  * The row dot S_j = sum_k a_jk X_k is formed EXACTLY in 128-bit integers
//    from three partial products per entry, hi*Xh, (hi + lo)*(Xh + Xl) and
//    lo*Xl (the cross term hi*Xl + lo*Xh is the middle one minus the outer
//    two), accumulated in 64-bit sums that cannot overflow for the bounded
//    column counts per lane.  b_j is put in the same units and r_j = b_j -
//    (A x)_j is formed exactly too, so r_j carries a single rounding when it
//    is converted to FP64.
//  * For c = A^T r, rho_j = r_j 2^(e_j - 1077) is put in 55-bit fixed point
//    with one exponent E per CTA (the largest seen so far; when a larger one
//    arrives the CTA's accumulators are shifted right first), and
//    sum_j a_jk P_j is accumulated exactly per column in 64-bit partial sums
//    (the same three products) that are folded every <= 32 rows into a
//    128-bit accumulator in units of 2^28 (the fold drops bits below 2^28 of
//    a value of order 2^110).
//  * The per-CTA accumulators are summed exactly by k_fx_reduce after
//    alignment to the largest CTA exponent, and rounded once to FP64.
// So r and c carry the rounding of A and x to 55 bits, one rounding each,
// and no summation error: well inside the normwise bounds the analysis of
// Sec. 4.3 (Eqs. (4.8)-(4.9)) asks of the residual and gradient, and tighter
// than FP64 dot products (which err by ~sqrt(n) u).  Sums are exact, so the
// results depend on the launch geometry only through the CTA exponents:
// bit-identical run to run.
//
// k_fx_pass is warp-specialized (11 warps, one CTA per SM): a TMA producer
// warp streams row tiles of the fixed-point A into a ring of shared stages,
// and asks L2 for the CTA's next tile as it loads one (cp.async.bulk
// .prefetch: with three 64 KB stages held by the pipeline, the load that
// refills a stage then comes from L2 instead of waiting on DRAM);
// warps 0-3 form the exact partial row dots of tile k (each lane two rows of
// the tile, in four independent accumulator sets per row, so that the
// integer multiply-add chains overlap) and hand them over through a two-slot
// ring; two epilogue warps, taking alternate tiles, finish the rows (r_j, the
// norms, the fixed point of r_j at the CTA's running exponent, which passes
// from one to the other) and hand them to warps 4-7, which accumulate A^T r
// for their columns.  The groups work on different tiles at once; every
// hand-off is an mbarrier and every wait is bounded by the context's wait
// limit (a group that gives up leaves its loop as a whole warp, so no
// barrier is left waiting).  Measured at m = 2e6, n = 1000 on the way:
// eight row and eight column warps, 4.47 ms against 4.24 with four each;
// one barrier per 256-column box instead of per tile (the row warps start on
// a tile's first box), 3.69 against 3.22 ms; tiles of 4 rows with 6 stages
// and three epilogue warps, 4.52 against 3.22 ms (the per-tile hand-offs
// cost more than the deeper ring won); eight row warps, 3.31 against 3.04 ms;
// eight column warps, 2.88 against 2.81 ms.
#include "ls_internal.cuh"
#include "fxarith.cuh"

namespace lsk {

namespace {

using namespace fx;

constexpr int kFxRW = 4;                        // row-group warps
constexpr int kFxCW = 4;                        // column-group warps
constexpr int kFxEW = 2;                        // epilogue warps (alternate tiles)
constexpr int kFxThreads = (kFxRW + kFxCW + 1 + kFxEW) * 32;   // + producer
constexpr int kFxFoldRows = 32;                 // column sums are folded at most every 32 rows

// Rows per tile of the instantiation NPT2 (1, 2, 4, 6, 8; it serves the n
// with ceil(n / 128) <= NPT2): 32 for n <= 256 (one box per row), 16 for
// n <= 512 (two boxes of 256 columns), 8 for n <= 1024 (three or four).
// fx_geometry picks the same; a compile-time value turns the shared-memory
// offsets of the inner loops into immediates.  NPT2 128 <= 256 nbox, so the
// column lanes' loads stay inside the stage's boxes.
__host__ __device__ constexpr int fx_tile_rows(int npt2) { return npt2 >= 5 ? 8 : (npt2 >= 3 ? 16 : 32); }

// Bounded wait for the phase with the given parity.  try_wait carries a
// suspend-time hint, so a waiting warp is parked by the hardware until the
// phase completes (or the hint runs out) instead of spinning: spinning
// waiters took issue slots and shared-memory bandwidth from the warps doing
// the work on the same sub-partition.  False once `ns` have passed.
__device__ __forceinline__ bool fx_try(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of a phase (cheaper than try_wait when it has completed).
__device__ __forceinline__ bool fx_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool fx_wait(uint64_t* bar, uint32_t parity, unsigned long long ns) {
  if (fx_test(bar, parity)) return true;   // the clock is read only when the phase is not complete yet
  const uint64_t deadline = gtimer() + ns;
  for (;;) {
    if (fx_try(bar, parity, 20000u)) return true;
    if (gtimer() > deadline) return false;
  }
}


}  // namespace

// ----------------------------------------------------------------- A -> fixed
// One warp per row: the row's binade bound, then every entry in fixed point.
__global__ void __launch_bounds__(256) k_to_fixed(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                  int2* __restrict__ Af, int64_t ldf, int* __restrict__ rexp,
                                                  unsigned int* status) {
  const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= m) return;
  const unsigned long long* row = reinterpret_cast<const unsigned long long*>(A + j * lda);
  int top = 1, bad = 0;
  for (int k = lane; k < n; k += 32) {
    const int e = (int)((__ldg(row + k) >> 52) & 0x7FF);
    bad |= (e == 0x7FF);
    top = max(top, e);
  }
  top = warp_max_int(top);
  bad = __any_sync(0xffffffffu, bad);
  if (bad && lane == 0) atomicOr(status, LS_DEV_NONFINITE);
  int2* out = Af + j * ldf;
  for (int k = lane; k < n; k += 32) out[k] = bad ? make_int2(0, 0) : fx_limbs(fx_of(__ldg(row + k), top));
  if (lane == 0) rexp[j] = top;
}

// ----------------------------------------------------------------- the pass
struct FxArgs {
  int64_t m;
  int n, boxw, nbox, tr, stages, ntiles;
  const int* rexp;           // e_j per row
  const double* b;
  const double* x;
  const double* r_prev;      // may be null
  double* r_out;             // may be null (may equal r_prev)
  long long* part;           // gridDim.x * (2 n + 4) words
  const IterState* st;       // null: always run
  unsigned int* status;
  unsigned long long wait_ns;
  int inject_skip;           // CTA 0's producer skips this tile (test hook; -1 none)
};

template <int NPT2>
__global__ void __launch_bounds__(kFxThreads, 1) k_fx_pass(const __grid_constant__ CUtensorMap map, FxArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (a.st && a.st->done) return;
  constexpr int tr = fx_tile_rows(NPT2);
  constexpr bool kBoxed = NPT2 >= 4;                // rows cut into boxes of 256 columns (n > 256)
  const int n = a.n, boxw = kBoxed ? 256 : a.boxw, nbox = a.nbox, S = a.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const size_t stage_elems = (size_t)tr * nbox * boxw;
  const int pitch = kBoxed ? 256 : boxw;            // elements between rows of one box
  // layout: tiles [S][stage] | p1 [2][kFxRW][tr] i128 | xs [n] int4 | rslot [S][tr] | rshift [S] | barriers
  int2* tiles = reinterpret_cast<int2*>(smem_raw);
  __int128* p1 = reinterpret_cast<__int128*>(tiles + S * stage_elems);
  int4* xs = reinterpret_cast<int4*>(p1 + 2 * kFxRW * tr);     // {lo, hi, lo + hi, 0} of x
  const int xlen = kBoxed ? nbox * 256 : n;          // boxed rows: zero-padded to whole boxes
  int2* rslot = reinterpret_cast<int2*>(xs + xlen);
  int* rshift = reinterpret_cast<int*>(rslot + S * tr);
  uint64_t* full = reinterpret_cast<uint64_t*>(rshift + ((S + 1) & ~1));
  uint64_t* empty = full + S;      // stage consumed (column group)
  uint64_t* rready = empty + S;    // P of a tile written (epilogue warp)
  uint64_t* rfree = rready + S;    // P of a tile consumed (column group)
  uint64_t* pready = rfree + S;    // [2] row-dot partials of a tile written (row warps)
  uint64_t* pfree = pready + 2;    // [2] row-dot partials read (epilogue warp)
  __shared__ int s_xtop, s_xbad;
  // the running CTA exponent handed from the epilogue warp of tile k to that
  // of tile k + 1 (value and barrier per parity of k), and the second
  // epilogue warp's sums for the partial written at the end
  __shared__ __align__(8) uint64_t s_eready[2];
  __shared__ int s_ecta[2];
  __shared__ double s_esum[2];
  __shared__ int s_eflag[2];

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kFxCW);
      mbar_init(&rready[s], 1);
      mbar_init(&rfree[s], kFxCW);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&pready[i], kFxRW);
      mbar_init(&pfree[i], 1);
      mbar_init(&s_eready[i], 1);
    }
    fence_mbar_init();
    s_xtop = 1;
    s_xbad = 0;
  }
  __syncthreads();
  // x in fixed point with one binade bound for the vector (the same in every CTA)
  {
    int top = 1, bad = 0;
    const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(a.x);
    for (int i = tid; i < n; i += blockDim.x) {
      const int e = (int)((xb[i] >> 52) & 0x7FF);
      bad |= (e == 0x7FF);
      top = max(top, e);
    }
    top = warp_max_int(top);
    if (__any_sync(0xffffffffu, bad) && lane == 0) s_xbad = 1;
    if (lane == 0) atomicMax(&s_xtop, top);
    __syncthreads();
    const int xt = s_xtop;
    for (int i = tid; i < xlen; i += blockDim.x) {
      const int2 l = (i < n) ? fx_limbs(fx_of(xb[i], xt)) : make_int2(0, 0);
      xs[i] = make_int4(l.x, l.y, l.x + l.y, 0);
    }
    __syncthreads();
  }
  const int xtop = s_xtop;
  long long* out = a.part + (size_t)blockIdx.x * (2 * n + 4);
  const uint32_t tile_bytes = (uint32_t)(stage_elems * sizeof(int2));

  if (warp == kFxRW + kFxCW) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      prefetch_tmap(&map);
      int k = 0;
      for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
        const int s = k % S;
        if (k >= S && !fx_wait(&empty[s], ((k / S) - 1) & 1, a.wait_ns)) {
          atomicOr(a.status, LS_DEV_TIMEOUT);
          break;
        }
        if (blockIdx.x == 0 && k == a.inject_skip) continue;   // test hook: this tile never arrives
        mbar_arrive_expect_tx(&full[s], tile_bytes);
        int2* dst = tiles + (size_t)s * stage_elems;
        for (int q = 0; q < nbox; ++q) tma_load_2d(dst + (size_t)q * tr * boxw, &map, q * boxw, t * tr, &full[s]);
        // pull the CTA's next tile into L2 now, so that its load (once a
        // stage frees) comes from L2; DRAM is read once either way
        const int tp = t + gridDim.x;
        if (tp < a.ntiles)
          for (int q = 0; q < nbox; ++q)
            asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)&map),
                         "r"(q * boxw), "r"(tp * tr)
                         : "memory");
      }
      // drain: every issued copy lands before the CTA can exit
      const int issued = k;
      for (int kk = max(0, issued - S); kk < issued; ++kk)
        fx_wait(&full[kk % S], (kk / S) & 1, a.wait_ns);
    }
    return;
  }

  if (warp < kFxRW) {
    // ------------------------------------------------------------ row warps
    // lane (rl, q) of warp w sums rows rl + g RG (g < RPL) over the columns
    // rho + i CS of each box (rotated by rl so that the rows of a warp sit on
    // different banks), in four independent accumulator sets per row; each x
    // value loaded serves RPL rows.  The lanes of a row are combined by
    // shuffles and each warp's row partials go to the epilogue warp.  Rows
    // past m read the TMA's zero fill, so every lane runs the same loop.
    constexpr int RPL = 2, LPR = 32 * RPL / tr, CS = kFxRW * LPR, RG = tr / RPL;
    const int rl = lane / LPR, q = lane - rl * LPR;
    const int rho = LPR * ((warp + rl) % kFxRW) + q;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
      const int s = k % S, slot = k & 1;
      bool ok = fx_wait(&full[s], (k / S) & 1, a.wait_ns);
      if (ok && k >= 2) ok = fx_wait(&pfree[slot], ((k >> 1) - 1) & 1, a.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(a.status, LS_DEV_TIMEOUT);
        break;
      }
      const int2* tl = tiles + (size_t)s * stage_elems;
      // Karatsuba: hi*xh, (hi + lo)*(xh + xl) and lo*xl per entry; the cross
      // term is TK - T2 - T0 (three multiply-adds instead of four)
      int64_t T2[RPL][4], TK[RPL][4], T0[RPL][4];
#pragma unroll
      for (int g = 0; g < RPL; ++g)
#pragma unroll
        for (int u = 0; u < 4; ++u) { T2[g][u] = 0; TK[g][u] = 0; T0[g][u] = 0; }
      if (kBoxed) {
        // every box is walked at its full 256 columns: columns past n hold
        // the TMA's zero fill and x is zero-padded there, so all lanes run
        // the same compile-time loop (NB blocks of eight columns per box)
        constexpr int NB = 256 / (8 * CS);
        static_assert(NB >= 1 && NB * 8 * CS == 256, "the row lanes must cover a box");
        for (int qb = 0; qb < nbox; ++qb) {
          const int2* bp = tl + (size_t)qb * tr * 256 + rl * 256 + rho;
          const int4* xp = xs + qb * 256 + rho;
#pragma unroll
          for (int blk = 0; blk < NB; ++blk) {
            int2 av[RPL][8];
            int4 xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              xv[u] = xp[(blk * 8 + u) * CS];
#pragma unroll
              for (int g = 0; g < RPL; ++g) av[g][u] = bp[g * RG * 256 + (blk * 8 + u) * CS];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
              for (int g = 0; g < RPL; ++g) {
                T2[g][u & 3] = mad_wide(av[g][u].y, xv[u].y, T2[g][u & 3]);
                TK[g][u & 3] = mad_wide(av[g][u].x + av[g][u].y, xv[u].z, TK[g][u & 3]);
                T0[g][u & 3] = mad_wide(av[g][u].x, xv[u].x, T0[g][u & 3]);
              }
          }
        }
      } else {
        const int2* bp = tl + rl * pitch;
        const int4* xp = xs;
        const int w = n;
        int c = rho;
        for (; c + 7 * CS < w; c += 8 * CS) {          // eight columns: all loads, then the products
          int2 av[RPL][8];
          int4 xv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            xv[u] = xp[c + u * CS];
#pragma unroll
            for (int g = 0; g < RPL; ++g) av[g][u] = bp[g * RG * pitch + c + u * CS];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int g = 0; g < RPL; ++g) {
              T2[g][u & 3] = mad_wide(av[g][u].y, xv[u].y, T2[g][u & 3]);
              TK[g][u & 3] = mad_wide(av[g][u].x + av[g][u].y, xv[u].z, TK[g][u & 3]);
              T0[g][u & 3] = mad_wide(av[g][u].x, xv[u].x, T0[g][u & 3]);
            }
        }
        for (; c < w; c += CS) {
          const int4 xv = xp[c];
#pragma unroll
          for (int g = 0; g < RPL; ++g) {
            const int2 av = bp[g * RG * pitch + c];
            T2[g][0] = mad_wide(av.y, xv.y, T2[g][0]);
            TK[g][0] = mad_wide(av.x + av.y, xv.z, TK[g][0]);
            T0[g][0] = mad_wide(av.x, xv.x, T0[g][0]);
          }
        }
      }
      // a set holds at most 13 of the lane's columns (8 for boxed rows; with
      // one box, n / 32 <= 8 plus a tail of up to 7 in set 0), so
      // |TK| < 13 (1.5 2^28)^2 < 2^62
#pragma unroll
      for (int g = 0; g < RPL; ++g) {
        int64_t S2 = 0, S1 = 0, S0 = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) { S2 += T2[g][u]; S1 += TK[g][u] - T2[g][u] - T0[g][u]; S0 += T0[g][u]; }
        __int128 V = ((__int128)S2 << 56) + ((__int128)S1 << 28) + (__int128)S0;
#pragma unroll
        for (int o = LPR >> 1; o > 0; o >>= 1) V += shfl_xor_i128(V, o);
        if (q == 0) p1[((size_t)slot * kFxRW + warp) * tr + rl + g * RG] = V;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pready[slot]);
    }
    return;
  }

  if (warp > kFxRW + kFxCW) {
    // ------------------------------------------------------------ epilogue warps
    // Epilogue warp e takes the tiles k = e, e + 2, ... of the CTA (its slot
    // of the row-dot ring is e).  Lane r finishes row r of a tile: the exact
    // row dot (the row warps' partials in warp order), r_j = b_j - (A x)_j,
    // the squared norms, and r_j 2^(e_j - 1077) in fixed point at the CTA's
    // running exponent, handed to the column group with the shift its sums
    // need first.  The running exponent is the one sequential step: tile k
    // takes tile k - 1's from the other warp (s_ecta / s_eready) after its
    // own rows are done, so the two warps' row work overlaps.
    const int e = warp - (kFxRW + kFxCW + 1);
    double rn2 = 0.0, dn2 = 0.0;
    int Ecta = kNoExp, bad = 0;
    // the row scalars (b, e_j, r_prev) of the warp's next tile are loaded one
    // tile ahead, so their global-memory latency is not on the hand-off path
    double nb = 0.0, nrp = 0.0;
    int ne = 0;
    auto load_next = [&](int tn) {
      nb = 0.0; nrp = 0.0; ne = 0;
      if (tn < a.ntiles) {
        const int64_t r0 = (int64_t)tn * tr;
        if (r0 + lane < a.m && lane < tr) {
          nb = a.b[r0 + lane];
          ne = a.rexp[r0 + lane];
          if (a.r_prev) nrp = a.r_prev[r0 + lane];
        }
      }
    };
    const int stride = kFxEW * gridDim.x;
    load_next(blockIdx.x + e * gridDim.x);
    int k = e;
    for (int t = blockIdx.x + e * gridDim.x; t < a.ntiles; t += stride, k += kFxEW) {
      const int s = k % S, slot = k & 1;
      const int64_t row0 = (int64_t)t * tr;
      const int rows = (int)((a.m - row0 < (int64_t)tr) ? (a.m - row0) : (int64_t)tr);
      const double bj = nb, rpj = nrp;
      const int ej = ne;
      load_next(t + stride);
      bool ok = fx_wait(&pready[slot], (k >> 1) & 1, a.wait_ns);
      if (ok && k >= S) ok = fx_wait(&rfree[s], ((k / S) - 1) & 1, a.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(a.status, LS_DEV_TIMEOUT);
        break;
      }
      // r_j = b_j - S_j 2^sc is formed exactly in 128 bits (b_j put at the
      // dot's scale; bits of b_j below 2^sc are rounded) and rounded once;
      // rho_j's fixed point is then taken from the exact R_j.  |R_j| is
      // normalised once (Nh: its top 64 bits, Ns: whether any bit below them
      // is set), and both roundings -- to 53 bits for r_j, to the CTA's fixed
      // point for P_j -- are taken from (Nh, Ns), ties to even.  A b_j too
      // large for that scale (or non-finite) takes the FP64 route.
      uint64_t rbits = 0, Nh = 0;
      int qj = kNoExp, Lx = 0;
      bool exact = false, Ns = false, neg = false;
      double rj = 0.0;
      const int sc = ej + xtop - 2154;
      if (lane < rows) {
        __int128 Sj = 0;
#pragma unroll
        for (int w = 0; w < kFxRW; ++w) Sj += p1[((size_t)slot * kFxRW + w) * tr + lane];
        const uint64_t bb = (uint64_t)__double_as_longlong(bj);
        uint64_t Mb;
        int beb;
        fx_decode(bb, Mb, beb);
        const int shb = beb - 1075 - sc;
        if (((bb >> 52) & 0x7FF) != 0x7FF && shb <= 72) {
          __int128 Bj = (shb >= 0) ? ((__int128)Mb << shb) : (__int128)fx_round_shift(Mb, shb);
          if (bb >> 63) Bj = -Bj;
          const __int128 Rx = Bj - Sj;
          exact = true;
          neg = Rx < 0;
          const unsigned __int128 mag = neg ? (unsigned __int128)(-Rx) : (unsigned __int128)Rx;
          if (mag != 0) {
            Lx = bitlen_u128(mag);
            const unsigned __int128 N = mag << (128 - Lx);
            Nh = (uint64_t)(N >> 64);
            Ns = (uint64_t)N != 0;
            rj = fx_round53(Nh, Ns, neg, Lx - 1 + sc);
          }
        } else {
          rj = bj - scale2(i128_to_double(Sj), sc);
        }
        rbits = (uint64_t)__double_as_longlong(rj);
        const int ex = (int)((rbits >> 52) & 0x7FF);
        if (ex == 0x7FF) {
          bad = 1;
          exact = false;
        } else if (exact) {
          if (Lx) qj = Lx + sc + 1022 + ej;
        } else if (rj != 0.0) {
          qj = (ex ? ex : 1) + ej;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pfree[slot]);
      const int qmax = __reduce_max_sync(0xffffffffu, qj);
      // the running exponent after tile k - 1 (the other warp's)
      int Eprev = kNoExp;
      if (k >= 1) {
        const int kp = k - 1;
        ok = fx_wait(&s_eready[kp & 1], (kp >> 1) & 1, a.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicOr(a.status, LS_DEV_TIMEOUT);
          break;
        }
        Eprev = s_ecta[kp & 1];
      }
      const int Enew = max(Eprev, qmax);
      const int shift = (Eprev == kNoExp || Enew == kNoExp) ? 0 : Enew - Eprev;
      Ecta = Enew;
      __syncwarp();
      if (lane == 0) {
        s_ecta[k & 1] = Enew;          // tile k + 1 read s_ecta[(k - 1) & 1] before
        mbar_arrive(&s_eready[k & 1]);   // this warp could pass its own wait
      }
      if (lane < tr) {
        int64_t P = 0;
        if (qj != kNoExp && exact) {
          P = fx_round_norm(Nh, Ns, Lx + sc + ej + 1077 - Ecta);   // |P| <= 2^55 since qj <= Ecta
          if (neg) P = -P;
        } else if (qj != kNoExp) {
          uint64_t M;
          int be;
          fx_decode(rbits, M, be);
          P = fx_round_shift(M, qj - Ecta + 2);
          if (rbits >> 63) P = -P;
        }
        rslot[s * tr + lane] = fx_limbs(P);
      }
      if (lane == 0) rshift[s] = shift;
      __syncwarp();
      if (lane == 0) mbar_arrive(&rready[s]);
      // off the hand-off path: r_out and the squared norms
      if (lane < rows) {
        rn2 += rj * rj;
        if (a.r_prev) { const double dl = rj - rpj; dn2 += dl * dl; }
        if (a.r_out) a.r_out[row0 + lane] = rj;
      }
    }
    rn2 = warp_sum(rn2);
    dn2 = warp_sum(dn2);
    bad = __any_sync(0xffffffffu, bad);
    // warp 1 hands its sums to warp 0, which writes the CTA's partial (the
    // two epilogue warps meet at named barrier 1; both leave their loops)
    if (e == 1 && lane == 0) {
      s_esum[0] = rn2;
      s_esum[1] = dn2;
      s_eflag[0] = bad;
      s_eflag[1] = Ecta;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kFxEW * 32) : "memory");
    if (e == 0 && lane == 0) {
      out[2 * n] = (long long)max(Ecta, s_eflag[1]);
      out[2 * n + 1] = __double_as_longlong(rn2 + s_esum[0]);
      out[2 * n + 2] = __double_as_longlong(dn2 + s_esum[1]);
      out[2 * n + 3] = s_xbad | ((bad | s_eflag[0]) ? 2 : 0);
    }
    return;
  }

  // -------------------------------------------------------------- column group
  const int tc = tid - kFxRW * 32;
  constexpr int kCT = kFxCW * 32;
  int64_t T2[NPT2], TK[NPT2], T0[NPT2];          // Karatsuba sums, as in the row dots
  __int128 W[NPT2];
  // element offset of (row 0, column) in a stage.  Columns past n still read
  // inside the stage (the TMA zero-filled box columns, or the row's last
  // column when one box holds the row), so the loads need no branch; their
  // sums are never written out.
  int off[NPT2];
#pragma unroll
  for (int u = 0; u < NPT2; ++u) {
    T2[u] = 0; TK[u] = 0; T0[u] = 0; W[u] = 0;
    const int c = tc + kCT * u;
    off[u] = kBoxed ? 0 : min(c, boxw - 1);         // boxed rows: compile-time offsets below
  }
  int since = 0;
  auto fold = [&]() {
#pragma unroll
    for (int u = 0; u < NPT2; ++u) {
      W[u] += ((__int128)T2[u] << 28) + (__int128)(TK[u] - T2[u] - T0[u]) + (__int128)(T0[u] >> 28);
      T2[u] = 0; TK[u] = 0; T0[u] = 0;
    }
  };
  int k = 0;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
    const int s = k % S;
    bool ok = fx_wait(&full[s], (k / S) & 1, a.wait_ns);
    if (ok) ok = fx_wait(&rready[s], (k / S) & 1, a.wait_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(a.status, LS_DEV_TIMEOUT);
      break;
    }
    const int2* tl = tiles + (size_t)s * stage_elems;
    const int2* rs = rslot + s * tr;
    const int64_t row0 = (int64_t)t * tr;
    const int rows = (int)((a.m - row0 < (int64_t)tr) ? (a.m - row0) : (int64_t)tr);
    const int sh = rshift[s];
    if (sh > 0) {                      // a larger exponent arrived: realign the sums
      fold();
      since = 0;
#pragma unroll
      for (int u = 0; u < NPT2; ++u) W[u] = (sh >= 120) ? (__int128)0 : (W[u] >> sh);
    }
    // boxed rows: lane tc holds the column pairs 2 tc + 256 v (box v), so
    // one 16-byte load brings columns u = 2 v and 2 v + 1
    const int2* cb = tl + (kBoxed ? 2 * tc : 0);
    auto col_row = [&](int r) {
      const int2 pv = rs[r];
      const int ps = pv.x + pv.y;
      int2 av[NPT2];
      if (kBoxed) {
#pragma unroll
        for (int v = 0; v < NPT2 / 2; ++v) {
          const int4 pr = *reinterpret_cast<const int4*>(cb + r * 256 + v * (tr * 256));
          av[2 * v] = make_int2(pr.x, pr.y);
          av[2 * v + 1] = make_int2(pr.z, pr.w);
        }
      } else {
#pragma unroll
        for (int u = 0; u < NPT2; ++u) av[u] = tl[r * pitch + off[u]];
      }
#pragma unroll
      for (int u = 0; u < NPT2; ++u) {
        T2[u] = mad_wide(av[u].y, pv.y, T2[u]);
        TK[u] = mad_wide(av[u].x + av[u].y, ps, TK[u]);
        T0[u] = mad_wide(av[u].x, pv.x, T0[u]);
      }
    };
    if (rows == tr) {
#pragma unroll
      for (int r = 0; r < tr; ++r) col_row(r);
    } else {
      for (int r = 0; r < rows; ++r) col_row(r);
    }
    since += rows;
    if (since + tr > kFxFoldRows) { fold(); since = 0; }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&rfree[s]);
      mbar_arrive(&empty[s]);
    }
  }
  fold();
#pragma unroll
  for (int u = 0; u < NPT2; ++u) {
    const int c = kBoxed ? 2 * tc + 256 * (u >> 1) + (u & 1) : tc + kCT * u;
    if (c < n) {
      out[2 * c] = (long long)(unsigned long long)W[u];
      out[2 * c + 1] = (long long)(W[u] >> 64);
    }
  }
}

// Sum the per-CTA fixed-point partials exactly (aligned to the largest CTA
// exponent) and round once: c[k] = 2^(E - 2126) sum_p W_kp; the squared norms
// are FP64 sums over the CTAs in a fixed tree order.  One warp per output
// (k < n: c[k]; k = n, n + 1: the norms); the lanes take the CTAs p = lane,
// lane + 32, ...  The integer sums are exact, so their order does not matter.
// Writes c (n) and norms (2); a non-finite x or r in any CTA makes c and
// norms NaN.
__global__ void k_fx_reduce(const long long* __restrict__ part, int nparts, int n, double* __restrict__ c,
                            double* __restrict__ norms, const IterState* st) {
  if (st && st->done) return;
  const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (k >= n + 2) return;                             // whole warps leave together
  const size_t stride = 2 * (size_t)n + 4;
  int flags = 0;
  for (int p = lane; p < nparts; p += 32) flags |= (int)part[p * stride + 2 * n + 3];
  flags = (int)__reduce_or_sync(0xffffffffu, (unsigned)flags);
  if (k >= n) {
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += __longlong_as_double(part[p * stride + 2 * n + 1 + (k - n)]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[k - n] = flags ? __longlong_as_double(0x7FF8000000000000ll) : s;
    return;
  }
  int E = kNoExp;
  for (int p = lane; p < nparts; p += 32) E = max(E, (int)part[p * stride + 2 * n]);
  E = __reduce_max_sync(0xffffffffu, E);
  __int128 sum = 0;
  if (E != kNoExp) {
    for (int p = lane; p < nparts; p += 32) {
      const int Ep = (int)part[p * stride + 2 * n];
      if (Ep == kNoExp) continue;
      const int sh = E - Ep;
      if (sh >= 120) continue;
      const __int128 w = ((__int128)part[p * stride + 2 * k + 1] << 64) |
                         (__int128)(unsigned long long)part[p * stride + 2 * k];
      sum += w >> sh;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += shfl_xor_i128(sum, o);
  }
  if (lane == 0) {
    double v = (E == kNoExp) ? 0.0 : scale2(i128_to_double(sum), E - 2126);
    if (flags) v = __longlong_as_double(0x7FF8000000000000ll);
    c[k] = v;
  }
}

// ------------------------------------------------------------------ host side
FxGeom fx_geometry(const ls_ctx* ctx, int64_t n, int64_t m) {
  FxGeom g;
  if (n <= 256) {
    g.boxw = (int)((n + 1) & ~1LL);
    g.nbox = 1;
    g.tr = 32;
  } else {
    g.boxw = 256;
    g.nbox = (int)((n + 255) / 256);
    g.tr = (g.nbox <= 2) ? 16 : 8;
  }
  const size_t stage = (size_t)g.tr * g.nbox * g.boxw * sizeof(int2);
  {
    // as many stages as fit beside the fixed parts (p1, xs, per-stage slots
    // and barriers; at most 8), within the 227 KB a CTA may use
    const size_t xl = (g.nbox > 1) ? (size_t)g.nbox * 256 : (size_t)n;
    const size_t fixed = (size_t)2 * kFxRW * g.tr * 16 + xl * 16 + 4 * 8 + 128 + 1024;
    const size_t per_stage = stage + (size_t)g.tr * 8 + 4 + 4 * 8;
    const size_t room = (227 * 1024 > fixed) ? (227 * 1024 - fixed) : 0;
    g.stages = (int)std::max<size_t>(2, std::min<size_t>(8, room / per_stage));
  }
  const int64_t ntiles = (m + g.tr - 1) / g.tr;
  g.grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms, ntiles));
  const size_t xlen = (g.nbox > 1) ? (size_t)g.nbox * 256 : (size_t)n;
  g.smem = g.stages * stage + (size_t)2 * kFxRW * g.tr * 16 + xlen * 16 +
           (size_t)g.stages * g.tr * 8 + (size_t)((g.stages + 1) & ~1) * 4 + (4 * (size_t)g.stages + 4) * 8 + 128;
  return g;
}

size_t fx_part_words(const FxGeom& g, int64_t n) { return (size_t)g.grid * (2 * (size_t)n + 4); }

cudaError_t launch_to_fixed(ls_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, int2* Af, int64_t ldf,
                            int* rexp) {
  const int64_t blocks = (m + 7) / 8;
  k_to_fixed<<<(unsigned)blocks, 256, 0, ctx->stream>>>(A, m, (int)n, lda, Af, ldf, rexp, ctx->d_status);
  ++ctx->launches;
  return cudaGetLastError();
}

typedef CUresult (*FxEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t make_fx_tensor_map(ls_ctx* ctx, CUtensorMap* map, const int2* Af, int64_t m, int64_t n, int64_t ldf,
                               const FxGeom& g) {
  if (!ctx->encode_tiled) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    ctx->encode_tiled = fn;
  }
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)ldf * sizeof(int2)};
  cuuint32_t box[2] = {(cuuint32_t)g.boxw, (cuuint32_t)g.tr};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ((FxEncodeTiledFn)ctx->encode_tiled)(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, (void*)Af, dims, strides,
                                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int NPT2>
static cudaError_t launch_fx_t(ls_ctx* ctx, const CUtensorMap& map, const FxGeom& g, const FxArgs& a) {
  if (g.tr != fx_tile_rows(NPT2) || (g.nbox > 1) != (NPT2 >= 4) ||
      (g.nbox > 1 && (g.boxw != 256 || NPT2 * 128 > g.nbox * 256)))
    return cudaErrorInvalidValue;                   // the kernel's compile-time tile shape
  cudaError_t e = cudaFuncSetAttribute(k_fx_pass<NPT2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  k_fx_pass<NPT2><<<g.grid, kFxThreads, g.smem, ctx->stream>>>(map, a);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_fx_pass(ls_ctx* ctx, const CUtensorMap& map, const FxGeom& g, int64_t m, int64_t n,
                           const int* rexp, const double* b, const double* x, const double* r_prev, double* r_out,
                           long long* part, const IterState* st) {
  FxArgs a;
  a.m = m; a.n = (int)n; a.boxw = g.boxw; a.nbox = g.nbox; a.tr = g.tr; a.stages = g.stages;
  a.ntiles = (int)((m + g.tr - 1) / g.tr);
  a.rexp = rexp; a.b = b; a.x = x; a.r_prev = r_prev; a.r_out = r_out; a.part = part; a.st = st;
  a.status = ctx->d_status;
  a.wait_ns = ctx->wait_ns;
  a.inject_skip = ctx->inject_skip_tile;
  ctx->inject_skip_tile = -1;                       // one-shot
  const int npt2 = (int)((n + 127) / 128);          // the instantiation NPT2 >= ceil(n / 128)
  if (npt2 <= 1) return launch_fx_t<1>(ctx, map, g, a);
  if (npt2 <= 2) return launch_fx_t<2>(ctx, map, g, a);
  if (npt2 <= 4) return launch_fx_t<4>(ctx, map, g, a);
  if (npt2 <= 6) return launch_fx_t<6>(ctx, map, g, a);
  if (npt2 <= 8) return launch_fx_t<8>(ctx, map, g, a);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fx_reduce(ls_ctx* ctx, const long long* part, int nparts, int64_t n, double* c, double* norms,
                             const IterState* st) {
  const int threads = 256;                          // eight outputs per block, a warp each
  const int grid = (int)((n + 2 + 7) / 8);
  k_fx_reduce<<<grid, threads, 0, ctx->stream>>>(part, nparts, (int)n, c, norms, st);
  ++ctx->launches;
  return cudaGetLastError();
}

}  // namespace lsk
